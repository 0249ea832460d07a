// C ABI of the STEV integrator: mechanism staging, launch configuration and
// the solve entry points declared in include/stev.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/stev.h"
#include "stev_device.cuh"
#include "stev_internal.h"
#include "stev_fp64.cuh"
#include "stev_mixed.cuh"
#include "stev_mlp.cuh"

using namespace stev;

// ----------------------------------------------------------------- errors
static thread_local std::string g_err;

namespace stev {
namespace host {
stev_status fail(stev_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}
void clear_error() { g_err.clear(); }
}  // namespace host
}  // namespace stev
using stev::host::fail;

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? STEV_ENOMEM : STEV_ECUDA,            \
                  "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

// -------------------------------------------------------------- mechanism
struct stev_mechanism {
  int device = 0;
  int S = 0, R = 0, Rrev = 0, n_gather = 0;
  stev_options opt{};
  int n_hi_bins = 0;
  double* d_sp = nullptr;
  double* d_rx = nullptr;
  int4* d_ri = nullptr;
  int4* d_rim = nullptr;  // the mixed kernels' copy (unused slot = S)
  int* d_gptr = nullptr;
  int* d_gent = nullptr;
  double* d_tw = nullptr;
  float* d_spf = nullptr;  // float tables of the mixed kernel
  float4* d_rxf = nullptr;
  float* d_twf = nullptr;
  // launch configuration of the persistent kernel
  int G = 32;              // lanes per cell
  int block = 0, grid = 0; // threads per CTA, CTAs
  int per_sm = 0, sms = 0;  // resident CTAs per SM, SMs
  int cells = 0;            // resident cells per CTA
  unsigned long long* d_net_stalls = nullptr;  // network answers that timed out
  // general rate laws (real stoichiometry / orders)
  int general = 0;
  double* d_rg = nullptr;
  double* d_gnu = nullptr;
  float* d_rgf = nullptr;
  float* d_gnuf = nullptr;
  size_t smem = 0;
  long long nslots = 0;    // cells resident at once
  unsigned long long* d_counter = nullptr;
  // device copies for the host-pointer entry point
  double *d_hT = nullptr, *d_hP = nullptr, *d_hY = nullptr, *d_hTo = nullptr, *d_hYo = nullptr;
  int* d_hit = nullptr;
  unsigned char* d_hst = nullptr;
  long long host_cap = 0;
  // batch descriptors of stev_solve_batched: [cap] BatchDesc + [cap+1] offsets
  BatchDesc* d_bdesc = nullptr;
  long long* d_boff = nullptr;
  int batch_cap = 0;
  // thermo network (Sec. 3)
  int mlp_out = 0, mlp_out_pad = 0, mlp_np = 0;
  float* d_mlp_params = nullptr;          // FP32 master parameters
  __nv_bfloat16* d_mlp_W2 = nullptr;      // [64][64]
  __nv_bfloat16* d_mlp_W3 = nullptr;      // [out_pad][64]
  float* d_mlp_misc = nullptr;            // W1, b1, b2 [64 each], b3, mean, std [out_pad each]
  unsigned char* d_mlp_frag = nullptr;    // the network in MMA fragment order (MlpFrag)
  bool mlp_ready = false;
  // the solver kernel: the generic instantiation, or one compiled for this
  // mechanism (options.specialize)
  const void* kfn = nullptr;
  cudaLibrary_t spec_lib = nullptr;
  cudaKernel_t spec_k = nullptr;
  stev::host::SpecKey spec_key{};
};

extern "C" void stev_default_options(stev_options* o) {
  if (!o) return;
  o->y_step_max = 1e-3;
  o->delta_max = 0.01;
  o->alpha = 1e-5;
  o->dft_n = 13;
  o->dft_hi_first = 4;
  o->tol_ring = 0.5;
  o->tol_freq = 1e-6;
  o->r_fac = 2.0;
  o->rof_min = 1e-30;
  o->max_iters = 200000;
  o->precision = STEV_FP64;
  o->thermo = STEV_THERMO_POLY;
  o->dft_on = 1;
  o->lanes_per_cell = 0;
  o->specialize = 0;
}

static stev_status check_options(const stev_options* o) {
  if (!(o->y_step_max > 0.0) || !std::isfinite(o->y_step_max))
    return fail(STEV_EINVAL, "y_step_max must be finite and > 0");
  if (!(o->delta_max > 0.0 && o->delta_max <= 1.0)) return fail(STEV_EINVAL, "delta_max must be in (0, 1]");
  if (!(o->alpha >= 0.0) || !std::isfinite(o->alpha)) return fail(STEV_EINVAL, "alpha must be finite and >= 0");
  if (o->dft_n < 2 || o->dft_n > kMaxDftN) return fail(STEV_EINVAL, "dft_n must be in [2, %d]", kMaxDftN);
  if (o->dft_hi_first < 1 || o->dft_hi_first > o->dft_n / 2)
    return fail(STEV_EINVAL, "dft_hi_first must be in [1, dft_n/2]");
  if (!(o->r_fac > 0.0) || !std::isfinite(o->r_fac)) return fail(STEV_EINVAL, "r_fac must be finite and > 0");
  if (!std::isfinite(o->tol_ring) || !std::isfinite(o->tol_freq)) return fail(STEV_EINVAL, "tolerances must be finite");
  if (!(o->rof_min > 0.0 && o->rof_min <= 1.0)) return fail(STEV_EINVAL, "rof_min must be in (0, 1]");
  if (o->max_iters < 1) return fail(STEV_EINVAL, "max_iters must be >= 1");
  if (o->precision != STEV_FP64 && o->precision != STEV_MIXED) return fail(STEV_EINVAL, "unknown precision");
  if (o->thermo != STEV_THERMO_POLY && o->thermo != STEV_THERMO_MLP && o->thermo != STEV_THERMO_MLP_CPH)
    return fail(STEV_EINVAL, "unknown thermo mode");
  if (o->lanes_per_cell != 0 && o->lanes_per_cell != 8 && o->lanes_per_cell != 16 &&
      o->lanes_per_cell != 32)
    return fail(STEV_EINVAL, "lanes_per_cell must be 0, 8, 16 or 32");
  if (o->thermo != STEV_THERMO_POLY && o->precision != STEV_MIXED)
    return fail(STEV_EINVAL, "the thermo network is used by the mixed-precision path only");
  if (o->specialize != 0 && o->specialize != 1) return fail(STEV_EINVAL, "specialize must be 0 or 1");
  return STEV_OK;
}

static void free_mech(stev_mechanism* m) {
  void* ptrs[] = {m->d_sp, m->d_rx, m->d_ri, m->d_rim, m->d_gptr, m->d_gent, m->d_tw, m->d_spf, m->d_rxf,
                  m->d_twf, m->d_counter, m->d_mlp_params, m->d_mlp_W2, m->d_mlp_W3, m->d_mlp_misc,
                  m->d_mlp_frag,
                  m->d_bdesc, m->d_boff, m->d_net_stalls, m->d_rg, m->d_gnu, m->d_rgf, m->d_gnuf,
                  m->d_hT, m->d_hP, m->d_hY, m->d_hTo, m->d_hYo, m->d_hit, m->d_hst};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (m->spec_lib) cudaLibraryUnload(m->spec_lib);
  delete m;
}

typedef void (*KernelFn)(Launch);

// The mixed kernels come with the DFT window fixed at the paper's N = 13
// (taps unrolled) and for any other N.
static KernelFn select_kernel(int precision, int G, int thermo, int dft_n) {
  if (precision == STEV_MIXED) {
    const bool n13 = dft_n == 13;
    if (thermo != STEV_THERMO_POLY) {
      switch (G) {
        case 8: return n13 ? stev_mixed_net_kernel<8, 13> : stev_mixed_net_kernel<8, 0>;
        case 16: return n13 ? stev_mixed_net_kernel<16, 13> : stev_mixed_net_kernel<16, 0>;
        default: return n13 ? stev_mixed_net_kernel<32, 13> : stev_mixed_net_kernel<32, 0>;
      }
    }
    switch (G) {
      case 8: return n13 ? stev_mixed_kernel<8, 13> : stev_mixed_kernel<8, 0>;
      case 16: return n13 ? stev_mixed_kernel<16, 13> : stev_mixed_kernel<16, 0>;
      default: return n13 ? stev_mixed_kernel<32, 13> : stev_mixed_kernel<32, 0>;
    }
  }
  switch (G) {
    case 8: return stev_fp64_kernel<8>;
    case 16: return stev_fp64_kernel<16>;
    default: return stev_fp64_kernel<32>;
  }
}

// Lanes per cell.  Per-cell scalar work (log T, 1/T, h, t_rem) is one warp
// instruction whatever the group size, so more cells per warp amortise it;
// fewer lanes per cell lengthen each cell's step (the tail of the variable
// load).  FP64: cover the species and most reactions in one or two rounds.
static int choose_group(int S, int R, const stev_options& o) {
  if (o.lanes_per_cell) return o.lanes_per_cell;
  if (S <= 8 && R <= 32) return 8;
  if (S <= 16 && R <= 64) return 16;
  return 32;
}

// Launch configuration of the persistent kernel: as many resident cells per
// CTA as shared memory holds (whole warps, <= the block limit), then as many
// CTAs as fit on every SM.  Atomic: on failure the mechanism keeps its
// previous configuration and kernel.
static stev_status configure(stev_mechanism* m) {
  cudaDeviceProp prop;
  CUDA_TRY(cudaGetDeviceProperties(&prop, m->device));
  const int G = choose_group(m->S, m->R, m->opt);
  const bool mixed = m->opt.precision == STEV_MIXED;
  const size_t tables =
      mixed ? table_smem_bytes_mixed(m->S, m->R, m->n_gather, m->n_hi_bins, m->opt.dft_n, m->general)
            : table_smem_bytes(m->S, m->R, m->n_gather, m->n_hi_bins, m->opt.dft_n, m->general);
  const bool net = m->opt.thermo != STEV_THERMO_POLY;
  const size_t cell = mixed ? cell_smem_bytes_mixed(m->S, m->R, m->Rrev, m->opt.dft_n, net)
                            : cell_smem_bytes_fp64(m->S, m->R, m->Rrev, m->opt.dft_n);
  const size_t limit = prop.sharedMemPerBlockOptin;
  const size_t per_cell = cell;
  const int max_cells = (mixed ? kMaxBlockMixed : kMaxBlock) / G;
  if (tables + per_cell > limit) return fail(STEV_EINVAL, "mechanism does not fit in shared memory");
  int cells = (int)((limit - tables) / per_cell);
  cells = std::min(cells, max_cells);
  const int per_warp = 32 / G;
  cells = (cells / per_warp) * per_warp;
  if (cells < per_warp) return fail(STEV_EINVAL, "mechanism too large for one warp per CTA");
  size_t smem = tables + (size_t)cells * per_cell;
  int block = cells * G;
  const void* k = reinterpret_cast<const void*>(select_kernel(m->opt.precision, G, m->opt.thermo,
                                                              m->opt.dft_n));
  // a kernel compiled for this mechanism: reused if its key is unchanged; a
  // new one replaces the old only once the whole configuration succeeded
  cudaLibrary_t new_lib = nullptr;
  cudaKernel_t new_k = nullptr;
  const stev::host::SpecKey key{m->S, m->R, m->Rrev, m->general, G, m->opt.dft_n == 13 ? 13 : 0,
                                net ? 1 : 0};
  if (mixed && m->opt.specialize) {
    if (m->spec_k && key == m->spec_key) {
      k = reinterpret_cast<const void*>(m->spec_k);
    } else {
      const stev_status st = stev::host::spec_load(key, &new_lib, &new_k);
      if (st != STEV_OK) return st;
      k = reinterpret_cast<const void*>(new_k);
    }
  }
  auto drop_new = [&]() {
    if (new_lib) cudaLibraryUnload(new_lib);
  };
  // a kernel compiled with a smaller launch bound than the block chosen above
  // holds fewer cells per CTA
  {
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, k) == cudaSuccess && fa.maxThreadsPerBlock > 0 &&
        block > fa.maxThreadsPerBlock) {
      cells = (fa.maxThreadsPerBlock / G) / per_warp * per_warp;
      if (cells < per_warp) {
        drop_new();
        return fail(STEV_EINVAL, "solver kernel's block limit is below one warp");
      }
      smem = tables + (size_t)cells * per_cell;
      block = cells * G;
    }
  }
  int per_sm = 0;
  // The attribute belongs to the kernel function, which mechanisms with the
  // same precision, lane group and thermo share: set it to the device's cap
  // (a ceiling, not a reservation), so that configuring a smaller mechanism
  // never lowers it below what an earlier, larger one launches with.
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
  if (e != cudaSuccess) {
    drop_new();
    return fail(STEV_ECUDA, "configuring the solver kernel: %s", cudaGetErrorString(e));
  }
  if (per_sm < 1) {
    drop_new();
    return fail(STEV_EINVAL, "persistent kernel cannot be resident");
  }
  if (!m->d_counter) {
    e = cudaMalloc(&m->d_counter, sizeof(unsigned long long));
    if (e != cudaSuccess) {
      drop_new();
      return fail(STEV_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
  }
  if (!m->d_net_stalls) {
    e = cudaMalloc(&m->d_net_stalls, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(m->d_net_stalls, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) {
      drop_new();
      return fail(STEV_ENOMEM, "cudaMalloc: %s", cudaGetErrorString(e));
    }
  }
  // commit
  if (new_lib) {
    if (m->spec_lib) cudaLibraryUnload(m->spec_lib);
    m->spec_lib = new_lib;
    m->spec_k = new_k;
    m->spec_key = key;
  }
  m->kfn = k;
  m->G = G;
  m->block = block;
  m->cells = cells;
  m->per_sm = per_sm;
  m->sms = prop.multiProcessorCount;
  m->grid = per_sm * prop.multiProcessorCount;
  m->smem = smem;
  m->nslots = (long long)m->grid * cells;
  return STEV_OK;
}

extern "C" stev_status stev_mechanism_create(int S, int R, const double* W, const double* nasa7,
                                             const double* t_range, const int* rxn_ptr,
                                             const int* rxn_species, const double* rxn_nu,
                                             const double* A, const double* beta, const double* Ea,
                                             const unsigned char* reversible,
                                             const stev_options* opt, stev_mechanism** out) {
  g_err.clear();
  if (out) *out = nullptr;
  if (rxn_ptr && rxn_nu && R >= 1 && R <= kMaxReactions && rxn_ptr[0] == 0) {
    for (int k = 0; k < rxn_ptr[R]; ++k) {
      const double a = std::fabs(rxn_nu[k]);
      if (!(a == 1.0 || a == 2.0))
        return fail(STEV_EINVAL, "rxn_nu[%d]: only elementary orders |nu| in {1,2} are supported "
                    "(global rate laws: stev_mechanism_create_orders)", k);
    }
  }
  return stev_mechanism_create_orders(S, R, W, nasa7, t_range, rxn_ptr, rxn_species, rxn_nu,
                                      nullptr, A, beta, Ea, reversible, opt, out);
}

extern "C" stev_status stev_mechanism_create_orders(
    int S, int R, const double* W, const double* nasa7, const double* t_range,
    const int* rxn_ptr, const int* rxn_species, const double* rxn_nu, const double* rxn_order,
    const double* A, const double* beta, const double* Ea, const unsigned char* reversible,
    const stev_options* opt, stev_mechanism** out) {
  g_err.clear();
  if (!out) return fail(STEV_EINVAL, "out is NULL");
  *out = nullptr;
  if (S < 1 || S > kMaxSpecies) return fail(STEV_EINVAL, "n_species must be in [1, %d]", kMaxSpecies);
  if (R < 1 || R > kMaxReactions) return fail(STEV_EINVAL, "n_reactions must be in [1, %d]", kMaxReactions);
  if (!W || !nasa7 || !t_range || !rxn_ptr || !rxn_species || !rxn_nu || !A || !beta || !Ea || !reversible)
    return fail(STEV_EINVAL, "NULL table pointer");
  stev_options o;
  if (opt) o = *opt; else stev_default_options(&o);
  stev_status st = check_options(&o);
  if (st != STEV_OK) return st;

  // species tables
  std::vector<double> sp((size_t)S * SP_STRIDE, 0.0);
  for (int i = 0; i < S; ++i) {
    if (!(W[i] > 0.0) || !std::isfinite(W[i])) return fail(STEV_EINVAL, "mol_weight[%d] must be finite and > 0", i);
    double* e = &sp[(size_t)i * SP_STRIDE];
    e[SP_W] = W[i];
    e[SP_INVW] = 1.0 / W[i];
    e[SP_TSPLIT] = t_range[3 * i + 1];
    if (!std::isfinite(e[SP_TSPLIT])) return fail(STEV_EINVAL, "t_range[%d] not finite", i);
    for (int rg = 0; rg < 2; ++rg) {
      const double* a = nasa7 + ((size_t)i * 2 + rg) * 7;
      for (int k = 0; k < 7; ++k)
        if (!std::isfinite(a[k])) return fail(STEV_EINVAL, "nasa7[%d][%d][%d] not finite", i, rg, k);
      double* b = e + (rg == 0 ? SP_LOW : SP_HIGH);
      for (int k = 0; k < 7; ++k) b[B_A0 + k] = a[k];
      b[B_H1] = a[1] / 2.0;
      b[B_H2] = a[2] / 3.0;
      b[B_H3] = a[3] / 4.0;
      b[B_H4] = a[4] / 5.0;
      b[B_G2] = a[2] / 6.0;
      b[B_G3] = a[3] / 12.0;
      b[B_G4] = a[4] / 20.0;
    }
  }

  // reaction tables.  Elementary mass action (every |nu| in {1, 2}, orders =
  // |nu|) packs each molecule into a slot; otherwise the mechanism is
  // "general": slots hold distinct species with their real nu and order.
  if (rxn_ptr[0] != 0) return fail(STEV_EINVAL, "rxn_ptr[0] must be 0");
  int general = 0;
  for (int k = 0; k < rxn_ptr[R]; ++k) {
    const double nu = rxn_nu[k];
    if (!std::isfinite(nu) || nu == 0.0) return fail(STEV_EINVAL, "rxn_nu[%d] must be finite and nonzero", k);
    if (rxn_order && (!(rxn_order[k] > 0.0) || !std::isfinite(rxn_order[k])))
      return fail(STEV_EINVAL, "rxn_order[%d] must be finite and > 0", k);
    if (!(std::fabs(nu) == 1.0 || std::fabs(nu) == 2.0)) general = 1;
    if (rxn_order && rxn_order[k] != std::fabs(nu)) general = 1;
  }
  std::vector<double> rx((size_t)R * RX_STRIDE, 0.0);
  std::vector<int4> ri(R);
  std::vector<double> rg((size_t)R * 8, 0.0);
  int nrev = 0;
  for (int r = 0; r < R; ++r) {
    const int lo = rxn_ptr[r], hi = rxn_ptr[r + 1];
    if (hi <= lo || hi - lo > 4) return fail(STEV_EINVAL, "reaction %d: bad rxn_ptr range", r);
    int reac[2], prod[2], nr = 0, np = 0;
    double bal = 0.0, mag = 0.0, dN = 0.0;
    for (int k = lo; k < hi; ++k) {
      const int s = rxn_species[k];
      const double nu = rxn_nu[k];
      if (s < 0 || s >= S) return fail(STEV_EINVAL, "reaction %d: species index %d out of range", r, s);
      for (int k2 = lo; k2 < k; ++k2)
        if (rxn_species[k2] == s) return fail(STEV_EINVAL, "reaction %d: species %d listed twice", r, s);
      if (general) {
        const double ord = rxn_order ? rxn_order[k] : std::fabs(nu);
        if (nu < 0) {
          if (nr == 2) return fail(STEV_EINVAL, "reaction %d: more than two reactant species", r);
          rg[(size_t)r * 8 + nr] = nu;
          rg[(size_t)r * 8 + 4 + nr] = ord;
          reac[nr++] = s;
        } else {
          if (np == 2) return fail(STEV_EINVAL, "reaction %d: more than two product species", r);
          rg[(size_t)r * 8 + 2 + np] = nu;
          rg[(size_t)r * 8 + 6 + np] = ord;
          prod[np++] = s;
        }
      } else {
        const int mult = (int)std::fabs(nu);
        for (int t = 0; t < mult; ++t) {
          if (nu < 0) { if (nr == 2) return fail(STEV_EINVAL, "reaction %d: more than two reactant molecules", r); reac[nr++] = s; }
          else        { if (np == 2) return fail(STEV_EINVAL, "reaction %d: more than two product molecules", r); prod[np++] = s; }
        }
      }
      bal += nu * W[s];
      mag += std::fabs(nu * W[s]);
      dN += nu;
    }
    if (nr == 0 || np == 0) return fail(STEV_EINVAL, "reaction %d needs reactants and products", r);
    if (std::fabs(bal) > 1e-12 * mag) return fail(STEV_EUNBALANCED, "reaction %d is not mass-balanced", r);
    if (!(A[r] >= 0.0) || !std::isfinite(A[r])) return fail(STEV_EINVAL, "A[%d] must be finite and >= 0", r);
    if (!std::isfinite(beta[r]) || !std::isfinite(Ea[r])) return fail(STEV_EINVAL, "beta/Ea[%d] not finite", r);
    double* e = &rx[(size_t)r * RX_STRIDE];
    e[RX_LNA] = std::log(A[r]);
    e[RX_BETA] = beta[r];
    e[RX_EAR] = Ea[r] / kRu;
    e[RX_DN] = general ? dN : (double)(np - nr);
    const int a0 = reac[0], a1 = nr > 1 ? reac[1] : kNone;
    const int p0 = prod[0], p1 = np > 1 ? prod[1] : kNone;
    ri[r].x = a0 | (a1 << 8) | (p0 << 16) | (p1 << 24);
    ri[r].y = np - nr;
    ri[r].z = reversible[r] ? 1 : 0;
    ri[r].w = reversible[r] ? nrev++ : -1;
  }

  // species-major gather lists in ascending reaction order (general rate
  // laws keep each entry's real nu beside it)
  std::vector<int> gptr(S + 1, 0), gent;
  std::vector<double> gnu;
  for (int i = 0; i < S; ++i) {
    for (int r = 0; r < R; ++r)
      for (int k = rxn_ptr[r]; k < rxn_ptr[r + 1]; ++k)
        if (rxn_species[k] == i) {
          gent.push_back(gather_pack(r, general ? 0 : (int)rxn_nu[k]));
          gnu.push_back(rxn_nu[k]);
        }
    gptr[i + 1] = (int)gent.size();
  }

  stev_mechanism* m = new stev_mechanism();
  m->S = S;
  m->R = R;
  m->Rrev = nrev;
  m->n_gather = (int)gent.size();
  m->general = general;
  m->opt = o;
  if (cudaGetDevice(&m->device) != cudaSuccess) { delete m; return fail(STEV_ECUDA, "no CUDA device"); }
  m->n_hi_bins = o.dft_n / 2 - o.dft_hi_first + 1;
  std::vector<double> tw((size_t)m->n_hi_bins * 2 * o.dft_n);
  for (int b = 0; b < m->n_hi_bins; ++b) {
    const int j = o.dft_hi_first + b;
    for (int k = 0; k < o.dft_n; ++k) {
      const double ang = -2.0 * M_PI * (double)j * (double)k / (double)o.dft_n;
      tw[(size_t)b * 2 * o.dft_n + k] = std::cos(ang);
      tw[(size_t)b * 2 * o.dft_n + o.dft_n + k] = std::sin(ang);
    }
  }
#define TRY_OR_FREE(expr)            \
  do {                               \
    stev_status s_ = (expr);         \
    if (s_ != STEV_OK) {             \
      free_mech(m);                  \
      return s_;                     \
    }                                \
  } while (0)
  auto upload = [&](void** dst, const void* src, size_t bytes) -> stev_status {
    CUDA_TRY(cudaMalloc(dst, bytes ? bytes : 16));
    if (bytes) CUDA_TRY(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    return STEV_OK;
  };
  TRY_OR_FREE(upload((void**)&m->d_sp, sp.data(), sp.size() * sizeof(double)));
  TRY_OR_FREE(upload((void**)&m->d_rx, rx.data(), rx.size() * sizeof(double)));
  TRY_OR_FREE(upload((void**)&m->d_ri, ri.data(), ri.size() * sizeof(int4)));
  std::vector<int4> rim(ri);
  for (int4& v : rim) {
    int x = 0;
    for (int k = 0; k < 4; ++k) {
      const int sl = (v.x >> (8 * k)) & 0xFF;
      x |= (sl == kNone ? S : sl) << (8 * k);
    }
    v.x = x;
  }
  TRY_OR_FREE(upload((void**)&m->d_rim, rim.data(), rim.size() * sizeof(int4)));
  TRY_OR_FREE(upload((void**)&m->d_tw, tw.data(), tw.size() * sizeof(double)));
  // float tables of the mixed kernel (log2 space for the MUFU exponentials),
  // coefficient-major: row k of species i at [k * S + i]
  std::vector<float> spf((size_t)SF_ROWS * S, 0.0f);
  auto put = [&](int row, int i, double v) { spf[(size_t)row * S + i] = (float)v; };
  auto put_pair = [&](int row, int i, double v) {  // hi row, then lo row
    const float h = (float)v;
    spf[(size_t)row * S + i] = h;
    spf[(size_t)(row + 1) * S + i] = (float)(v - (double)h);
  };
  const double ln_pref = std::log(kPatm / kRu);
  for (int i = 0; i < S; ++i) {
    const double* e = &sp[(size_t)i * SP_STRIDE];
    put(SF_W, i, e[SP_W]);
    put(SF_INVW, i, e[SP_INVW]);
    put_pair(SF_SPLIT_H, i, e[SP_TSPLIT]);
    for (int rg = 0; rg < 2; ++rg) {
      const double* b = e + (rg == 0 ? SP_LOW : SP_HIGH);
      const int fb = rg == 0 ? SF_LOW : SF_HIGH;
      for (int k = 0; k < 6; ++k) put(fb + BF_A0 + k, i, b[B_A0 + k]);
      put(fb + BF_H1, i, b[B_H1]);
      put(fb + BF_H2, i, b[B_H2]);
      put(fb + BF_H3, i, b[B_H3]);
      put(fb + BF_H4, i, b[B_H4]);
      // g2 = log2 e (G/RT - ln(P_atm/R_u) + ln T) over the basis
      // 1, ln T, 1/T, T, T^2, T^3, T^4 (G/RT of Eq. 16's NASA-7 form)
      const double c[7] = {kLog2e * (b[B_A0] - b[B_A6] - ln_pref), kLog2e * (1.0 - b[B_A0]),
                           kLog2e * b[B_A5], -kLog2e * b[B_H1], -kLog2e * b[B_G2],
                           -kLog2e * b[B_G3], -kLog2e * b[B_G4]};
      const int gb = rg == 0 ? SF_GLOW : SF_GHIGH;
      for (int k = 0; k < 7; ++k) put_pair(gb + 2 * k, i, c[k]);
    }
  }
  std::vector<float4> rxf(R);
  for (int r = 0; r < R; ++r) {
    const double* e = &rx[(size_t)r * RX_STRIDE];
    rxf[r] = make_float4((float)(e[RX_LNA] * kLog2e), (float)e[RX_BETA],
                         (float)(e[RX_EAR] * kLog2e), (float)e[RX_DN]);
  }
  std::vector<float> twf(tw.begin(), tw.end());
  TRY_OR_FREE(upload((void**)&m->d_spf, spf.data(), spf.size() * sizeof(float)));
  TRY_OR_FREE(upload((void**)&m->d_rxf, rxf.data(), rxf.size() * sizeof(float4)));
  TRY_OR_FREE(upload((void**)&m->d_twf, twf.data(), twf.size() * sizeof(float)));
  TRY_OR_FREE(upload((void**)&m->d_gptr, gptr.data(), gptr.size() * sizeof(int)));
  TRY_OR_FREE(upload((void**)&m->d_gent, gent.data(), gent.size() * sizeof(int)));
  if (general) {
    std::vector<float> rgf(rg.begin(), rg.end()), gnuf(gnu.begin(), gnu.end());
    TRY_OR_FREE(upload((void**)&m->d_rg, rg.data(), rg.size() * sizeof(double)));
    TRY_OR_FREE(upload((void**)&m->d_gnu, gnu.data(), gnu.size() * sizeof(double)));
    TRY_OR_FREE(upload((void**)&m->d_rgf, rgf.data(), rgf.size() * sizeof(float)));
    TRY_OR_FREE(upload((void**)&m->d_gnuf, gnuf.data(), gnuf.size() * sizeof(float)));
  }
  TRY_OR_FREE(configure(m));
  *out = m;
  return STEV_OK;
}

// The DFT twiddles of the high bins for window N and first high bin n
// (Eq. 9), in FP64 and FP32.  On failure the mechanism has none (kfn cleared:
// no solve runs until options are set successfully).
static stev_status upload_twiddles(stev_mechanism* m, int N, int hi_first) {
  const int nb = N / 2 - hi_first + 1;
  std::vector<double> tw((size_t)nb * 2 * N);
  for (int b = 0; b < nb; ++b) {
    const int j = hi_first + b;
    for (int k = 0; k < N; ++k) {
      const double ang = -2.0 * M_PI * (double)j * (double)k / (double)N;
      tw[(size_t)b * 2 * N + k] = std::cos(ang);
      tw[(size_t)b * 2 * N + N + k] = std::sin(ang);
    }
  }
  std::vector<float> twf(tw.begin(), tw.end());
  CUDA_TRY(cudaDeviceSynchronize());
  if (m->d_tw) cudaFree(m->d_tw);
  if (m->d_twf) cudaFree(m->d_twf);
  m->d_tw = nullptr;
  m->d_twf = nullptr;
  cudaError_t e = cudaMalloc(&m->d_tw, tw.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(m->d_tw, tw.data(), tw.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&m->d_twf, twf.size() * sizeof(float));
  if (e == cudaSuccess)
    e = cudaMemcpy(m->d_twf, twf.data(), twf.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    m->kfn = nullptr;
    return fail(STEV_ECUDA, "twiddle table: %s", cudaGetErrorString(e));
  }
  m->n_hi_bins = nb;
  return STEV_OK;
}

// New options take effect only if the kernel configuration for them
// succeeds; otherwise the previous options, tables and kernel stay.
extern "C" stev_status stev_mechanism_set_options(stev_mechanism* m, const stev_options* opt) {
  g_err.clear();
  if (!m || !opt) return fail(STEV_EINVAL, "NULL argument");
  stev_status st = check_options(opt);
  if (st != STEV_OK) return st;
  const stev_options old = m->opt;
  const bool tw_change = opt->dft_n != old.dft_n || opt->dft_hi_first != old.dft_hi_first;
  if (tw_change) {
    st = upload_twiddles(m, opt->dft_n, opt->dft_hi_first);
    if (st != STEV_OK) return st;
  }
  m->opt = *opt;
  st = configure(m);
  if (st == STEV_OK) return STEV_OK;
  const std::string msg = g_err;
  m->opt = old;
  if (tw_change && upload_twiddles(m, old.dft_n, old.dft_hi_first) != STEV_OK) m->kfn = nullptr;
  return fail(st, "%s (previous options kept)", msg.c_str());
}

extern "C" stev_status stev_mechanism_get_options(const stev_mechanism* m, stev_options* opt) {
  if (!m || !opt) return fail(STEV_EINVAL, "NULL argument");
  *opt = m->opt;
  return STEV_OK;
}

extern "C" long stev_resident_slots(const stev_mechanism* m) { return m ? (long)m->nslots : 0; }

extern "C" int stev_is_specialized(const stev_mechanism* m) {
  return m && m->spec_k && m->kfn == reinterpret_cast<const void*>(m->spec_k) ? 1 : 0;
}

extern "C" long long stev_mlp_stalls(const stev_mechanism* m) {
  if (!m || !m->d_net_stalls) return 0;
  unsigned long long v = 0;
  if (cudaMemcpy(&v, m->d_net_stalls, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  return (long long)v;
}

static MlpInfer mlp_infer_view(const stev_mechanism* m);

static Launch make_launch(stev_mechanism* m, long long n, double dt) {
  Launch L{};
  L.S = m->S;
  L.R = m->R;
  L.Rrev = m->Rrev;
  L.n_gather = m->n_gather;
  L.sp_tab = m->d_sp;
  L.rx_tab = m->d_rx;
  L.rx_idx = m->d_ri;
  L.rx_idx_m = m->d_rim;
  L.g_ptr = m->d_gptr;
  L.g_ent = m->d_gent;
  L.dft_tw = m->d_tw;
  L.sp_tab_f = m->d_spf;
  L.rx_tab_f = m->d_rxf;
  L.dft_tw_f = m->d_twf;
  L.n_hi_bins = m->n_hi_bins;
  L.dft_n = m->opt.dft_n;
  L.dft_on = m->opt.dft_on;
  L.max_iters = m->opt.max_iters;
  L.y_step_max = m->opt.y_step_max;
  L.delta_max = m->opt.delta_max;
  L.alpha = m->opt.alpha;
  L.tol_ring = m->opt.tol_ring;
  L.tol_freq = m->opt.tol_freq;
  L.r_fac = m->opt.r_fac;
  L.rof_min = m->opt.rof_min;
  L.y_step_max_f = (float)m->opt.y_step_max;
  L.alpha_f = (float)m->opt.alpha;
  L.tol_ring_f = (float)m->opt.tol_ring;
  L.tol_freq_f = (float)m->opt.tol_freq;
  L.r_fac_f = (float)m->opt.r_fac;
  L.inv_r_fac_f = 1.0f / (float)m->opt.r_fac;
  L.rof_min_f = (float)m->opt.rof_min;
  L.ln_patm_over_ru = std::log(kPatm / kRu);
  L.n_cells = n;
  L.dt = dt;
  L.counter = m->d_counter;
  if (m->opt.thermo != STEV_THERMO_POLY && m->mlp_ready) {
    L.mlp = mlp_infer_view(m);
    L.mlp_h = m->opt.thermo == STEV_THERMO_MLP_CPH;
    L.mlp_needed = (L.mlp_h ? 2 : 1) * m->S;
  }
  L.general = m->general;
  L.rg_tab = m->d_rg;
  L.g_nu = m->d_gnu;
  L.rg_tab_f = m->d_rgf;
  L.g_nu_f = m->d_gnuf;
  return L;
}

static stev_status check_solve_args(stev_mechanism* m, long n, const void* T, const void* P,
                                    const void* Y, double dt, const void* To, const void* Yo,
                                    const void* it, const void* cs) {
  if (!m) return fail(STEV_EINVAL, "mechanism is NULL");
  if (m->opt.thermo != STEV_THERMO_POLY && !m->mlp_ready)
    return fail(STEV_EINVAL, "thermo = MLP needs a trained network (stev_mlp_train or stev_mlp_set_params)");
  if (n < 0) return fail(STEV_EINVAL, "n_cells < 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(STEV_EINVAL, "dt_cfd must be finite and > 0");
  if (n > 0 && (!T || !P || !Y || !To || !Yo || !it || !cs)) return fail(STEV_EINVAL, "NULL array");
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != m->device) return fail(STEV_EINVAL, "mechanism lives on device %d, current is %d", m->device, dev);
  return STEV_OK;
}

// Launches the mechanism's solver kernel (generic or specialised) with the
// launch configuration chosen by configure().
static cudaError_t launch_solver(const stev_mechanism* m, int grid, const Launch& L,
                                 cudaStream_t s) {
  if (!m->kfn) return cudaErrorInvalidDeviceFunction;  // no valid configuration
  Launch arg = L;
  void* args[] = {&arg};
  const cudaError_t e =
      cudaLaunchKernel(m->kfn, dim3((unsigned)grid), dim3((unsigned)m->block), args, m->smem, s);
  return e != cudaSuccess ? e : cudaGetLastError();
}

static stev_status launch_persistent(stev_mechanism* m, const Launch& L, cudaStream_t s) {
  CUDA_TRY(cudaMemsetAsync(m->d_counter, 0, sizeof(unsigned long long), s));
  CUDA_TRY(launch_solver(m, m->grid, L, s));
  return STEV_OK;
}

static stev_status solve_impl(stev_mechanism* m, long n, const double* T, const double* P,
                              const double* Y, double dt, double* T_out, double* Y_out,
                              int* iters, unsigned char* cell_status, void* stream, int soa) {
  g_err.clear();
  stev_status st = check_solve_args(m, n, T, P, Y, dt, T_out, Y_out, iters, cell_status);
  if (st != STEV_OK || n == 0) return st;
  Launch L = make_launch(m, n, dt);
  L.T = T; L.P = P; L.Y = Y;
  L.T_out = T_out; L.Y_out = Y_out; L.iters = iters; L.status = cell_status;
  L.y_soa = soa;
  return launch_persistent(m, L, (cudaStream_t)stream);
}

extern "C" stev_status stev_solve(stev_mechanism* m, long n, const double* T, const double* P,
                                  const double* Y, double dt, double* T_out, double* Y_out,
                                  int* iters, unsigned char* cell_status, void* stream) {
  return solve_impl(m, n, T, P, Y, dt, T_out, Y_out, iters, cell_status, stream, 0);
}

extern "C" stev_status stev_solve_soa(stev_mechanism* m, long n, const double* T, const double* P,
                                      const double* Y, double dt, double* T_out, double* Y_out,
                                      int* iters, unsigned char* cell_status, void* stream) {
  return solve_impl(m, n, T, P, Y, dt, T_out, Y_out, iters, cell_status, stream, 1);
}

extern "C" stev_status stev_solve_batched(stev_mechanism* m, int n_batches, const long* n_cells,
                                          const double* const* T, const double* const* P,
                                          const double* const* Y, const double* dt,
                                          double* const* T_out, double* const* Y_out,
                                          int* const* iters, unsigned char* const* cell_status,
                                          void* stream) {
  g_err.clear();
  if (!m) return fail(STEV_EINVAL, "mechanism is NULL");
  if (n_batches < 0) return fail(STEV_EINVAL, "n_batches < 0");
  if (n_batches == 0) return STEV_OK;
  if (!n_cells || !T || !P || !Y || !dt || !T_out || !Y_out || !iters || !cell_status)
    return fail(STEV_EINVAL, "NULL argument");
  std::vector<BatchDesc> desc;
  std::vector<long long> off(1, 0);
  for (int b = 0; b < n_batches; ++b) {
    if (n_cells[b] < 0) return fail(STEV_EINVAL, "n_cells[%d] < 0", b);
    if (n_cells[b] == 0) continue;
    if (!(dt[b] > 0.0) || !std::isfinite(dt[b])) return fail(STEV_EINVAL, "dt[%d] must be finite and > 0", b);
    if (!T[b] || !P[b] || !Y[b] || !T_out[b] || !Y_out[b] || !iters[b] || !cell_status[b])
      return fail(STEV_EINVAL, "NULL array in batch %d", b);
    BatchDesc d;
    d.T = T[b]; d.P = P[b]; d.Y = Y[b]; d.T_out = T_out[b]; d.Y_out = Y_out[b];
    d.iters = iters[b]; d.status = cell_status[b]; d.dt = dt[b]; d.n = n_cells[b];
    desc.push_back(d);
    off.push_back(off.back() + n_cells[b]);
  }
  if (desc.empty()) return STEV_OK;
  stev_status st = check_solve_args(m, (long)off.back(), desc[0].T, desc[0].P, desc[0].Y, desc[0].dt,
                                    desc[0].T_out, desc[0].Y_out, desc[0].iters, desc[0].status);
  if (st != STEV_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int nb = (int)desc.size();
  if (nb > m->batch_cap) {
    CUDA_TRY(cudaStreamSynchronize(s));
    if (m->d_bdesc) cudaFree(m->d_bdesc);
    if (m->d_boff) cudaFree(m->d_boff);
    m->d_bdesc = nullptr;
    m->d_boff = nullptr;
    m->batch_cap = 0;
    CUDA_TRY(cudaMalloc(&m->d_bdesc, (size_t)nb * sizeof(BatchDesc)));
    CUDA_TRY(cudaMalloc(&m->d_boff, (size_t)(nb + 1) * sizeof(long long)));
    m->batch_cap = nb;
  }
  // pageable sources: the copies are staged before cudaMemcpyAsync returns
  CUDA_TRY(cudaMemcpyAsync(m->d_bdesc, desc.data(), desc.size() * sizeof(BatchDesc),
                           cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(m->d_boff, off.data(), off.size() * sizeof(long long),
                           cudaMemcpyHostToDevice, s));
  Launch L = make_launch(m, off.back(), desc[0].dt);
  L.nb = nb;
  L.boff = m->d_boff;
  L.bdesc = m->d_bdesc;
  L.y_soa = 0;
  return launch_persistent(m, L, s);
}

extern "C" stev_status stev_solve_host(stev_mechanism* m, long n, const double* T, const double* P,
                                       const double* Y, double dt, double* T_out, double* Y_out,
                                       int* iters, unsigned char* cell_status, void* stream) {
  g_err.clear();
  if (!m) return fail(STEV_EINVAL, "mechanism is NULL");
  if (n < 0) return fail(STEV_EINVAL, "n_cells < 0");
  if (n == 0) return STEV_OK;
  if (!T || !P || !Y || !T_out || !Y_out || !iters || !cell_status) return fail(STEV_EINVAL, "NULL array");
  cudaStream_t s = (cudaStream_t)stream;
  if (n > m->host_cap) {
    CUDA_TRY(cudaStreamSynchronize(s));
    void** bufs[] = {(void**)&m->d_hT, (void**)&m->d_hP, (void**)&m->d_hY, (void**)&m->d_hTo,
                     (void**)&m->d_hYo, (void**)&m->d_hit, (void**)&m->d_hst};
    for (void** b : bufs) { if (*b) cudaFree(*b); *b = nullptr; }
    m->host_cap = 0;
    const size_t sz[] = {(size_t)n * 8, (size_t)n * 8, (size_t)n * m->S * 8, (size_t)n * 8,
                         (size_t)n * m->S * 8, (size_t)n * 4, (size_t)n};
    for (int k = 0; k < 7; ++k) CUDA_TRY(cudaMalloc(bufs[k], sz[k]));
    m->host_cap = n;
  }
  CUDA_TRY(cudaMemcpyAsync(m->d_hT, T, (size_t)n * 8, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(m->d_hP, P, (size_t)n * 8, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(m->d_hY, Y, (size_t)n * m->S * 8, cudaMemcpyHostToDevice, s));
  stev_status st = stev_solve(m, n, m->d_hT, m->d_hP, m->d_hY, dt, m->d_hTo, m->d_hYo, m->d_hit,
                              m->d_hst, stream);
  if (st != STEV_OK) return st;
  CUDA_TRY(cudaMemcpyAsync(T_out, m->d_hTo, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(Y_out, m->d_hYo, (size_t)n * m->S * 8, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(iters, m->d_hit, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(cell_status, m->d_hst, (size_t)n, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return STEV_OK;
}

// ------------------------------------------------------ serving interface
namespace stev {
namespace host {

stev_status serve_config(const stev_mechanism* m, ServeConfig* out) {
  if (!m) return fail(STEV_EINVAL, "mechanism is NULL");
  if (m->opt.thermo != STEV_THERMO_POLY && !m->mlp_ready)
    return fail(STEV_EINVAL, "thermo = MLP needs a trained network (stev_mlp_train or stev_mlp_set_params)");
  out->device = m->device;
  out->S = m->S;
  out->ctas_per_sm = m->per_sm;
  out->sms = m->sms;
  out->cells_per_cta = m->cells;
  return STEV_OK;
}

stev_status serve_launch(stev_mechanism* m, ServeCtl* ctl, ServeSlot* slots,
                         volatile long long* mail, int q, long long idle_ns, int grid,
                         cudaStream_t s) {
  Launch L = make_launch(m, 0, 1.0);
  L.serve = 1;
  L.ctl = ctl;
  L.slots = slots;
  L.smail = mail;
  L.serve_q = q;
  L.idle_ns = idle_ns;
  L.serve_warps = grid * (m->cells * m->G / 32);  // warps holding cells
  L.y_soa = 0;
  CUDA_TRY(cudaMemsetAsync(&ctl->idle_warps, 0, 2 * sizeof(int), s));  // idle_warps, exiting
  CUDA_TRY(launch_solver(m, grid, L, s));
  return STEV_OK;
}

}  // namespace host
}  // namespace stev

extern "C" void stev_destroy(stev_mechanism* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  free_mech(m);
}

extern "C" const char* stev_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------ solve without allocating
// Some callers may not allocate device memory at solve time: a CFD code whose
// device memory is owned by its own pool allocator and budget, a real-time or
// host-callback context where cudaMalloc's implicit device synchronisation is
// not acceptable, or a process that must not grow its footprint after start-up.
// stev_solve_host_noalloc serves them: it stages the host arrays through one
// file-scope device array of fixed size instead of mechanism-owned buffers,
// and calls no cudaMalloc, cudaFree or other allocating routine.
//
// Layout of the array for n cells of S species, each piece 256-byte aligned:
// [work counter][T][P][Y n*S][T_out][Y_out n*S][iters][status].
static constexpr size_t kNoAllocBytes = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static constexpr int kNoAllocMaxDevices = 64;
static void* g_noalloc_ptr[kNoAllocMaxDevices];  // device address per device, set once
static std::mutex g_noalloc_mutex;

static size_t noalloc_align(size_t b) { return (b + 255) & ~(size_t)255; }

// Cells the array could hold if nothing were padded: 16 S + 21 bytes per cell
// (T, P, T_out: 8 each; Y, Y_out: 8 S each; iters 4; status 1).  Any n above
// it is rejected before noalloc_bytes() multiplies (no size_t wrap-around).
static long noalloc_cell_bound(int S) { return (long)(kNoAllocBytes / (16 * (size_t)S + 21)); }

static size_t noalloc_bytes(long n, int S) {
  const size_t nn = (size_t)n;
  return noalloc_align(sizeof(unsigned long long)) + 2 * noalloc_align(nn * 8) +
         noalloc_align(nn * S * 8) + noalloc_align(nn * 8) + noalloc_align(nn * S * 8) +
         noalloc_align(nn * 4) + noalloc_align(nn);
}

extern "C" stev_status stev_solve_host_noalloc(stev_mechanism* m, long n, const double* T,
                                               const double* P, const double* Y, double dt,
                                               double* T_out, double* Y_out, int* iters,
                                               unsigned char* cell_status, void* stream) {
  g_err.clear();
  if (!m) return fail(STEV_EINVAL, "mechanism is NULL");
  if (n < 0) return fail(STEV_EINVAL, "n_cells < 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(STEV_EINVAL, "dt_cfd must be finite and > 0");
  if (n == 0) return STEV_OK;
  if (!T || !P || !Y || !T_out || !Y_out || !iters || !cell_status)
    return fail(STEV_EINVAL, "NULL array");
  if (m->opt.thermo != STEV_THERMO_POLY && !m->mlp_ready)
    return fail(STEV_EINVAL, "thermo = MLP needs a trained network (stev_mlp_train or stev_mlp_set_params)");
  if (n > noalloc_cell_bound(m->S) || noalloc_bytes(n, m->S) > kNoAllocBytes) {
    long lo = 0, hi = std::min(n, noalloc_cell_bound(m->S) + 1);  // lo fits, hi does not
    while (hi - lo > 1) {
      const long mid = (lo + hi) / 2;
      if (noalloc_bytes(mid, m->S) <= kNoAllocBytes) lo = mid; else hi = mid;
    }
    return fail(STEV_EINVAL,
                "stev_solve_host_noalloc: %ld cells of %d species need more than the %zu bytes "
                "of staging its fixed device array holds (at most %ld cells)",
                n, m->S, kNoAllocBytes, lo);
  }
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != m->device) return fail(STEV_EINVAL, "mechanism lives on device %d, current is %d", m->device, dev);
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(STEV_EINVAL, "device index %d out of range", dev);
  unsigned char* base = nullptr;
  {
    // set-up, once per device: the array's device address (host code only
    // knows a stand-in for it).  Like the mechanisms' own device buffers, the
    // cached address does not outlive the device's context (cudaDeviceReset).
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_ptr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  }
  const size_t nn = (size_t)n;
  unsigned char* q = base;
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(q);
  q += noalloc_align(sizeof(unsigned long long));
  double* dT = reinterpret_cast<double*>(q);   q += noalloc_align(nn * 8);
  double* dP = reinterpret_cast<double*>(q);   q += noalloc_align(nn * 8);
  double* dY = reinterpret_cast<double*>(q);   q += noalloc_align(nn * m->S * 8);
  double* dTo = reinterpret_cast<double*>(q);  q += noalloc_align(nn * 8);
  double* dYo = reinterpret_cast<double*>(q);  q += noalloc_align(nn * m->S * 8);
  int* dit = reinterpret_cast<int*>(q);        q += noalloc_align(nn * 4);
  unsigned char* dst = q;
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(dT, T, nn * 8, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(dP, P, nn * 8, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(dY, Y, nn * m->S * 8, cudaMemcpyHostToDevice, s));
  // the counter must start at zero; it keeps the previous call's value
  CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
  Launch L = make_launch(m, n, dt);
  L.T = dT; L.P = dP; L.Y = dY;
  L.T_out = dTo; L.Y_out = dYo; L.iters = dit; L.status = dst;
  L.y_soa = 0;
  L.counter = counter;
  CUDA_TRY(launch_solver(m, m->grid, L, s));
  CUDA_TRY(cudaMemcpyAsync(T_out, dTo, nn * 8, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(Y_out, dYo, nn * m->S * 8, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(iters, dit, nn * 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(cell_status, dst, nn, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return STEV_OK;
}

// ------------------------------------------------------- thermo network
// Fragment-ordered copy of the network (MlpFrag): sizes and offsets of its
// parts in one buffer, each 16-byte aligned.
static int mlp_frag_mt3(int n_out) { return (n_out + 15) / 16; }
static size_t mlp_frag_bytes(int n_out) {
  const size_t mt3 = (size_t)mlp_frag_mt3(n_out);
  return 16 * 32 * 16 + mt3 * 4 * 32 * 16 + 4 * 32 * 8 + mt3 * 32 * 16 + kHid * 8;
}

static stev_status mlp_ensure(stev_mechanism* m) {
  if (m->d_mlp_params) return STEV_OK;
  m->mlp_out = 3 * m->S;
  m->mlp_out_pad = (m->mlp_out + 7) / 8 * 8;
  m->mlp_np = mlp_n_params(m->mlp_out);
  CUDA_TRY(cudaMalloc(&m->d_mlp_params, (size_t)m->mlp_np * sizeof(float)));
  CUDA_TRY(cudaMalloc(&m->d_mlp_W2, (size_t)kHid * kHid * sizeof(__nv_bfloat16)));
  CUDA_TRY(cudaMalloc(&m->d_mlp_W3, (size_t)m->mlp_out_pad * kHid * sizeof(__nv_bfloat16)));
  CUDA_TRY(cudaMalloc(&m->d_mlp_misc, (size_t)(3 * kHid + 3 * m->mlp_out_pad) * sizeof(float)));
  CUDA_TRY(cudaMalloc(&m->d_mlp_frag, mlp_frag_bytes(m->mlp_out)));
  return STEV_OK;
}


// BF16 pair (lo in the low half) of two FP32 values, rounded to nearest even.
static unsigned pack_bf16_host(float lo, float hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
  unsigned short ua, ub;
  std::memcpy(&ua, &a, 2);
  std::memcpy(&ub, &b, 2);
  return (unsigned)ua | ((unsigned)ub << 16);
}

// The A fragment words of tile (mt, kt) of a row-major [rows][64] weight
// matrix W for lane l (rows beyond n_rows are zero): see MlpFrag.
static void frag_tile(const float* W, int n_rows, int mt, int kt, int l, unsigned out[4]) {
  const int g = l / 4, q = l % 4;
  auto w = [&](int r, int c) { return r < n_rows ? W[(size_t)r * kHid + c] : 0.0f; };
  const int r0 = 16 * mt + g, r1 = r0 + 8, c0 = 16 * kt + 2 * q, c1 = c0 + 8;
  out[0] = pack_bf16_host(w(r0, c0), w(r0, c0 + 1));
  out[1] = pack_bf16_host(w(r1, c0), w(r1, c0 + 1));
  out[2] = pack_bf16_host(w(r0, c1), w(r0, c1 + 1));
  out[3] = pack_bf16_host(w(r1, c1), w(r1, c1 + 1));
}

// FP32 master parameters (host copy) + standardisation -> inference buffers
static stev_status mlp_pack(stev_mechanism* m, const std::vector<float>& P,
                            const std::vector<float>& mean, const std::vector<float>& stdv) {
  const MlpOffsets o = mlp_offsets(m->mlp_out);
  {
    // fragment order: W2 tiles, W3 tiles, b2 pairs, layer-3 (scale, offset), (W1, b1)
    const int no = m->mlp_out, mt3 = mlp_frag_mt3(no);
    std::vector<unsigned char> buf(mlp_frag_bytes(no), 0);
    unsigned* w2f = reinterpret_cast<unsigned*>(buf.data());
    unsigned* w3f = w2f + 16 * 32 * 4;
    float* b2f = reinterpret_cast<float*>(w3f + (size_t)mt3 * 4 * 32 * 4);
    float* o3f = b2f + 4 * 32 * 2;
    float* w1f = o3f + (size_t)mt3 * 32 * 4;
    for (int mt = 0; mt < 4; ++mt)
      for (int kt = 0; kt < 4; ++kt)
        for (int l = 0; l < 32; ++l) frag_tile(&P[o.W2], kHid, mt, kt, l, w2f + ((mt * 4 + kt) * 32 + l) * 4);
    for (int mt = 0; mt < mt3; ++mt)
      for (int kt = 0; kt < 4; ++kt)
        for (int l = 0; l < 32; ++l) frag_tile(&P[o.W3], no, mt, kt, l, w3f + ((mt * 4 + kt) * 32 + l) * 4);
    for (int mt = 0; mt < 4; ++mt)
      for (int l = 0; l < 32; ++l) {
        b2f[(mt * 32 + l) * 2] = P[o.b2 + 16 * mt + l / 4];
        b2f[(mt * 32 + l) * 2 + 1] = P[o.b2 + 16 * mt + l / 4 + 8];
      }
    for (int mt = 0; mt < mt3; ++mt)
      for (int l = 0; l < 32; ++l)
        for (int h = 0; h < 2; ++h) {
          const int r = 16 * mt + l / 4 + 8 * h;
          const float sd = r < no ? stdv[r] : 1.0f, mu = r < no ? mean[r] : 0.0f;
          const float b3 = r < no ? P[o.b3 + r] : 0.0f;
          o3f[(mt * 32 + l) * 4 + 2 * h] = sd;
          o3f[(mt * 32 + l) * 4 + 2 * h + 1] = std::fmaf(b3, sd, mu);
        }
    for (int k = 0; k < kHid; ++k) {
      w1f[2 * k] = P[o.W1 + k];
      w1f[2 * k + 1] = P[o.b1 + k];
    }
    CUDA_TRY(cudaMemcpy(m->d_mlp_frag, buf.data(), buf.size(), cudaMemcpyHostToDevice));
  }
  std::vector<__nv_bfloat16> w2((size_t)kHid * kHid), w3((size_t)m->mlp_out_pad * kHid);
  for (int k = 0; k < kHid * kHid; ++k) w2[k] = __float2bfloat16_rn(P[o.W2 + k]);
  for (int r = 0; r < m->mlp_out_pad; ++r)
    for (int k = 0; k < kHid; ++k)
      w3[(size_t)r * kHid + k] = __float2bfloat16_rn(r < m->mlp_out ? P[o.W3 + r * kHid + k] : 0.0f);
  std::vector<float> misc((size_t)3 * kHid + 3 * m->mlp_out_pad, 0.0f);
  for (int k = 0; k < kHid; ++k) {
    misc[k] = P[o.W1 + k];
    misc[kHid + k] = P[o.b1 + k];
    misc[2 * kHid + k] = P[o.b2 + k];
  }
  float* b3 = misc.data() + 3 * kHid;
  float* mu = b3 + m->mlp_out_pad;
  float* sd = mu + m->mlp_out_pad;
  for (int r = 0; r < m->mlp_out_pad; ++r) {
    b3[r] = r < m->mlp_out ? P[o.b3 + r] : 0.0f;
    mu[r] = r < m->mlp_out ? mean[r] : 0.0f;
    sd[r] = r < m->mlp_out ? stdv[r] : 1.0f;
  }
  CUDA_TRY(cudaMemcpy(m->d_mlp_params, P.data(), P.size() * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(m->d_mlp_W2, w2.data(), w2.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(m->d_mlp_W3, w3.data(), w3.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(m->d_mlp_misc, misc.data(), misc.size() * sizeof(float), cudaMemcpyHostToDevice));
  m->mlp_ready = true;
  return STEV_OK;
}

static MlpInfer mlp_infer_view(const stev_mechanism* m) {
  MlpInfer w;
  w.W2 = m->d_mlp_W2;
  w.W3 = m->d_mlp_W3;
  w.W1 = m->d_mlp_misc;
  w.b1 = m->d_mlp_misc + kHid;
  w.b2 = m->d_mlp_misc + 2 * kHid;
  w.b3 = m->d_mlp_misc + 3 * kHid;
  w.mean = w.b3 + m->mlp_out_pad;
  w.stdv = w.mean + m->mlp_out_pad;
  w.n_out = m->mlp_out_pad;
  w.n_valid = m->mlp_out;
  const int mt3 = mlp_frag_mt3(m->mlp_out);
  const unsigned char* base = m->d_mlp_frag;
  w.frag.W2 = reinterpret_cast<const uint4*>(base);
  w.frag.W3 = w.frag.W2 + 16 * 32;
  w.frag.b2 = reinterpret_cast<const float2*>(w.frag.W3 + (size_t)mt3 * 4 * 32);
  w.frag.o3 = reinterpret_cast<const float4*>(w.frag.b2 + 4 * 32);
  w.frag.w1 = reinterpret_cast<const float2*>(w.frag.o3 + (size_t)mt3 * 32);
  w.frag.mt3 = mt3;
  return w;
}

extern "C" long stev_mlp_num_params(const stev_mechanism* m) {
  return m ? (long)mlp_n_params(3 * m->S) : 0;
}

extern "C" stev_status stev_mlp_set_params(stev_mechanism* m, const float* params, long n_params,
                                           const float* mean, const float* stdv) {
  g_err.clear();
  if (!m || !params || !mean || !stdv) return fail(STEV_EINVAL, "NULL argument");
  if (n_params != mlp_n_params(3 * m->S))
    return fail(STEV_EINVAL, "expected %d parameters, got %ld", mlp_n_params(3 * m->S), n_params);
  for (long k = 0; k < n_params; ++k)
    if (!std::isfinite(params[k])) return fail(STEV_EINVAL, "parameter %ld not finite", k);
  for (int r = 0; r < 3 * m->S; ++r)
    if (!std::isfinite(mean[r]) || !(stdv[r] > 0.0f)) return fail(STEV_EINVAL, "bad standardisation %d", r);
  stev_status st = mlp_ensure(m);
  if (st != STEV_OK) return st;
  std::vector<float> P(params, params + n_params), mu(mean, mean + 3 * m->S), sd(stdv, stdv + 3 * m->S);
  return mlp_pack(m, P, mu, sd);
}

extern "C" stev_status stev_mlp_get_params(const stev_mechanism* m, float* params, long n_params,
                                           float* mean, float* stdv) {
  g_err.clear();
  if (!m || !params || !mean || !stdv) return fail(STEV_EINVAL, "NULL argument");
  if (!m->mlp_ready) return fail(STEV_EINVAL, "the thermo network has not been trained or set");
  if (n_params != m->mlp_np) return fail(STEV_EINVAL, "expected %d parameters", m->mlp_np);
  CUDA_TRY(cudaMemcpy(params, m->d_mlp_params, (size_t)n_params * sizeof(float), cudaMemcpyDeviceToHost));
  const float* base = m->d_mlp_misc + 3 * kHid + m->mlp_out_pad;
  CUDA_TRY(cudaMemcpy(mean, base, (size_t)m->mlp_out * sizeof(float), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(stdv, base + m->mlp_out_pad, (size_t)m->mlp_out * sizeof(float), cudaMemcpyDeviceToHost));
  return STEV_OK;
}

// Per-tile gradients and squared errors of the network with parameters
// `params` on n samples (standardised targets), through the training kernel:
// part [tiles][n_params], loss_part [tiles], tiles = ceil(n / kMlpTile).
static stev_status mlp_grad_device(stev_mechanism* m, const float* d_params, const double* d_T,
                                   const float* d_target, long long n, long long n_total,
                                   float* d_part, double* d_loss_part, cudaStream_t s) {
  const size_t smem = mlp_grad_smem_bytes(m->mlp_out);
  CUDA_TRY(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int blocks = (int)((n + kMlpTile - 1) / kMlpTile);
  mlp_grad_kernel<<<blocks, kMlpTile, smem, s>>>(d_params, m->mlp_out, d_T, d_target, n, n_total,
                                                 d_part, d_loss_part);
  CUDA_TRY(cudaGetLastError());
  return STEV_OK;
}

extern "C" stev_status stev_mlp_loss_grad(stev_mechanism* m, const float* params, const double* T,
                                          const float* target, long n, float* grad,
                                          double* loss) {
  g_err.clear();
  if (!m || !params || !T || !target || !grad || !loss) return fail(STEV_EINVAL, "NULL argument");
  if (n < 1) return fail(STEV_EINVAL, "n < 1");
  const int np = mlp_n_params(3 * m->S), no = 3 * m->S;
  m->mlp_out = no;
  const int tiles = (int)((n + kMlpTile - 1) / kMlpTile);
  float *dp = nullptr, *dt = nullptr, *dg = nullptr, *dpart = nullptr;
  double *dT = nullptr, *dl = nullptr, *dlp = nullptr;
  stev_status st = STEV_OK;
  auto cleanup = [&]() {
    cudaFree(dp); cudaFree(dt); cudaFree(dg); cudaFree(dT); cudaFree(dl); cudaFree(dpart);
    cudaFree(dlp);
  };
#define TRY_CLEAN(expr)                                                                     \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      cleanup();                                                                            \
      return fail(STEV_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));                     \
    }                                                                                       \
  } while (0)
  TRY_CLEAN(cudaMalloc(&dp, (size_t)np * 4));
  TRY_CLEAN(cudaMalloc(&dg, (size_t)np * 4));
  TRY_CLEAN(cudaMalloc(&dt, (size_t)n * no * 4));
  TRY_CLEAN(cudaMalloc(&dT, (size_t)n * 8));
  TRY_CLEAN(cudaMalloc(&dl, 8));
  TRY_CLEAN(cudaMalloc(&dpart, (size_t)tiles * np * 4));
  TRY_CLEAN(cudaMalloc(&dlp, (size_t)tiles * 8));
  TRY_CLEAN(cudaMemcpy(dp, params, (size_t)np * 4, cudaMemcpyHostToDevice));
  TRY_CLEAN(cudaMemcpy(dt, target, (size_t)n * no * 4, cudaMemcpyHostToDevice));
  TRY_CLEAN(cudaMemcpy(dT, T, (size_t)n * 8, cudaMemcpyHostToDevice));
  TRY_CLEAN(cudaMemset(dl, 0, 8));
  st = mlp_grad_device(m, dp, dT, dt, n, n, dpart, dlp, 0);
  if (st == STEV_OK) {
    mlp_sum_kernel<<<(np + 255) / 256, 256>>>(dpart, tiles, np, dlp, dg, dl);
    TRY_CLEAN(cudaGetLastError());
    TRY_CLEAN(cudaMemcpy(grad, dg, (size_t)np * 4, cudaMemcpyDeviceToHost));
    TRY_CLEAN(cudaMemcpy(loss, dl, 8, cudaMemcpyDeviceToHost));
    *loss /= (double)n * no;
  }
#undef TRY_CLEAN
  cleanup();
  return st;
}

// Training targets at n DEVICE temperatures: the NASA-7 polynomials (FP64,
// stored FP32) standardised per output.  fresh: compute each output's mean and
// standard deviation (per-block partial sums added in a fixed order);
// otherwise mean / stdv are inputs (continuing a trained network).
static stev_status mlp_make_targets(stev_mechanism* m, const double* dT, long long n,
                                    float* dtarget, std::vector<float>& mean,
                                    std::vector<float>& stdv, bool fresh) {
  const int no = m->mlp_out;
  const long long tot = n * m->S;
  mlp_targets_kernel<<<(unsigned)((tot + 255) / 256), 256>>>(m->d_sp, m->S, dT, n, dtarget);
  CUDA_TRY(cudaGetLastError());
  if (fresh) {
    const int mom_blocks = 64;
    double* dsum = nullptr;
    CUDA_TRY(cudaMalloc(&dsum, (size_t)2 * no * mom_blocks * 8));
    mlp_moments_kernel<<<dim3(mom_blocks, no), 256>>>(dtarget, n, no, dsum);
    std::vector<double> parts((size_t)2 * no * mom_blocks);
    const cudaError_t e = cudaMemcpy(parts.data(), dsum, parts.size() * 8, cudaMemcpyDeviceToHost);
    cudaFree(dsum);
    CUDA_TRY(e);
    mean.assign(no, 0.0f);
    stdv.assign(no, 1.0f);
    for (int c = 0; c < no; ++c) {
      double s1 = 0.0, s2 = 0.0;
      for (int b = 0; b < mom_blocks; ++b) {
        s1 += parts[((size_t)c * mom_blocks + b) * 2];
        s2 += parts[((size_t)c * mom_blocks + b) * 2 + 1];
      }
      const double mu = s1 / n;
      const double var = std::max(s2 / n - mu * mu, 0.0);
      mean[c] = (float)mu;
      stdv[c] = (float)std::max(std::sqrt(var), 1e-6 * std::max(1.0, std::fabs(mu)));
    }
  }
  std::vector<float> stat((size_t)2 * no);
  for (int c = 0; c < no; ++c) {
    stat[c] = mean[c];
    stat[no + c] = 1.0f / stdv[c];
  }
  float* dstat = nullptr;
  CUDA_TRY(cudaMalloc(&dstat, stat.size() * 4));
  cudaError_t e = cudaMemcpy(dstat, stat.data(), stat.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    mlp_standardise_kernel<<<(unsigned)((n * no + 255) / 256), 256>>>(dtarget, n, no, dstat,
                                                                       dstat + no);
    e = cudaDeviceSynchronize();
  }
  cudaFree(dstat);
  CUDA_TRY(e);
  return STEV_OK;
}

static inline uint64_t splitmix64(uint64_t& x) {
  uint64_t z = (x += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

extern "C" stev_status stev_mlp_train(stev_mechanism* m, const double* T_samples, long n,
                                      int epochs, int batch, float lr, unsigned long long seed,
                                      float* loss_per_epoch) {
  g_err.clear();
  if (!m || !T_samples) return fail(STEV_EINVAL, "NULL argument");
  if (n < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f)) return fail(STEV_EINVAL, "bad training sizes");
  for (long k = 0; k < n; ++k)
    if (!(T_samples[k] > 0.0) || !std::isfinite(T_samples[k])) return fail(STEV_EINVAL, "T_samples[%ld] invalid", k);
  stev_status st = mlp_ensure(m);
  if (st != STEV_OK) return st;
  const int no = m->mlp_out, np = m->mlp_np;
  const int mb_tiles = (int)((std::min((long long)batch, (long long)n) + kMlpTile - 1) / kMlpTile);
  double *dT = nullptr, *dlp = nullptr, *dlep = nullptr;
  float *dtarget = nullptr, *dpart = nullptr, *dm1 = nullptr, *dm2 = nullptr;
  float4* dsched = nullptr;
  auto cleanup = [&]() {
    cudaFree(dT); cudaFree(dtarget); cudaFree(dpart); cudaFree(dm1); cudaFree(dm2);
    cudaFree(dlp); cudaFree(dlep); cudaFree(dsched);
  };
#define TRY_CLEAN(expr)                                                                     \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      cleanup();                                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? STEV_ENOMEM : STEV_ECUDA, "%s: %s",     \
                  #expr, cudaGetErrorString(e_));                                           \
    }                                                                                       \
  } while (0)
  TRY_CLEAN(cudaMalloc(&dT, (size_t)n * 8));
  TRY_CLEAN(cudaMalloc(&dtarget, (size_t)n * no * 4));
  TRY_CLEAN(cudaMalloc(&dpart, (size_t)mb_tiles * np * 4));
  TRY_CLEAN(cudaMalloc(&dlp, (size_t)mb_tiles * 8));
  TRY_CLEAN(cudaMalloc(&dm1, (size_t)np * 4));
  TRY_CLEAN(cudaMalloc(&dm2, (size_t)np * 4));
  TRY_CLEAN(cudaMemcpy(dT, T_samples, (size_t)n * 8, cudaMemcpyHostToDevice));
  // targets: the polynomials in FP64, standardised per output column
  std::vector<float> mean, stdv;
  st = mlp_make_targets(m, dT, n, dtarget, mean, stdv, true);
  if (st != STEV_OK) { cleanup(); return st; }
  // Xavier-uniform initialisation from splitmix64(seed), zero biases
  const MlpOffsets o = mlp_offsets(no);
  std::vector<float> P(np, 0.0f);
  uint64_t rs = seed;
  auto uni = [&](float a) { return (float)(((splitmix64(rs) >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0) * a; };
  for (int k = 0; k < kHid; ++k) P[o.W1 + k] = uni(std::sqrt(6.0f / (1 + kHid)));
  for (int k = 0; k < kHid * kHid; ++k) P[o.W2 + k] = uni(std::sqrt(6.0f / (kHid + kHid)));
  for (int k = 0; k < no * kHid; ++k) P[o.W3 + k] = uni(std::sqrt(6.0f / (kHid + no)));
  TRY_CLEAN(cudaMemcpy(m->d_mlp_params, P.data(), (size_t)np * 4, cudaMemcpyHostToDevice));
  TRY_CLEAN(cudaMemset(dm1, 0, (size_t)np * 4));
  TRY_CLEAN(cudaMemset(dm2, 0, (size_t)np * 4));
  // Adam over minibatches in sample order (the samples are drawn
  // independently), the step size decaying from lr to lr/100 along a cosine;
  // every step in one cooperative launch (mlp_train_kernel), the schedule
  // computed here
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const long long per_epoch = (n + batch - 1) / batch, total = per_epoch * epochs;
  std::vector<float4> sched((size_t)total);
  for (long long step = 0; step < total; ++step) {
    const double frac = (double)step / (double)std::max(total - 1, 1LL);
    const float lr_t = (float)(lr * (0.01 + 0.99 * 0.5 * (1.0 + std::cos(M_PI * frac))));
    const float t = (float)(step + 1);
    sched[(size_t)step] = make_float4(lr_t, 1.0f - std::pow(b1, t), 1.0f - std::pow(b2, t), 0.0f);
  }
  TRY_CLEAN(cudaMalloc(&dsched, sched.size() * sizeof(float4)));
  TRY_CLEAN(cudaMalloc(&dlep, (size_t)epochs * 8));
  TRY_CLEAN(cudaMemcpy(dsched, sched.data(), sched.size() * sizeof(float4), cudaMemcpyHostToDevice));
  TRY_CLEAN(cudaMemset(dlep, 0, (size_t)epochs * 8));
  {
    const size_t smem = mlp_grad_smem_bytes(no);
    TRY_CLEAN(cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0, dev = 0, sms = 0;
    TRY_CLEAN(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mlp_train_kernel, kMlpTile, smem));
    TRY_CLEAN(cudaGetDevice(&dev));
    TRY_CLEAN(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (per_sm < 1) { cleanup(); return fail(STEV_EINVAL, "training kernel cannot be resident"); }
    const int grid = std::min(mb_tiles, per_sm * sms);
    int no_ = no;
    long long n_ = n, total_ = total, per_epoch_ = per_epoch;
    int batch_ = batch;
    float* pp = m->d_mlp_params;
    float b1_ = b1, b2_ = b2, eps_ = eps;
    void* args[] = {&pp, &no_, &dT, &dtarget, &n_, &batch_, &dsched, &total_, &per_epoch_, &dpart,
                    &dlp, &dm1, &dm2, &dlep, &b1_, &b2_, &eps_};
    TRY_CLEAN(cudaLaunchCooperativeKernel((const void*)mlp_train_kernel, dim3(grid), dim3(kMlpTile),
                                          args, smem, 0));
    TRY_CLEAN(cudaGetLastError());
  }
  if (loss_per_epoch) {
    std::vector<double> l(epochs);
    TRY_CLEAN(cudaMemcpy(l.data(), dlep, (size_t)epochs * 8, cudaMemcpyDeviceToHost));
    for (int ep = 0; ep < epochs; ++ep) loss_per_epoch[ep] = (float)(l[ep] / ((double)n * no));
  }
  TRY_CLEAN(cudaMemcpy(P.data(), m->d_mlp_params, (size_t)np * 4, cudaMemcpyDeviceToHost));
#undef TRY_CLEAN
  cleanup();
  return mlp_pack(m, P, mean, stdv);
}

// --------------------------------------- Levenberg-Marquardt training
static stev_status launch_jacobian_t(int no, const float* dp, const double* dT, const float* dtg,
                                     long long nsamp, float* dJt, long long ldk, float* dr) {
  const size_t smem = mlp_jacobian_smem_bytes(no);
  CUDA_TRY(cudaFuncSetAttribute(mlp_jacobian_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  mlp_jacobian_t_kernel<<<(unsigned)nsamp, kJacThreads, smem>>>(dp, no, dT, dtg, dJt, ldk, dr);
  CUDA_TRY(cudaGetLastError());
  return STEV_OK;
}

extern "C" stev_status stev_mlp_jacobian(stev_mechanism* m, const float* params, const double* T,
                                         long n, float* J) {
  g_err.clear();
  if (!m || !params || !T || !J) return fail(STEV_EINVAL, "NULL argument");
  if (n < 1 || n > 4096) return fail(STEV_EINVAL, "n must be in [1, 4096]");
  const int no = 3 * m->S, np = mlp_n_params(no);
  const long long rows = (long long)n * no, ldk = (rows + 3) / 4 * 4;
  float *dp = nullptr, *dJt = nullptr, *dtg = nullptr, *dr = nullptr;
  double* dT = nullptr;
  auto cleanup = [&]() { cudaFree(dp); cudaFree(dJt); cudaFree(dtg); cudaFree(dr); cudaFree(dT); };
#define TRY_CLEAN(expr)                                                                     \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      cleanup();                                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? STEV_ENOMEM : STEV_ECUDA, "%s: %s",     \
                  #expr, cudaGetErrorString(e_));                                           \
    }                                                                                       \
  } while (0)
  TRY_CLEAN(cudaMalloc(&dp, (size_t)np * 4));
  TRY_CLEAN(cudaMalloc(&dJt, (size_t)np * ldk * 4));
  TRY_CLEAN(cudaMalloc(&dtg, (size_t)rows * 4));
  TRY_CLEAN(cudaMalloc(&dr, (size_t)rows * 4));
  TRY_CLEAN(cudaMalloc(&dT, (size_t)n * 8));
  TRY_CLEAN(cudaMemcpy(dp, params, (size_t)np * 4, cudaMemcpyHostToDevice));
  TRY_CLEAN(cudaMemcpy(dT, T, (size_t)n * 8, cudaMemcpyHostToDevice));
  TRY_CLEAN(cudaMemset(dtg, 0, (size_t)rows * 4));
  {
    const stev_status st = launch_jacobian_t(no, dp, dT, dtg, n, dJt, ldk, dr);
    if (st != STEV_OK) { cleanup(); return st; }
  }
  std::vector<float> jt((size_t)np * ldk);
  TRY_CLEAN(cudaMemcpy(jt.data(), dJt, jt.size() * 4, cudaMemcpyDeviceToHost));
  for (long long r = 0; r < rows; ++r)
    for (int q = 0; q < np; ++q) J[(size_t)r * np + q] = jt[(size_t)q * ldk + r];
#undef TRY_CLEAN
  cleanup();
  return STEV_OK;
}

extern "C" stev_status stev_mlp_train_lm(stev_mechanism* m, const double* T_samples, long n,
                                         int iterations, int batch, double lambda0, int init,
                                         unsigned long long seed, float* loss_per_iter) {
  g_err.clear();
  if (!m || !T_samples) return fail(STEV_EINVAL, "NULL argument");
  if (n < 1 || iterations < 1 || batch < 1 || !(lambda0 > 0.0) || !std::isfinite(lambda0))
    return fail(STEV_EINVAL, "bad training sizes");
  if (init != 0 && init != 1) return fail(STEV_EINVAL, "init must be 0 or 1");
  if (init == 1 && !m->mlp_ready) return fail(STEV_EINVAL, "init = 1 needs a trained network");
  for (long k = 0; k < n; ++k)
    if (!(T_samples[k] > 0.0) || !std::isfinite(T_samples[k])) return fail(STEV_EINVAL, "T_samples[%ld] invalid", k);
  stev_status st = mlp_ensure(m);
  if (st != STEV_OK) return st;
  const int no = m->mlp_out, np = m->mlp_np;
  const long long nb = std::min((long long)batch, (long long)n);
  const long long rows = nb * no, ldk = (rows + 3) / 4 * 4, lda = ((long long)np + 3) / 4 * 4;
  if ((double)np * ldk * 4 > 8e9) return fail(STEV_EINVAL, "batch too large (Jacobian over 8 GB)");
  double *dT = nullptr, *dse = nullptr;
  float *dtarget = nullptr, *dJt = nullptr, *dr = nullptr, *dA = nullptr, *dg = nullptr;
  float *dd = nullptr, *dp = nullptr, *dpn = nullptr;
  int* derr = nullptr;
  stev::host::CgWork cgw{};
  auto cleanup = [&]() {
    cudaFree(dT); cudaFree(dse); cudaFree(dtarget); cudaFree(dJt); cudaFree(dr); cudaFree(dA);
    cudaFree(dg); cudaFree(dd); cudaFree(dp); cudaFree(dpn); cudaFree(derr);
    stev::host::cg_work_free(&cgw);
  };
#define TRY_CLEAN(expr)                                                                     \
  do {                                                                                      \
    cudaError_t e_ = (expr);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      cleanup();                                                                            \
      return fail(e_ == cudaErrorMemoryAllocation ? STEV_ENOMEM : STEV_ECUDA, "%s: %s",     \
                  #expr, cudaGetErrorString(e_));                                           \
    }                                                                                       \
  } while (0)
#define ST_CLEAN(expr)                 \
  do {                                 \
    const stev_status s_ = (expr);     \
    if (s_ != STEV_OK) {               \
      cleanup();                       \
      return s_;                       \
    }                                  \
  } while (0)
  TRY_CLEAN(cudaMalloc(&dT, (size_t)n * 8));
  TRY_CLEAN(cudaMalloc(&dtarget, (size_t)n * no * 4));
  TRY_CLEAN(cudaMalloc(&dJt, (size_t)np * ldk * 4));
  TRY_CLEAN(cudaMalloc(&dr, (size_t)ldk * 4));
  TRY_CLEAN(cudaMalloc(&dA, (size_t)np * lda * 4));
  TRY_CLEAN(cudaMalloc(&dg, (size_t)np * 4));
  TRY_CLEAN(cudaMalloc(&dd, (size_t)np * 4));
  TRY_CLEAN(cudaMalloc(&dse, (size_t)nb * 8));
  TRY_CLEAN(cudaMalloc(&dp, (size_t)np * 4));
  TRY_CLEAN(cudaMalloc(&dpn, (size_t)np * 4));
  TRY_CLEAN(cudaMalloc(&derr, sizeof(int)));
  TRY_CLEAN(cudaMemset(derr, 0, sizeof(int)));
  TRY_CLEAN(cudaMemset(dr, 0, (size_t)ldk * 4));
  ST_CLEAN(stev::host::cg_work_alloc(&cgw, np));
  TRY_CLEAN(cudaMemcpy(dT, T_samples, (size_t)n * 8, cudaMemcpyHostToDevice));

  // targets (statistics kept when continuing) and starting parameters
  std::vector<float> P(np, 0.0f), mean, stdv;
  if (init == 1) {
    mean.resize(no);
    stdv.resize(no);
    ST_CLEAN(stev_mlp_get_params(m, P.data(), np, mean.data(), stdv.data()));
  }
  ST_CLEAN(mlp_make_targets(m, dT, n, dtarget, mean, stdv, init == 0));
  if (init == 0) {
    const MlpOffsets o = mlp_offsets(no);
    uint64_t rs = seed;
    auto uni = [&](float a) { return (float)(((splitmix64(rs) >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0) * a; };
    for (int k = 0; k < kHid; ++k) P[o.W1 + k] = uni(std::sqrt(6.0f / (1 + kHid)));
    for (int k = 0; k < kHid * kHid; ++k) P[o.W2 + k] = uni(std::sqrt(6.0f / (kHid + kHid)));
    for (int k = 0; k < no * kHid; ++k) P[o.W3 + k] = uni(std::sqrt(6.0f / (kHid + no)));
  }
  TRY_CLEAN(cudaMemcpy(dp, P.data(), (size_t)np * 4, cudaMemcpyHostToDevice));

  // the batch's mean squared error with parameters p (per-sample sums in order)
  std::vector<double> se(nb);
  auto batch_loss = [&](const float* p, long long s0, double* out) -> bool {
    mlp_sqerr_kernel<<<(unsigned)((nb + 127) / 128), 128>>>(p, no, dT + s0, dtarget + s0 * no, nb, dse);
    if (cudaMemcpy(se.data(), dse, (size_t)nb * 8, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    double t = 0.0;
    for (long long k = 0; k < nb; ++k) t += se[k];
    *out = t / (double)rows;
    return true;
  };
  // Per iteration: the batch's transposed Jacobian, the Gauss-Newton matrix
  // A = J^T J (TF32 tensor cores, FP32 accumulation) and g = J^T r; then
  // Marquardt's damped system (A + lambda diag A) d = g by preconditioned
  // conjugate gradients (relative residual 1e-3, at most kLmCgIters steps: an
  // inexact Levenberg-Marquardt step), accepted if the batch loss falls.
  const int kLmCgIters = 400;
  const double kLmCgTol = 1e-3, kLmEps = 1e-12;
  double lambda = lambda0;
  for (int it = 0; it < iterations; ++it) {
    const long long s0 = ((long long)it * nb) % std::max(1LL, (long long)n - nb + 1);
    ST_CLEAN(launch_jacobian_t(no, dp, dT + s0, dtarget + s0 * no, nb, dJt, ldk, dr));
    ST_CLEAN(stev::host::gram_tf32(dJt, np, rows, ldk, dA, lda, derr, 0));
    ST_CLEAN(stev::host::rows_dot(dJt, np, rows, ldk, dr, dg, 0));
    double loss0 = 0.0, loss1 = 0.0;
    if (!batch_loss(dp, s0, &loss0)) { cleanup(); return fail(STEV_ECUDA, "loss copy failed"); }
    int herr = 0;
    TRY_CLEAN(cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) { cleanup(); return fail(STEV_ETIMEOUT, "Gauss-Newton matrix: a pipeline wait timed out"); }
    bool accepted = false;
    for (int attempt = 0; attempt < 8 && !accepted; ++attempt) {
      int cg_it = 0;
      ST_CLEAN(stev::host::damped_cg(dA, np, lda, dg, lambda, kLmEps, dd, kLmCgIters, kLmCgTol, &cg_it,
                                     &cgw, 0));
      mlp_step_kernel<<<(np + 255) / 256, 256>>>(dp, dd, np, dpn);
      TRY_CLEAN(cudaGetLastError());
      if (!batch_loss(dpn, s0, &loss1)) { cleanup(); return fail(STEV_ECUDA, "loss copy failed"); }
      if (std::isfinite(loss1) && loss1 < loss0) {
        std::swap(dp, dpn);
        lambda = std::max(lambda / 3.0, 1e-9);
        accepted = true;
      } else {
        lambda *= 2.0;
      }
    }
    if (loss_per_iter) loss_per_iter[it] = (float)(accepted ? loss1 : loss0);
  }
  TRY_CLEAN(cudaMemcpy(P.data(), dp, (size_t)np * 4, cudaMemcpyDeviceToHost));
#undef TRY_CLEAN
#undef ST_CLEAN
  cleanup();
  return mlp_pack(m, P, mean, stdv);
}

extern "C" stev_status stev_mlp_eval(stev_mechanism* m, const double* T, long n, float* props,
                                     void* stream) {
  g_err.clear();
  if (!m) return fail(STEV_EINVAL, "mechanism is NULL");
  if (!m->mlp_ready) return fail(STEV_EINVAL, "the thermo network has not been trained or set");
  if (n < 0) return fail(STEV_EINVAL, "n < 0");
  if (n == 0) return STEV_OK;
  if (!T || !props) return fail(STEV_EINVAL, "NULL array");
  const int warps = 8;
  const size_t smem = mlp_eval_smem_bytes(warps);
  const long long groups = (n + 15) / 16;
  const int blocks = (int)std::min<long long>((groups + warps - 1) / warps, 148LL * 16);
  mlp_eval_kernel<<<blocks, warps * 32, smem, (cudaStream_t)stream>>>(mlp_infer_view(m), T, n, props);
  CUDA_TRY(cudaGetLastError());
  return STEV_OK;
}
