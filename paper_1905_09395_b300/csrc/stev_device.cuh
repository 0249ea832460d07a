// Device-side data layout shared by the STEV kernels (not by the oracle).
//
// Mechanism tables are built once on the host (stev_capi.cu) and staged into
// shared memory by every CTA of the persistent kernel:
//   species  : SP_STRIDE doubles each: W, 1/W, T_split, pad, low block, high block
//              (species-major in global memory; the FP64 kernel stages it
//              transposed, [row][S], and the mixed kernels use the float
//              table described at SF_* below, also [row][S])
//   block    : a0..a6 of NASA-7 plus pre-divided coefficients so that
//              cp/R = a0 + T(a1 + T(a2 + T(a3 + T a4)))                (Eq. 15)
//              H/RT = a0 + T(a1/2 + T(a2/3 + T(a3/4 + T a4/5))) + a5/T (Eq. 16)
//              G/RT = H/RT - S/R
//                   = a0(1 - lnT) - T(a1/2 + T(a2/6 + T(a3/12 + T a4/20))) + a5/T - a6
//   reaction : lnA, beta, Ea/R (Eq. 29 in log form), dN, and an int4 with the
//              packed species slots (two reactant, two product, 0xFF = none;
//              a species of order 2 fills both slots), dN = sum(nu), the
//              reversible flag and the reaction's index among reversible ones.
//   gather   : species-major lists of (reaction, nu) in ascending reaction
//              order, so that wdot_i = sum_r nu_ir q_r is summed in the same
//              order as a reaction-major scatter would add into it.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#ifndef __CUDACC_RTC__  // run-time compiled copies (stev_spec.cu) get these from NVRTC
#include <cstdint>
#endif

#include "stev_layout.h"

namespace stev {

constexpr int kMaxSpecies = 64;
constexpr int kMaxReactions = 512;
constexpr int kMaxDftN = 32;
constexpr int kMaxGatherEntries = 4 * kMaxReactions;
constexpr double kRu = 8.314462618;     // J/(mol K)
constexpr double kPatm = 101325.0;      // Pa, standard state of Eq. 30
constexpr int kNone = 0xFF;
constexpr int kMaxBlock = 512;       // threads per CTA of the FP64 persistent kernel
constexpr int kMaxBlockMixed = 768;  // threads per CTA of the mixed persistent kernel

enum { SP_W = 0, SP_INVW = 1, SP_TSPLIT = 2, SP_LOW = 4, SP_HIGH = 18, SP_STRIDE = 32 };
enum { B_A0 = 0, B_A1, B_A2, B_A3, B_A4, B_A5, B_A6, B_H1, B_H2, B_H3, B_H4, B_G2, B_G3, B_G4,
       B_SIZE };
enum { RX_LNA = 0, RX_BETA = 1, RX_EAR = 2, RX_DN = 3, RX_STRIDE = 4 };
// Float species table of the mixed kernels, coefficient-major ([row][S], so
// that lane i reading species i walks consecutive banks): W, 1/W, T_split as
// a float pair; per range a0..a5 and the H/RT coefficients a1/2..a4/5 (FP32);
// per range the seven coefficients of the species' Gibbs term in log2 units,
//   g2(T) = c0 + c1 lnT + c2/T + c3 T + c4 T^2 + c5 T^3 + c6 T^4
//         = log2 e (G/RT - ln(P_atm/R_u) + lnT)         (Eq. 30's exponent),
// each as a float pair (hi row, lo row) holding the FP64 value to ~2^-48.
enum { SF_W = 0, SF_INVW = 1, SF_SPLIT_H = 2, SF_SPLIT_L = 3, SF_LOW = 4, SF_HIGH = 14,
       SF_GLOW = 24, SF_GHIGH = 38, SF_ROWS = 52 };
enum { BF_A0 = 0, BF_A1, BF_A2, BF_A3, BF_A4, BF_A5, BF_H1, BF_H2, BF_H3, BF_H4, BF_SIZE };
enum { GF_SIZE = 14 };  // rows of one range's Gibbs block: c_k hi at 2k, lo at 2k + 1

// gather entry: reaction index * 16 + (nu + 8); the FP64 kernel reads the
// stoichiometric factor back from kNuOf[] (no integer-to-double conversion),
// the mixed kernels form it from the entry's bits (nu_of_code)
__host__ __device__ inline int gather_pack(int r, int nu) { return r * 16 + (nu + 8); }
__constant__ double kNuOf[16] = {0, 0, 0, 0, 0, 0, -2.0, -1.0, 0, 1.0, 2.0, 0, 0, 0, 0, 0};

// The network's weights in MMA fragment order for inference inside the solver
// (the weights are the A operand of m16n8k16, 16 output units per tile; the
// cells are the columns of B): for tile (mt, kt) lane l holds the four 32-bit
// words a0..a3 of the A layout of the PTX ISA, BF16 pairs of
//   a0: W[16 mt + g][16 kt + 2 q + {0, 1}]      a1: the same for row g + 8
//   a2: W[16 mt + g][16 kt + 8 + 2 q + {0, 1}]  a3: the same for row g + 8
// with g = l / 4, q = l % 4, so that one 16-byte load per lane fetches a tile.
struct MlpFrag {
  const uint4* W2;   // [4 mt][4 kt][32 lanes]
  const uint4* W3;   // [mt3][4 kt][32 lanes], rows = outputs (cp/R, H/R, S/R of each species)
  const float2* b2;  // [4 mt][32 lanes]: b2 of rows 16 mt + g and 16 mt + g + 8
  const float4* o3;  // [mt3][32 lanes]: (scale, offset) of the same two rows of layer 3,
                     //   value = (W3 a2) * scale + offset, scale = std, offset = b3 std + mean
  const float2* w1;  // [64]: (W1, b1) of each hidden unit of layer 1
  int mt3;           // m-tiles of W3 packed: 3S output rows rounded up to 16
};

// Inference weights: W2 and W3 rows in BF16 (row-major [out][in]: a row of W
// is a column of the MMA's B operand, so B fragments are direct 32-bit loads),
// W1, b1, b2, b3, mean, std in FP32 (the batched evaluation kernel); and the
// same network in fragment order (the solver kernels).
struct MlpInfer {
  const __nv_bfloat16* W2;  // [64][64]
  const __nv_bfloat16* W3;  // [n_out][64]
  const float* W1;          // [64]
  const float* b1;          // [64]
  const float* b2;          // [64]
  const float* b3;          // [n_out]
  const float* mean;        // [n_out]
  const float* stdv;        // [n_out]
  int n_out;                // padded to a multiple of 8
  int n_valid;              // 3S: columns written to the caller's array
  MlpFrag frag;
};



// Everything a launch needs, passed by value.
struct Launch {
  // mechanism
  int S, R, Rrev, n_gather;
  const double* sp_tab;   // [S][SP_STRIDE]
  const double* rx_tab;   // [R][RX_STRIDE]
  const int4* rx_idx;     // [R]
  const int4* rx_idx_m;   // [R] the same for the mixed kernels, an unused slot = S
  const int* g_ptr;       // [S+1] species-major gather lists
  const int* g_ent;       // [n_gather]
  const double* dft_tw;   // [n_hi_bins][2][dft_n]: cos, sin of -2 pi j m / N
  const float* sp_tab_f;  // [SF_ROWS][S]           (mixed kernel)
  const float4* rx_tab_f; // [R] lg2 A, beta, Ea/R log2 e, dN (mixed kernel)
  const float* dft_tw_f;  // float twiddles          (mixed kernel)
  // general rate laws (real stoichiometry and orders, e.g. Eqs. 26-29): per
  // reaction nu then order of the slots a0, a1, p0, p1 (distinct species,
  // unused slots 0), and the real nu of every gather entry
  int general;
  const double* rg_tab;   // [R][8]
  const double* g_nu;     // [n_gather]
  const float* rg_tab_f;  // [R][8]       (mixed kernel)
  const float* g_nu_f;    // [n_gather]   (mixed kernel)
  int n_hi_bins;
  // options (Secs. 2.1-2.3)
  int dft_n, dft_on, max_iters;
  double y_step_max, delta_max, alpha, tol_ring, tol_freq, r_fac, rof_min;
  double ln_patm_over_ru;  // ln(P_atm / R_u)
  // work
  long long n_cells;
  double dt;
  const double* T;        // [n]
  const double* P;        // [n]
  const double* Y;        // [n][S] if !y_soa else [S][n]
  double* T_out;          // [n]
  double* Y_out;          // same layout as Y
  int* iters;             // [n]
  unsigned char* status;  // [n]
  int y_soa;
  unsigned long long* counter;  // next unclaimed cell
  // batched launches: nb > 0 batches, cell id c belongs to the batch b with
  // boff[b] <= c < boff[b+1]; the single-batch fields above are then unused
  int nb;
  const long long* boff;  // [nb+1]
  const BatchDesc* bdesc; // [nb]
  // serving (resident kernel fed by the host): ids below ctl->published are
  // claimable; the request of an id is found among the newest serve_q slots;
  // the last finished cell of a request writes its slot key to smail
  // (host-mapped, one word per slot, then one error word)
  int serve;
  ServeCtl* ctl;
  ServeSlot* slots;
  volatile long long* smail;
  int serve_q;
  long long idle_ns;      // the kernel leaves once every warp has been idle this long
  int serve_warps;        // warps in the grid
  // the options in FP32 for the mixed kernels (converted once, not per use)
  float y_step_max_f, alpha_f, tol_ring_f, tol_freq_f, r_fac_f, inv_r_fac_f, rof_min_f;
  MlpInfer mlp;           // thermo network (mixed kernel, thermo = MLP)
  int mlp_needed;         // network output rows the solver reads: S (cp/R) or 2S (and H/R)
  int mlp_h;              // 1: H/RT from the network as well
};

constexpr double kMlpTLow = 300.0, kMlpTHigh = 3000.0;  // network's training range (K)

// Shared-memory footprint of the tables (bytes, 16-byte aligned); general
// rate laws add their per-reaction and per-gather-entry tables at the end.
__host__ __device__ inline size_t table_smem_bytes(int S, int R, int n_gather, int n_hi_bins,
                                                   int dft_n, int general = 0) {
  size_t b = (size_t)S * SP_STRIDE * 8 + (size_t)R * RX_STRIDE * 8 + (size_t)R * 16 +
             (size_t)n_hi_bins * 2 * dft_n * 8 + (size_t)(S + 1 + n_gather) * 4;
  b = (b + 15) & ~(size_t)15;
  if (general) b += (size_t)R * 8 * 8 + (((size_t)n_gather * 8 + 15) & ~(size_t)15);
  return b;
}

// Shared-memory footprint of one resident cell in the FP64 kernel: Y, C, G/RT,
// H/RT (S each), effective rates (R), history [N][Rrev] and rOF (Rrev).
__host__ __device__ inline size_t cell_smem_bytes_fp64(int S, int R, int Rrev, int dft_n) {
  size_t b = ((size_t)4 * S + R + (size_t)dft_n * Rrev + Rrev) * 8;
  return (b + 15) & ~(size_t)15;
}

__host__ __device__ inline size_t table_smem_bytes_mixed(int S, int R, int n_gather, int n_hi_bins,
                                                         int dft_n, int general = 0) {
  size_t b = (size_t)R * 16 + (size_t)R * 16 + (size_t)S * SF_ROWS * 4 +
             (size_t)n_hi_bins * 2 * dft_n * 4 + (size_t)(S + 1 + n_gather) * 4;
  b = (b + 15) & ~(size_t)15;
  if (general) b += (size_t)R * 8 * 4 + (((size_t)n_gather * 4 + 15) & ~(size_t)15);
  return b;
}

// Mixed kernel cell: the Gibbs terms g2 as float pairs (S + 1: the last is
// the unused-slot entry), Y as float pairs in two arrays (hi, lo), C (S + 1)
// and H/RT (S), rates (R), history [Rrev][N | 1] and rOF (Rrev) in FP32.
// With the thermo network the rate array also holds, at the start of each
// step before the rates are computed, the cell's network activations and
// outputs (mixed_q_len).
__host__ __device__ inline int mixed_q_len(int S, int R, bool mlp) {
  // network scratch: layer-1 and layer-2 activations (64 BF16 each = 64
  // floats' room), then the outputs cp/R and H/R (2S, whole 16-row tiles)
  const int net = 64 + (2 * S + 15) / 16 * 16;
  return mlp ? (R > net ? R : net) : R;
}
__host__ __device__ inline size_t cell_smem_bytes_mixed(int S, int R, int Rrev, int dft_n,
                                                       bool mlp = false) {
  size_t b = (size_t)8 * (S + 1) +
             ((size_t)4 * S + 1 + mixed_q_len(S, R, mlp) + (size_t)(dft_n | 1) * Rrev + Rrev) * 4;
  return (b + 15) & ~(size_t)15;
}
}  // namespace stev
