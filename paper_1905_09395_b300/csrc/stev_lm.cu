// Linear algebra of the Levenberg-Marquardt trainer (Sec. 3: the thermo
// network is fitted with the Levenberg-Marquardt algorithm) on the library's
// own kernels:
//   gram_tf32   G = X X^T for the transposed Jacobian X = J^T ([params][rows]):
//               the Gauss-Newton matrix J^T J, on the 5th-generation tensor
//               cores (tcgen05.mma kind::tf32, FP32 accumulators in tensor
//               memory), operand tiles brought into shared memory by TMA;
//   rows_dot    g = X r: the gradient J^T r, one warp per row of X;
//   damped_cg   (A + lambda diag(A) + eps I) x = b by conjugate gradients with
//               the Jacobi preconditioner, the matrix-vector product one warp
//               per row of A, dot products reduced in a fixed order.
//
// Gram kernel layout.  One CTA of 4 warps per 128 x 256 tile of G (rows ti,
// columns tj; the column blocks of a row block run up to its diagonal).  The
// K dimension (the rows of J) runs in blocks of 32 FP32 values (128 bytes, the
// 128-byte swizzle of the TMA and of the MMA's shared-memory descriptors)
// through a 4-stage ring of 48 KB (A: 128 rows, B: 256 rows in two TMA
// boxes): warp 0 issues the TMA loads, warp 1 the MMAs (one thread each;
// 4 MMAs of M = 128, N = 256, K = 8 per block), and all four warps read the
// 128 x 256 FP32 accumulator back from tensor memory (warp w: lanes 32w ..
// 32w + 31) and store every element on or below the diagonal twice, as
// G[r][c] and G[c][r], so G is full and exactly symmetric.  A 256-column B
// tile reads each A row block half as often as square 128 x 128 tiles do
// (measured at 10,624 x 49,152: 10.4 ms against 11.5 ms with square tiles
// and six stages, 14.1 ms with four).  Every wait is bounded by time; on a
// timeout the kernel records it in *err, waits (bounded) for the loads it
// issued, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "stev_internal.h"

namespace stev {
namespace lm {

constexpr int kTile = 128;          // M of the MMA: rows of a tile (the A operand)
constexpr int kTileN = 256;         // N of the MMA: columns of a tile (the B operand)
constexpr int kKBlock = 32;         // FP32 values per 128-byte row of a stage
constexpr int kStages = 4;
constexpr int kStageBytes = kTile * kKBlock * 4;   // 16 KB: A, and each half of B
constexpr int kStageBytesB = kTileN * kKBlock * 4; // 32 KB
constexpr int kGramThreads = 128;
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait
// dynamic shared memory: 1024-byte alignment slack, A and B rings, barriers
constexpr size_t kGramSmem = 1024 + kStages * (kStageBytes + kStageBytesB) + 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// Waits for the phase with parity `parity` of the barrier to complete; false
// after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = now_ns();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (now_ns() - t0 > kWaitNs) return false;
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with the 128-byte swizzle: 8-row atoms of 128-byte rows, 1024 bytes apart
// (stride byte offset), the start address advanced by 32 bytes per K = 8
// step inside the atom; descriptor version 1, swizzle mode 2 (128 bytes).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor of kind::tf32: D in FP32, A and B TF32, both
// K-major, M = 128, N = 256.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTileN >> 3) << 17) |
                                ((uint32_t)(kTile >> 4) << 24);

__device__ __forceinline__ void umma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(kIdescTf32), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (one lane per thread)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// Tiles before row block ti: row block t (128 rows) holds the column blocks
// tj = 0 .. t / 2 (256 columns) that reach the diagonal, so C(2m) = m (m + 1)
// and C(2m + 1) = (m + 1)^2.
__host__ __device__ __forceinline__ long long tiles_before(long long ti) {
  const long long m = ti / 2;
  return (ti & 1) ? (m + 1) * (m + 1) : m * (m + 1);
}
// Tile (ti, tj) of the lower triangle from the linear tile index.
__device__ __forceinline__ void tile_of(int t, int& ti, int& tj) {
  int i = (int)(2.0 * sqrt((double)t));
  while (i > 0 && tiles_before(i) > t) --i;
  while (tiles_before(i + 1) <= t) ++i;
  ti = i;
  tj = (int)(t - tiles_before(i));
}

__global__ void __launch_bounds__(kGramThreads, 1)
    gram_tf32_kernel(const __grid_constant__ CUtensorMap xmap, int n, long long k, float* __restrict__ G,
                     long long ldg, int* __restrict__ err) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char* sa = base;                                  // [kStages][128][32] FP32
  unsigned char* sb = base + kStages * kStageBytes;          // [kStages][256][32] FP32
  uint64_t* bars = reinterpret_cast<uint64_t*>(sb + kStages * kStageBytesB);
  // bars[0 .. S-1] full, [S .. 2S-1] empty, [2S] done; the TMEM address after
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 1);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ti, tj;
  tile_of(blockIdx.x, ti, tj);
  const int nk = (int)((k + kKBlock - 1) / kKBlock);

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < 2 * kStages + 1; ++s) mbar_init(smem_u32(bars + s), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kTileN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;  // producer: blocks whose loads were issued
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      if (kb >= kStages && !mbar_wait(smem_u32(bars + kStages + s), ((kb / kStages) - 1) & 1)) {
        atomicExch(&s_fail, 1);
        break;
      }
      if (*(volatile int*)&s_fail) break;
      const uint32_t full = smem_u32(bars + s);
      mbar_expect_tx(full, kStageBytes + kStageBytesB);
      tma_load_2d(smem_u32(sa + s * kStageBytes), &xmap, kb * kKBlock, ti * kTile, full);
      tma_load_2d(smem_u32(sb + s * kStageBytesB), &xmap, kb * kKBlock, tj * kTileN, full);
      tma_load_2d(smem_u32(sb + s * kStageBytesB + kStageBytes), &xmap, kb * kKBlock,
                  tj * kTileN + kTile, full);
      issued = kb + 1;
    }
  } else if (warp == 1 && lane == 0) {
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % kStages;
      if (!mbar_wait(smem_u32(bars + s), (kb / kStages) & 1)) {
        atomicExch(&s_fail, 1);
        break;
      }
      tc_fence_after();
      const uint32_t a0 = smem_u32(sa + s * kStageBytes), b0 = smem_u32(sb + s * kStageBytesB);
#pragma unroll
      for (int kk = 0; kk < kKBlock / 8; ++kk)
        umma_tf32(tmem, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), (kb | kk) != 0);
      umma_commit(smem_u32(bars + kStages + s));  // the stage is free once these MMAs are done
    }
    umma_commit(smem_u32(bars + 2 * kStages));    // the accumulator is complete
  }
  __syncwarp();
  // epilogue: every thread reads its row of the tile (TMEM lane 32 w + lane)
  const bool done = mbar_wait(smem_u32(bars + 2 * kStages), 0);
  tc_fence_after();
  if (done && !*(volatile int*)&s_fail) {
    const int r = ti * kTile + warp * 32 + lane;
    const int cmax = min(r, n - 1);  // G[r][c] for c <= r, and its mirror
    for (int c0 = 0; c0 < kTileN; c0 += 32) {
      const int cb = tj * kTileN + c0;
      if (cb > ti * kTile + kTile - 1) break;  // warp-uniform: past every row's diagonal
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (r < n) {
        // mirror (coalesced: consecutive lanes, consecutive rows of G^T)
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (cb + j <= cmax) G[(long long)(cb + j) * ldg + r] = v[j];
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (cb + j < cmax) G[(long long)r * ldg + cb + j] = v[j];
      }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
  }
  // a failed producer / consumer pair: wait (bounded) for the loads issued
  // but not consumed, so that no copy lands after the CTA has left
  if (warp == 0 && lane == 0 && *(volatile int*)&s_fail) {
    for (int kb = max(0, issued - kStages); kb < issued; ++kb)
      mbar_wait(smem_u32(bars + kb % kStages), (kb / kStages) & 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTileN)
                 : "memory");
  }
}

// g[p] = sum_j X[p][j] r[j]: one warp per row, lanes over j (float4), the
// lane sums added in a fixed butterfly order.
__global__ void rows_dot_kernel(const float* __restrict__ X, long long n, long long k,
                                long long ldx, const float* __restrict__ r, float* __restrict__ g) {
  const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* x = X + row * ldx;
  float acc = 0.0f;
  const long long k4 = (k / 4) * 4;
  for (long long j = (long long)lane * 4; j < k4; j += 128) {
    const float4 a = *reinterpret_cast<const float4*>(x + j);
    const float4 b = *reinterpret_cast<const float4*>(r + j);
    acc = fmaf(a.x, b.x, acc);
    acc = fmaf(a.y, b.y, acc);
    acc = fmaf(a.z, b.z, acc);
    acc = fmaf(a.w, b.w, acc);
  }
  for (long long j = k4 + lane; j < k; j += 32) acc = fmaf(x[j], r[j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) g[row] = acc;
}

// The conjugate-gradient solver's scalars live on the device, so that its
// steps are queued without a host round trip each: every kernel of a step
// reads `done` first and does nothing once the solve has stopped.
struct CgState {
  double rz;     // r . z of the current direction
  double r0;     // |r| at the start
  double rtol;   // stop once |r| <= rtol r0
  float alpha, beta;
  int done;      // converged, or a direction of non-positive curvature
  int it;        // steps completed
};

// y = (A + lambda diag(A) + eps I) p, one warp per row (A symmetric, row-major).
// vec: the rows of A are 16-byte aligned (A aligned, lda a multiple of 4) and
// are read as float4 (p, a work array, always is).
__global__ void damped_symv_kernel(const float* __restrict__ A, long long n, long long lda,
                                   float lambda, float eps, const float* __restrict__ p,
                                   float* __restrict__ y, bool vec, const CgState* cs) {
  if (cs->done) return;
  const long long row = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* a = A + row * lda;
  float acc = 0.0f;
  const long long n4 = vec ? (n / 4) * 4 : 0;
  for (long long j = (long long)lane * 4; j < n4; j += 128) {
    const float4 v = *reinterpret_cast<const float4*>(a + j);
    const float4 q = *reinterpret_cast<const float4*>(p + j);
    acc = fmaf(v.x, q.x, acc);
    acc = fmaf(v.y, q.y, acc);
    acc = fmaf(v.z, q.z, acc);
    acc = fmaf(v.w, q.w, acc);
  }
  for (long long j = n4 + lane; j < n; j += 32) acc = fmaf(a[j], p[j], acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[row] = acc + (lambda * a[row] + eps) * p[row];
}

// Partial dot products in FP64, one per block (fixed order), then summed in
// block order by the step kernels below: part[2b] = sum x y, part[2b + 1] =
// sum x z (if z).
constexpr int kDotBlocks = 256, kDotThreads = 256;
__global__ void dot_partial_kernel(const float* __restrict__ x, const float* __restrict__ y,
                                   const float* __restrict__ z, long long n,
                                   double* __restrict__ part, const CgState* cs) {
  if (cs->done) return;
  __shared__ double s0[kDotThreads], s1[kDotThreads];
  double a = 0.0, b = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    a += (double)x[i] * (double)y[i];
    if (z) b += (double)x[i] * (double)z[i];
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s0[threadIdx.x] += s0[threadIdx.x + w];
      s1[threadIdx.x] += s1[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s0[0];
    part[2 * blockIdx.x + 1] = s1[0];
  }
}
__device__ __forceinline__ void sum_parts(const double* part, int nb, double& a, double& b) {
  a = 0.0;
  b = 0.0;
  for (int i = 0; i < nb; ++i) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
}
// start: rz = r . z, r0 = |r| (part from dot(r, z, r)); nothing to do if r0 = 0
__global__ void cg_start_kernel(const double* __restrict__ part, int nb, double rtol,
                                CgState* cs) {
  if (threadIdx.x != 0) return;
  double a, b;
  sum_parts(part, nb, a, b);
  cs->rz = a;
  cs->r0 = sqrt(b);
  cs->rtol = rtol;
  cs->it = 0;
  cs->done = !(cs->r0 > 0.0);
}
// alpha = rz / (p . q) (part from dot(p, q)); stop on non-positive curvature
__global__ void cg_alpha_kernel(const double* __restrict__ part, int nb, CgState* cs) {
  if (threadIdx.x != 0 || cs->done) return;
  double pq, unused;
  sum_parts(part, nb, pq, unused);
  if (!(pq > 0.0)) {
    cs->done = 1;  // stop with the current x
    return;
  }
  cs->alpha = (float)(cs->rz / pq);
}
// after the update: rz' = r . z, |r| (part from dot(r, z, r)); the step is
// complete; stop once |r| <= rtol r0, else beta = rz' / rz
__global__ void cg_beta_kernel(const double* __restrict__ part, int nb, CgState* cs) {
  if (threadIdx.x != 0 || cs->done) return;
  double rz1, rr;
  sum_parts(part, nb, rz1, rr);
  cs->it += 1;
  if (sqrt(rr) <= cs->rtol * cs->r0) {
    cs->done = 1;
    return;
  }
  cs->beta = (float)(rz1 / cs->rz);
  cs->rz = rz1;
}

// z = r / m, m = diag(A)(1 + lambda) + eps (the Jacobi preconditioner)
__global__ void precond_kernel(const float* __restrict__ A, long long n, long long lda, float lambda,
                               float eps, const float* __restrict__ r, float* __restrict__ z,
                               const CgState* cs) {
  if (cs->done) return;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = r[i] / (A[i * lda + i] * (1.0f + lambda) + eps);
}
// x += alpha p; r -= alpha q
__global__ void cg_update_kernel(long long n, const float* __restrict__ p,
                                 const float* __restrict__ q, float* __restrict__ x,
                                 float* __restrict__ r, const CgState* cs) {
  if (cs->done) return;
  const float alpha = cs->alpha;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    x[i] = fmaf(alpha, p[i], x[i]);
    r[i] = fmaf(-alpha, q[i], r[i]);
  }
}
// p = z + beta p
__global__ void cg_direction_kernel(long long n, const float* __restrict__ z,
                                    float* __restrict__ p, const CgState* cs) {
  if (cs->done) return;
  const float beta = cs->beta;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = fmaf(beta, p[i], z[i]);
}

}  // namespace lm

namespace host {

namespace {
typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}
}  // namespace

stev_status gram_tf32(const float* X, long long n, long long k, long long ldx, float* G,
                      long long ldg, int* d_err, cudaStream_t s) {
  if (n < 1 || k < 1) return fail(STEV_EINVAL, "gram: n and k must be >= 1");
  if (ldx < k || ldx % 4 != 0) return fail(STEV_EINVAL, "gram: ldx must be >= k and a multiple of 4");
  if (ldg < n) return fail(STEV_EINVAL, "gram: ldg must be >= n");
  if (reinterpret_cast<uintptr_t>(X) % 16 != 0) return fail(STEV_EINVAL, "gram: X must be 16-byte aligned");
  if (n > (1LL << 24) || k > (1LL << 31)) return fail(STEV_EINVAL, "gram: sizes too large");
  EncodeTiled enc = encode_fn();
  if (!enc) return fail(STEV_ECUDA, "cuTensorMapEncodeTiled is not available");
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)ldx * 4};
  const cuuint32_t box[2] = {(cuuint32_t)lm::kKBlock, (cuuint32_t)lm::kTile};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(STEV_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  const long long nt = (n + lm::kTile - 1) / lm::kTile;
  const long long tiles = lm::tiles_before(nt);
  cudaError_t e = cudaFuncSetAttribute(lm::gram_tf32_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lm::kGramSmem);
  if (e != cudaSuccess) return fail(STEV_ECUDA, "gram: %s", cudaGetErrorString(e));
  lm::gram_tf32_kernel<<<(unsigned)tiles, lm::kGramThreads, lm::kGramSmem, s>>>(map, (int)n, k, G, ldg,
                                                                                d_err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(STEV_ECUDA, "gram launch: %s", cudaGetErrorString(e));
  return STEV_OK;
}

stev_status rows_dot(const float* X, long long n, long long k, long long ldx, const float* r,
                     float* g, cudaStream_t s) {
  if (ldx % 4 != 0 || reinterpret_cast<uintptr_t>(X) % 16 || reinterpret_cast<uintptr_t>(r) % 16)
    return fail(STEV_EINVAL, "rows_dot: 16-byte aligned rows needed");
  const long long threads = n * 32;
  lm::rows_dot_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(X, n, k, ldx, r, g);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? STEV_OK : fail(STEV_ECUDA, "rows_dot: %s", cudaGetErrorString(e));
}

stev_status damped_cg(const float* A, long long n, long long lda, const float* b, double lambda,
                      double eps, float* x, int max_iters, double rtol, int* iters,
                      CgWork* w, cudaStream_t s) {
  if (n < 1 || lda < n || max_iters < 1 || !(rtol > 0.0))
    return fail(STEV_EINVAL, "damped_cg: bad arguments");
  const float lam = (float)lambda, ep = (float)eps;
  const bool vec = lda % 4 == 0 && reinterpret_cast<uintptr_t>(A) % 16 == 0;
  const unsigned vb = (unsigned)((n + 255) / 256), mb = (unsigned)((n * 32 + 255) / 256);
  float *r = w->r, *z = w->z, *p = w->p, *q = w->q;
  double* part = w->part;
  lm::CgState* cs = static_cast<lm::CgState*>(w->state);
  lm::CgState h{};
#define CG_TRY(expr)                                                                        \
  do {                                                                                      \
    const cudaError_t e_ = (expr);                                                          \
    if (e_ != cudaSuccess) return fail(STEV_ECUDA, "damped_cg: %s", cudaGetErrorString(e_)); \
  } while (0)
  // x = 0, r = b, z = M^-1 r, p = z; rz and r0 on the device
  CG_TRY(cudaMemsetAsync(cs, 0, sizeof(lm::CgState), s));
  CG_TRY(cudaMemsetAsync(x, 0, (size_t)n * 4, s));
  CG_TRY(cudaMemcpyAsync(r, b, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
  lm::precond_kernel<<<vb, 256, 0, s>>>(A, n, lda, lam, ep, r, z, cs);
  CG_TRY(cudaMemcpyAsync(p, z, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
  lm::dot_partial_kernel<<<lm::kDotBlocks, lm::kDotThreads, 0, s>>>(r, z, r, n, part, cs);
  lm::cg_start_kernel<<<1, 32, 0, s>>>(part, lm::kDotBlocks, rtol, cs);
  // steps queued kCgBatch at a time; the host reads the state once per batch
  // (a step queued after the solve stopped does nothing)
  constexpr int kCgBatch = 16;
  int queued = 0;
  do {
    const int k = std::min(kCgBatch, max_iters - queued);
    for (int j = 0; j < k; ++j) {
      lm::damped_symv_kernel<<<mb, 256, 0, s>>>(A, n, lda, lam, ep, p, q, vec, cs);
      lm::dot_partial_kernel<<<lm::kDotBlocks, lm::kDotThreads, 0, s>>>(p, q, nullptr, n, part, cs);
      lm::cg_alpha_kernel<<<1, 32, 0, s>>>(part, lm::kDotBlocks, cs);
      lm::cg_update_kernel<<<vb, 256, 0, s>>>(n, p, q, x, r, cs);
      lm::precond_kernel<<<vb, 256, 0, s>>>(A, n, lda, lam, ep, r, z, cs);
      lm::dot_partial_kernel<<<lm::kDotBlocks, lm::kDotThreads, 0, s>>>(r, z, r, n, part, cs);
      lm::cg_beta_kernel<<<1, 32, 0, s>>>(part, lm::kDotBlocks, cs);
      lm::cg_direction_kernel<<<vb, 256, 0, s>>>(n, z, p, cs);
    }
    queued += k;
    CG_TRY(cudaGetLastError());
    CG_TRY(cudaMemcpyAsync(&h, cs, sizeof h, cudaMemcpyDeviceToHost, s));
    CG_TRY(cudaStreamSynchronize(s));
  } while (!h.done && queued < max_iters);
#undef CG_TRY
  if (iters) *iters = h.it;
  return STEV_OK;
}

}  // namespace host
}  // namespace stev

// ------------------------------------------------------------- C ABI
namespace {
template <typename T>
T* dev_alloc(size_t count) {
  void* p = nullptr;
  return cudaMalloc(&p, count * sizeof(T)) == cudaSuccess ? static_cast<T*>(p) : nullptr;
}
}  // namespace

extern "C" stev_status stev_gram_tf32(long n, long k, const float* X, long ldx, float* G, long ldg,
                                      void* stream) {
  stev::host::clear_error();
  if (!X || !G) return stev::host::fail(STEV_EINVAL, "NULL array");
  // the error flag from the stream's memory pool: no device-wide
  // synchronisation, unlike cudaMalloc / cudaFree
  cudaStream_t s = (cudaStream_t)stream;
  int* d_err = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&d_err), sizeof(int), s) != cudaSuccess || !d_err)
    return stev::host::fail(STEV_ENOMEM, "cudaMallocAsync failed");
  stev_status st = STEV_OK;
  if (cudaMemsetAsync(d_err, 0, sizeof(int), s) != cudaSuccess)
    st = stev::host::fail(STEV_ECUDA, "cudaMemsetAsync failed");
  if (st == STEV_OK) st = stev::host::gram_tf32(X, n, k, ldx, G, ldg, d_err, s);
  int h_err = 0;
  if (st == STEV_OK && (cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
    st = stev::host::fail(STEV_ECUDA, "gram: %s", cudaGetErrorString(cudaGetLastError()));
  if (st == STEV_OK && h_err) st = stev::host::fail(STEV_ETIMEOUT, "gram: a pipeline wait timed out");
  cudaFreeAsync(d_err, s);
  return st;
}

extern "C" stev_status stev_damped_cg(long n, const float* A, long lda, const float* b, double lambda,
                                      double eps, float* x, int max_iters, double rtol, int* iters,
                                      void* stream) {
  stev::host::clear_error();
  if (!A || !b || !x) return stev::host::fail(STEV_EINVAL, "NULL array");
  if (n < 1) return stev::host::fail(STEV_EINVAL, "n must be >= 1");
  stev::host::CgWork w{};
  if (stev::host::cg_work_alloc(&w, n) != STEV_OK) return STEV_ENOMEM;
  const stev_status st = stev::host::damped_cg(A, n, lda, b, lambda, eps, x, max_iters, rtol, iters,
                                               &w, (cudaStream_t)stream);
  stev::host::cg_work_free(&w);
  return st;
}

namespace stev {
namespace host {
stev_status cg_work_alloc(CgWork* w, long long n) {
  *w = CgWork{};
  w->r = dev_alloc<float>((size_t)n);
  w->z = dev_alloc<float>((size_t)n);
  w->p = dev_alloc<float>((size_t)n);
  w->q = dev_alloc<float>((size_t)n);
  w->part = dev_alloc<double>(2 * lm::kDotBlocks);
  w->state = dev_alloc<lm::CgState>(1);
  if (!w->r || !w->z || !w->p || !w->q || !w->part || !w->state) {
    cg_work_free(w);
    return fail(STEV_ENOMEM, "cudaMalloc failed (conjugate-gradient work arrays)");
  }
  return STEV_OK;
}
void cg_work_free(CgWork* w) {
  cudaFree(w->r);
  cudaFree(w->z);
  cudaFree(w->p);
  cudaFree(w->q);
  cudaFree(w->part);
  cudaFree(w->state);
  *w = CgWork{};
}
}  // namespace host
}  // namespace stev
