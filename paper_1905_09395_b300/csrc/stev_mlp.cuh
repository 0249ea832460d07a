// Thermo network (Sec. 3: a neural network of temperature stands in for the
// NASA-7 species properties): training and inference kernels.
//
// Network: t = (T - 1650)/1350, a1 = tanh(W1 t + b1) [64],
// a2 = tanh(W2 a1 + b2) [64], y = W3 a2 + b3 [3S] standardised outputs
// (cp/R of every species, then H/R in K, then S/R), value = y * std + mean.
// Parameters are one flat FP32 array in the order W1[64], b1[64], W2[64][64],
// b2[64], W3[3S][64], b3[3S] (rows = outputs).
//
// Training (FP32, off the hot path): the forward pass, the mean-squared-error
// gradient and the weight gradients of a 64-sample tile are computed entirely
// in shared memory by one CTA and written as the tile's partial gradient; one
// cooperative launch runs every Adam step (tiles, grid barrier, update, grid
// barrier).
// Inference (BF16 weights and activations, FP32 accumulation): warp-level
// tensor-core MMAs m16n8k16, on 16 temperatures at a time (batched
// evaluation) or on the cells of one warp inside the solver's step.
#pragma once
#ifndef __CUDACC_RTC__  // the trainer is not part of the run-time compiled solver
#include <cooperative_groups.h>
#endif
#include <cuda_bf16.h>
#include "stev_device.cuh"

namespace stev {

constexpr int kHid = 64;

#ifndef __CUDACC_RTC__
// Grid-wide barrier of a cooperative launch (every CTA resident, so it cannot
// deadlock), with the memory ordering of a release / acquire at GPU scope.
__device__ __forceinline__ void grid_barrier() { cooperative_groups::this_grid().sync(); }
#endif
constexpr float kTMid = 1650.0f, kTHalf = 1350.0f;
constexpr int kMlpTile = 64;  // samples per CTA in training

__host__ __device__ inline int mlp_n_params(int n_out) {
  return kHid + kHid + kHid * kHid + kHid + n_out * kHid + n_out;
}
struct MlpOffsets {
  int W1, b1, W2, b2, W3, b3, total;
};
__host__ __device__ inline MlpOffsets mlp_offsets(int n_out) {
  MlpOffsets o;
  o.W1 = 0;
  o.b1 = o.W1 + kHid;
  o.W2 = o.b1 + kHid;
  o.b2 = o.W2 + kHid * kHid;
  o.W3 = o.b2 + kHid;
  o.b3 = o.W3 + n_out * kHid;
  o.total = o.b3 + n_out;
  return o;
}

// ----------------------------------------------------- training targets
// NASA-7 properties (Eqs. 15-16, S/R = H/RT - G/RT) of every species at every
// sample temperature, in FP64, stored as float: out[s][o], o = i (cp/R),
// S+i (H/R = H/RT * T, in K: smooth over the range, unlike H/RT whose a6/T
// term grows steeply at low T), 2S+i (S/R).
__global__ void mlp_targets_kernel(const double* __restrict__ sp_tab, int S,
                                   const double* __restrict__ T, long long n,
                                   float* __restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * S) return;
  const long long s = idx / S;
  const int i = (int)(idx - s * S);
  const double t = T[s];
  const double* sp = sp_tab + i * SP_STRIDE;
  const double* b = sp + (t < sp[SP_TSPLIT] ? SP_LOW : SP_HIGH);
  const double lnT = log(t), invT = 1.0 / t;
  const double cpR = fma(fma(fma(fma(b[B_A4], t, b[B_A3]), t, b[B_A2]), t, b[B_A1]), t, b[B_A0]);
  const double hp = fma(fma(fma(b[B_H4], t, b[B_H3]), t, b[B_H2]), t, b[B_H1]);
  const double hRT = fma(hp, t, b[B_A0]) + b[B_A5] * invT;
  const double gp = fma(fma(fma(b[B_G4], t, b[B_G3]), t, b[B_G2]), t, b[B_H1]);
  const double gRT = fma(b[B_A0], 1.0 - lnT, fma(b[B_A5], invT, -b[B_A6])) - gp * t;
  float* o = out + s * (3 * S);
  o[i] = (float)cpR;
  o[S + i] = (float)(hRT * t);
  o[2 * S + i] = (float)(hRT - gRT);
}

// Column sums and sums of squares (FP64) for standardisation: block
// (x, col) writes its partial pair to part[(col * gridDim.x + x) * 2]; the
// host adds the partials in order (no atomics: the result is reproducible).
__global__ void mlp_moments_kernel(const float* __restrict__ v, long long n, int m,
                                   double* __restrict__ part) {
  __shared__ double wa[32], wb[32];
  const int col = blockIdx.y;
  double a = 0.0, b = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    const double x = v[r * m + col];
    a += x;
    b += x * x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    wa[threadIdx.x >> 5] = a;
    wb[threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sa += wa[w];
      sb += wb[w];
    }
    double* o = part + ((size_t)col * gridDim.x + blockIdx.x) * 2;
    o[0] = sa;
    o[1] = sb;
  }
}

__global__ void mlp_standardise_kernel(float* __restrict__ v, long long n, int m,
                                       const float* __restrict__ mean,
                                       const float* __restrict__ inv_std) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * m) return;
  const int col = (int)(idx % m);
  v[idx] = (v[idx] - mean[col]) * inv_std[col];
}

// ------------------------------------------------ fused forward + backward
// One CTA of kMlpTile threads: thread s owns sample s of the tile.  Shared
// memory: the parameters, then feature-major activations a1, a2, dz1, dz2
// [64][tile+1] and dy [n_out][tile+1] (the +1 keeps rows on distinct banks).
// Writes the tile's d loss / d params to part[blockIdx.x][params] and its sum
// of squared errors to loss_part[blockIdx.x] (the loss is the mean over
// n_total samples and n_out outputs); mlp_train_kernel / mlp_sum_kernel add
// the tiles in order, so training is reproducible run to run.
// The tile's work as a device function: tile `tile` of the n samples, shared
// memory sm (mlp_grad_smem_bytes) and se_w (kMlpTile / 32 doubles).  The
// parameters are read around L1 (__ldcg): the persistent trainer rewrites
// them between tiles.
__device__ __forceinline__ void mlp_grad_tile(
    const float* __restrict__ params, int n_out, const double* __restrict__ T,
    const float* __restrict__ target, long long n, long long n_total, float* __restrict__ part,
    double* __restrict__ loss_part, int tile, float* sm, double* se_w) {
  const MlpOffsets off = mlp_offsets(n_out);
  float* P = sm;
  const int ld = kMlpTile + 1;
  float* a1 = P + off.total;
  float* a2 = a1 + kHid * ld;
  float* z1 = a2 + kHid * ld;   // dz1
  float* z2 = z1 + kHid * ld;   // dz2
  float* dy = z2 + kHid * ld;   // [n_out][ld]
  float* ts = dy + n_out * ld;  // [tile]
  for (int k = threadIdx.x; k < off.total; k += blockDim.x) P[k] = __ldcg(params + k);
  const long long s0 = (long long)tile * kMlpTile;
  const int s = threadIdx.x;
  const bool valid = s0 + s < n;
  __syncthreads();

  // forward
  const float t = valid ? ((float)T[s0 + s] - kTMid) / kTHalf : 0.0f;
  ts[s] = t;
  for (int j = 0; j < kHid; ++j) a1[j * ld + s] = tanhf(fmaf(P[off.W1 + j], t, P[off.b1 + j]));
  for (int j = 0; j < kHid; ++j) {
    float acc = P[off.b2 + j];
    for (int k = 0; k < kHid; ++k) acc = fmaf(P[off.W2 + j * kHid + k], a1[k * ld + s], acc);
    a2[j * ld + s] = tanhf(acc);
  }
  const float scale = 2.0f / (float)((double)n_total * n_out);
  double se = 0.0;
  for (int o = 0; o < n_out; ++o) {
    float acc = P[off.b3 + o];
    for (int k = 0; k < kHid; ++k) acc = fmaf(P[off.W3 + o * kHid + k], a2[k * ld + s], acc);
    const float d = valid ? acc - target[(s0 + s) * n_out + o] : 0.0f;
    se += (double)d * d;
    dy[o * ld + s] = d * scale;
  }
  // backward through the activations
  for (int j = 0; j < kHid; ++j) {
    float acc = 0.0f;
    for (int o = 0; o < n_out; ++o) acc = fmaf(P[off.W3 + o * kHid + j], dy[o * ld + s], acc);
    const float a = a2[j * ld + s];
    z2[j * ld + s] = acc * (1.0f - a * a);
  }
  for (int j = 0; j < kHid; ++j) {
    float acc = 0.0f;
    for (int o = 0; o < kHid; ++o) acc = fmaf(P[off.W2 + o * kHid + j], z2[o * ld + s], acc);
    const float a = a1[j * ld + s];
    z1[j * ld + s] = acc * (1.0f - a * a);
  }
  for (int o = 16; o > 0; o >>= 1) se += __shfl_xor_sync(0xffffffffu, se, o);
  if ((threadIdx.x & 31) == 0) se_w[threadIdx.x >> 5] = se;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kMlpTile / 32; ++w) t += se_w[w];
    loss_part[tile] = t;
  }

  // weight gradients: sums over the tile's samples
  const int nt = (int)min((long long)kMlpTile, n - s0);
  for (int k = threadIdx.x; k < off.total; k += blockDim.x) {
    float acc = 0.0f;
    if (k < off.b1) {                       // W1[j], input t
      const int j = k - off.W1;
      for (int q = 0; q < nt; ++q) acc = fmaf(z1[j * ld + q], ts[q], acc);
    } else if (k < off.W2) {                // b1
      const int j = k - off.b1;
      for (int q = 0; q < nt; ++q) acc += z1[j * ld + q];
    } else if (k < off.b2) {                // W2[j][i]
      const int j = (k - off.W2) / kHid, i = (k - off.W2) % kHid;
      for (int q = 0; q < nt; ++q) acc = fmaf(z2[j * ld + q], a1[i * ld + q], acc);
    } else if (k < off.W3) {                // b2
      const int j = k - off.b2;
      for (int q = 0; q < nt; ++q) acc += z2[j * ld + q];
    } else if (k < off.b3) {                // W3[o][i]
      const int o = (k - off.W3) / kHid, i = (k - off.W3) % kHid;
      for (int q = 0; q < nt; ++q) acc = fmaf(dy[o * ld + q], a2[i * ld + q], acc);
    } else {                                // b3
      const int o = k - off.b3;
      for (int q = 0; q < nt; ++q) acc += dy[o * ld + q];
    }
    part[(size_t)tile * off.total + k] = acc;
  }
  __syncthreads();  // the tile's shared memory is reused by the caller's next tile
}

__global__ void __launch_bounds__(kMlpTile) mlp_grad_kernel(
    const float* __restrict__ params, int n_out, const double* __restrict__ T,
    const float* __restrict__ target, long long n, long long n_total, float* __restrict__ part,
    double* __restrict__ loss_part) {
  __shared__ double se_w[kMlpTile / 32];
  extern __shared__ __align__(16) float sm[];
  mlp_grad_tile(params, n_out, T, target, n, n_total, part, loss_part, blockIdx.x, sm, se_w);
}

// grad[k] = sum over tiles of part[tile][k], tiles in order; thread 0 also
// adds the tiles' squared errors, in order, to *loss_acc.
__global__ void mlp_sum_kernel(const float* __restrict__ part, int tiles, int n,
                               const double* __restrict__ loss_part, float* __restrict__ grad,
                               double* __restrict__ loss_acc) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) {
    double t = 0.0;
    for (int b = 0; b < tiles; ++b) t += loss_part[b];
    *loss_acc += t;
  }
  if (k >= n) return;
  float g = 0.0f;
  for (int b = 0; b < tiles; ++b) g += part[(size_t)b * n + k];
  grad[k] = g;
}

__host__ __device__ inline size_t mlp_grad_smem_bytes(int n_out) {
  return ((size_t)mlp_n_params(n_out) + (size_t)(4 * kHid + n_out) * (kMlpTile + 1) + kMlpTile) *
         sizeof(float);
}

#ifndef __CUDACC_RTC__
// Every Adam step (Kingma & Ba 2015) of a training run in one cooperative
// launch (all CTAs resident; grid-wide barriers between the phases).  Per
// step: the minibatch's tiles (grid-stride over CTAs, each tile by
// mlp_grad_tile), a barrier, then Adam on every parameter, its gradient the
// sum of the tile partials in tile order (one thread adds the tiles' squared
// errors, in order, to the epoch's loss), a barrier.  sched[step] = (step
// size, 1 - b1^t, 1 - b2^t) as the host computes them.  The same inputs train
// the same network bit for bit.  Reads of data other CTAs wrote go around L1.
__global__ void __launch_bounds__(kMlpTile) mlp_train_kernel(
    float* __restrict__ p, int n_out, const double* __restrict__ T,
    const float* __restrict__ target, long long n, int batch, const float4* __restrict__ sched,
    long long steps, long long per_epoch, float* __restrict__ part, double* __restrict__ loss_part,
    float* __restrict__ m1, float* __restrict__ m2, double* __restrict__ loss_epoch, float beta1,
    float beta2, float eps) {
  __shared__ double se_w[kMlpTile / 32];
  extern __shared__ __align__(16) float sm[];
  const int np = mlp_n_params(n_out);
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  for (long long step = 0; step < steps; ++step) {
    const long long ep = step / per_epoch;
    const long long s0 = (step - ep * per_epoch) * batch;
    const long long nb = min((long long)batch, n - s0);
    const int tiles = (int)((nb + kMlpTile - 1) / kMlpTile);
    for (int t = blockIdx.x; t < tiles; t += gridDim.x)
      mlp_grad_tile(p, n_out, T + s0, target + s0 * n_out, nb, nb, part, loss_part, t, sm, se_w);
    grid_barrier();
    const float4 sc = sched[step];
    if (gtid == 0) {
      double acc = 0.0;
      for (int b = 0; b < tiles; ++b) acc += __ldcg(loss_part + b);
      loss_epoch[ep] += acc;
    }
    for (long long k = gtid; k < np; k += nthreads) {
      float gk = 0.0f;
      for (int b = 0; b < tiles; ++b) gk += __ldcg(part + (size_t)b * np + k);
      const float a = beta1 * m1[k] + (1.0f - beta1) * gk;
      const float bb = beta2 * m2[k] + (1.0f - beta2) * gk * gk;
      m1[k] = a;
      m2[k] = bb;
      p[k] -= sc.x * (a / sc.y) / (sqrtf(bb / sc.z) + eps);
    }
    grid_barrier();
  }
}
#endif

// --------------------------------------- Levenberg-Marquardt (Sec. 3)
// Jacobian of the standardised outputs with respect to every parameter and
// the residuals y - target, one CTA per sample, written TRANSPOSED: Jt
// [n_params][ldk], column s * n_out + o holds d y_o(sample s) / d param, so
// that each parameter's row is contiguous in the samples (the K-major operand
// of the Gram kernel, and one coalesced segment of n_out values per parameter
// and sample).  With d2_oj = W3[o][j] (1 - a2_j^2) and
// d1_ok = (1 - a1_k^2) sum_j W2[j][k] d2_oj the entries are
//   W1[k]: d1_ok t,  b1[k]: d1_ok,  W2[j][k]: d2_oj a1_k,  b2[j]: d2_oj,
//   W3[o'][k]: a2_k if o' == o else 0,  b3[o']: 1 if o' == o else 0.
// Shared memory: a1, a2 [64], d2 and d1 [n_out][64] (mlp_jacobian_smem_bytes).
constexpr int kJacThreads = 256;
__host__ __device__ inline size_t mlp_jacobian_smem_bytes(int n_out) {
  return ((size_t)2 * kHid + (size_t)2 * n_out * kHid) * sizeof(float);
}
__global__ void __launch_bounds__(kJacThreads) mlp_jacobian_t_kernel(
    const float* __restrict__ params, int n_out, const double* __restrict__ T,
    const float* __restrict__ target, float* __restrict__ Jt, long long ldk,
    float* __restrict__ resid) {
  extern __shared__ __align__(16) float jsm[];
  float* a1 = jsm;
  float* a2 = a1 + kHid;
  float* d2 = a2 + kHid;               // [n_out][64]
  float* d1 = d2 + (size_t)n_out * kHid;  // [n_out][64]
  const MlpOffsets off = mlp_offsets(n_out);
  const int s = blockIdx.x, tid = threadIdx.x;
  const float t = ((float)T[s] - kTMid) / kTHalf;
  if (tid < kHid) a1[tid] = tanhf(fmaf(params[off.W1 + tid], t, params[off.b1 + tid]));
  __syncthreads();
  if (tid < kHid) {
    float acc = params[off.b2 + tid];
    for (int i = 0; i < kHid; ++i) acc = fmaf(params[off.W2 + tid * kHid + i], a1[i], acc);
    a2[tid] = tanhf(acc);
  }
  __syncthreads();
  for (int o = tid; o < n_out; o += blockDim.x) {
    float y = params[off.b3 + o];
    for (int j = 0; j < kHid; ++j) y = fmaf(params[off.W3 + o * kHid + j], a2[j], y);
    resid[(size_t)s * n_out + o] = y - target[(size_t)s * n_out + o];
  }
  for (int q = tid; q < n_out * kHid; q += blockDim.x) {
    const int o = q / kHid, j = q % kHid;
    d2[q] = params[off.W3 + o * kHid + j] * (1.0f - a2[j] * a2[j]);
  }
  __syncthreads();
  for (int q = tid; q < n_out * kHid; q += blockDim.x) {
    const int o = q / kHid, k = q % kHid;
    float g = 0.0f;
    for (int j = 0; j < kHid; ++j) g = fmaf(params[off.W2 + j * kHid + k], d2[o * kHid + j], g);
    d1[q] = g * (1.0f - a1[k] * a1[k]);
  }
  __syncthreads();
  float* col = Jt + (size_t)s * n_out;
  const long long total = (long long)off.total * n_out;
  for (long long q = tid; q < total; q += blockDim.x) {
    const int p = (int)(q / n_out), o = (int)(q % n_out);
    float v;
    if (p < off.b1) {
      v = d1[o * kHid + (p - off.W1)] * t;
    } else if (p < off.W2) {
      v = d1[o * kHid + (p - off.b1)];
    } else if (p < off.b2) {
      const int j = (p - off.W2) / kHid, k = (p - off.W2) % kHid;
      v = d2[o * kHid + j] * a1[k];
    } else if (p < off.W3) {
      v = d2[o * kHid + (p - off.b2)];
    } else if (p < off.b3) {
      const int oo = (p - off.W3) / kHid, k = (p - off.W3) % kHid;
      v = (oo == o) ? a2[k] : 0.0f;
    } else {
      v = (p - off.b3 == o) ? 1.0f : 0.0f;
    }
    col[(size_t)p * ldk + o] = v;
  }
}

// Squared error of each sample (FP32 forward, FP64 sum over its outputs).
__global__ void mlp_sqerr_kernel(const float* __restrict__ params, int n_out,
                                 const double* __restrict__ T, const float* __restrict__ target,
                                 long long n, double* __restrict__ se) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const MlpOffsets off = mlp_offsets(n_out);
  const float t = ((float)T[s] - kTMid) / kTHalf;
  float a1[kHid], a2[kHid];
  for (int k = 0; k < kHid; ++k) a1[k] = tanhf(fmaf(params[off.W1 + k], t, params[off.b1 + k]));
  for (int j = 0; j < kHid; ++j) {
    float acc = params[off.b2 + j];
    for (int k = 0; k < kHid; ++k) acc = fmaf(params[off.W2 + j * kHid + k], a1[k], acc);
    a2[j] = tanhf(acc);
  }
  double e = 0.0;
  for (int o = 0; o < n_out; ++o) {
    float y = params[off.b3 + o];
    for (int j = 0; j < kHid; ++j) y = fmaf(params[off.W3 + o * kHid + j], a2[j], y);
    const double d = (double)y - (double)target[s * n_out + o];
    e += d * d;
  }
  se[s] = e;
}

// p_new = p - d
__global__ void mlp_step_kernel(const float* __restrict__ p, const float* __restrict__ d, int n,
                                float* __restrict__ p_new) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) p_new[k] = p[k] - d[k];
}

// ------------------------------------------------------------- inference
__device__ __forceinline__ float tanh_approx(float x) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_bf16_16816(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

// m16n8k16 with the A fragment as one 16-byte word per lane (fragment-ordered
// weights, MlpFrag).
__device__ __forceinline__ void mma_bf16_16816_a(float* d, uint4 a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b[0]), "r"(b[1]));
}

// Offsets (32-bit words) in a cell's network scratch: layer-1 activations
// (64 BF16), layer-2 activations (64 BF16), then the outputs (FP32 rows).
constexpr int kNetH1Off = 0, kNetH2Off = 32, kNetOutOff = 64;

// The network of every cell a warp holds, inside the solver's step (Sec. 3:
// the network stands in for the NASA-7 evaluation).  The warp holds CPW =
// 32 / G cells (lane groups of G); column c of the MMAs' B operand carries
// cell c mod CPW, and the weights are the A operand (16 output units per
// tile), so a cell's layer 2 is 16 MMAs and each 16 output rows of layer 3
// four more, whatever CPW.  t: this lane's cell's scaled temperature
// (T - 1650) / 1350.  q0: the network scratch of the warp's first cell
// (kNet*Off), cell k's at q0 + k * cell_ld (32-bit words); rows
// 0 .. n_rows - 1 of each cell's outputs (cp/R of each species, then H/R)
// are written, with the rest of their 16-row tile (mixed_q_len leaves room).
// Warp-collective.
template <int G>
__device__ __forceinline__ void net_eval_cells(const MlpFrag& f, float t, float* q0, int cell_ld,
                                               int n_rows) {
  constexpr int CPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, q = lane & 3;
  unsigned* w0 = reinterpret_cast<unsigned*>(q0);
  // layer 1 (1 -> 64, FP32 FMA and tanh): lane l of cell k takes hidden units
  // l, l + G, ...
  {
    __nv_bfloat16* h1 = reinterpret_cast<__nv_bfloat16*>(w0 + (lane / G) * cell_ld + kNetH1Off);
#pragma unroll
    for (int u = 0; u < kHid / G; ++u) {
      const int j = lane % G + G * u;
      const float2 wb = f.w1[j];
      h1[j] = __float2bfloat16_rn(tanh_approx(fmaf(wb.x, t, wb.y)));
    }
  }
  __syncwarp();
  // B fragments: column g is cell g mod CPW; rows (hidden inputs) 2q, 2q + 1
  // and 2q + 8, 2q + 9 of each 16-row k-tile
  const unsigned* hb = w0 + (g % CPW) * cell_ld;
  unsigned b[4][2];
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) {
    b[kt][0] = hb[kNetH1Off + kt * 8 + q];
    b[kt][1] = hb[kNetH1Off + kt * 8 + 4 + q];
  }
  // layer 2 (64 -> 64): D[j][c] = sum_i W2[j][i] h1_c[i] + b2[j], four m-tiles
  float d[4][4];
#pragma unroll
  for (int mt = 0; mt < 4; ++mt) {
    const float2 bb = f.b2[mt * 32 + lane];
    d[mt][0] = bb.x;
    d[mt][1] = bb.x;
    d[mt][2] = bb.y;
    d[mt][3] = bb.y;
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) mma_bf16_16816_a(d[mt], __ldg(f.W2 + (mt * 4 + kt) * 32 + lane), b[kt]);
  }
  // tanh into the cells' layer-2 activations: lane (g, q) holds rows
  // 16 mt + g and 16 mt + g + 8 of columns 2q and 2q + 1, i.e. of cells
  // (2q + half) mod CPW.  Lanes whose columns repeat the same cells split the
  // m-tiles between them, so that each activation is computed once: with one
  // cell per warp lane (g, q) takes m-tile q; with two cells, m-tile q of both;
  // with four, m-tiles 2 (q / 2) and 2 (q / 2) + 1 of its two cells.
  {
    constexpr int kMtPerLane = CPW == 1 ? 1 : (CPW == 2 ? 1 : 2);
    constexpr int kHalves = CPW == 1 ? 1 : 2;
    const int mt0 = CPW == 4 ? 2 * (q >> 1) : q;
#pragma unroll
    for (int u = 0; u < kMtPerLane; ++u) {
      const int mt = mt0 + u;
      float v[4];
#pragma unroll
      for (int e = 0; e < 4; ++e)  // d[mt][e] with mt known per lane only at run time
        v[e] = mt == 0 ? d[0][e] : mt == 1 ? d[1][e] : mt == 2 ? d[2][e] : d[3][e];
#pragma unroll
      for (int half = 0; half < kHalves; ++half) {
        __nv_bfloat16* h2 = reinterpret_cast<__nv_bfloat16*>(
            w0 + ((2 * q + half) % CPW) * cell_ld + kNetH2Off) + mt * 16 + g;
        h2[0] = __float2bfloat16_rn(tanh_approx(v[half]));
        h2[8] = __float2bfloat16_rn(tanh_approx(v[2 + half]));
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int kt = 0; kt < 4; ++kt) {
    b[kt][0] = hb[kNetH2Off + kt * 8 + q];
    b[kt][1] = hb[kNetH2Off + kt * 8 + 4 + q];
  }
  // layer 3 (64 -> outputs), the m-tiles holding rows below n_rows (whole
  // tiles are written: the output rows have room for them); the bias and the
  // standardisation are folded into (scale, offset)
  const int n_mt = (n_rows + 15) >> 4;
  for (int mt = 0; mt < n_mt; ++mt) {
    float e[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) mma_bf16_16816_a(e, __ldg(f.W3 + (mt * 4 + kt) * 32 + lane), b[kt]);
    const float4 so = f.o3[mt * 32 + lane];
#pragma unroll
    for (int half = 0; half < (CPW > 1 ? 2 : 1); ++half) {
      float* out = q0 + ((2 * q + half) % CPW) * cell_ld + kNetOutOff + mt * 16 + g;
      out[0] = fmaf(e[half], so.x, so.y);
      out[8] = fmaf(e[2 + half], so.z, so.w);
    }
  }
  __syncwarp();
}

// One warp evaluates the network at 16 temperatures (rows).  act is a warp-
// private shared buffer of 16 x (64+8) BF16 for the activations.  out[r][o]
// receives value(o) for o in [o_begin, o_end) (a multiple of 8 wide), rows
// r < n_rows; out_ld is the row stride of out.
__device__ void mlp_eval_warp16(const MlpInfer& w, const float* t16, __nv_bfloat16* act,
                                float* out, int out_ld, int n_rows, int o_begin, int o_end) {
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, tg = lane & 3;
  constexpr int lda = kHid + 8;  // BF16 elements per activation row
  // layer 1 (1 -> 64) on the SIMT pipes: lane handles 2 hidden units for all rows
  for (int r = 0; r < 16; ++r) {
    const int j = lane * 2;
    const float t = t16[r];
    const float h0 = tanh_approx(fmaf(w.W1[j], t, w.b1[j]));
    const float h1 = tanh_approx(fmaf(w.W1[j + 1], t, w.b1[j + 1]));
    *reinterpret_cast<unsigned*>(act + r * lda + j) = pack_bf16(h0, h1);
  }
  __syncwarp();
  // layer 2 (64 -> 64): 8 n-tiles x 4 k-steps of m16n8k16
  float acc[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = w.b2[nt * 8 + tg * 2], b1v = w.b2[nt * 8 + tg * 2 + 1];
    acc[nt][0] = b0; acc[nt][1] = b1v; acc[nt][2] = b0; acc[nt][3] = b1v;
  }
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const int k0 = ks * 16;
    unsigned a[4];
    a[0] = *reinterpret_cast<const unsigned*>(act + g * lda + k0 + tg * 2);
    a[1] = *reinterpret_cast<const unsigned*>(act + (g + 8) * lda + k0 + tg * 2);
    a[2] = *reinterpret_cast<const unsigned*>(act + g * lda + k0 + 8 + tg * 2);
    a[3] = *reinterpret_cast<const unsigned*>(act + (g + 8) * lda + k0 + 8 + tg * 2);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const __nv_bfloat16* wr = w.W2 + (nt * 8 + g) * kHid + k0 + tg * 2;
      unsigned b[2];
      b[0] = __ldg(reinterpret_cast<const unsigned*>(wr));
      b[1] = __ldg(reinterpret_cast<const unsigned*>(wr + 8));
      mma_bf16_16816(acc[nt], a, b);
    }
  }
  __syncwarp();
  // tanh, back to BF16 in the same buffer (every lane has finished reading it)
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int c = nt * 8 + tg * 2;
    *reinterpret_cast<unsigned*>(act + g * lda + c) =
        pack_bf16(tanh_approx(acc[nt][0]), tanh_approx(acc[nt][1]));
    *reinterpret_cast<unsigned*>(act + (g + 8) * lda + c) =
        pack_bf16(tanh_approx(acc[nt][2]), tanh_approx(acc[nt][3]));
  }
  __syncwarp();
  // layer 3 (64 -> outputs), one n-tile of 8 outputs at a time
  unsigned a[4][4];
#pragma unroll
  for (int ks = 0; ks < 4; ++ks) {
    const int k0 = ks * 16;
    a[ks][0] = *reinterpret_cast<const unsigned*>(act + g * lda + k0 + tg * 2);
    a[ks][1] = *reinterpret_cast<const unsigned*>(act + (g + 8) * lda + k0 + tg * 2);
    a[ks][2] = *reinterpret_cast<const unsigned*>(act + g * lda + k0 + 8 + tg * 2);
    a[ks][3] = *reinterpret_cast<const unsigned*>(act + (g + 8) * lda + k0 + 8 + tg * 2);
  }
  for (int o0 = o_begin; o0 < o_end; o0 += 8) {
    const int c = o0 + tg * 2;
    float d[4] = {w.b3[c], w.b3[c + 1], w.b3[c], w.b3[c + 1]};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const __nv_bfloat16* wr = w.W3 + (o0 + g) * kHid + ks * 16 + tg * 2;
      unsigned b[2];
      b[0] = __ldg(reinterpret_cast<const unsigned*>(wr));
      b[1] = __ldg(reinterpret_cast<const unsigned*>(wr + 8));
      mma_bf16_16816(d, a[ks], b);
    }
    const float m0 = w.mean[c], m1 = w.mean[c + 1], s0 = w.stdv[c], s1 = w.stdv[c + 1];
    const bool c0ok = c < w.n_valid, c1ok = c + 1 < w.n_valid;
    if (g < n_rows) {
      if (c0ok) out[g * out_ld + c - o_begin] = fmaf(d[0], s0, m0);
      if (c1ok) out[g * out_ld + c + 1 - o_begin] = fmaf(d[1], s1, m1);
    }
    if (g + 8 < n_rows) {
      if (c0ok) out[(g + 8) * out_ld + c - o_begin] = fmaf(d[2], s0, m0);
      if (c1ok) out[(g + 8) * out_ld + c + 1 - o_begin] = fmaf(d[3], s1, m1);
    }
  }
  __syncwarp();
}

// Batched inference: every warp takes 16 temperatures.  out [n][n_out].
__global__ void mlp_eval_kernel(MlpInfer w, const double* __restrict__ T, long long n,
                                float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __nv_bfloat16* act = reinterpret_cast<__nv_bfloat16*>(smem) + warp * 16 * (kHid + 8);
  float* t16 = reinterpret_cast<float*>(smem + (blockDim.x / 32) * 16 * (kHid + 8) * 2) + warp * 16;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * 16; base < n;
       base += nwarps * 16) {
    if (lane < 16) t16[lane] = base + lane < n ? ((float)T[base + lane] - kTMid) / kTHalf : 0.0f;
    __syncwarp();
    const int rows = (int)min((long long)16, n - base);
    mlp_eval_warp16(w, t16, act, out + base * w.n_valid, w.n_valid, rows, 0, w.n_out);
  }
}

#ifndef __CUDACC_RTC__
__host__ inline size_t mlp_eval_smem_bytes(int warps) {
  return (size_t)warps * 16 * (kHid + 8) * 2 + (size_t)warps * 16 * 4;
}
#endif

}  // namespace stev
