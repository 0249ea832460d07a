// Pieces shared by the FP64 and mixed-precision persistent kernels: group
// reductions over the G lanes that own one cell, the per-group cell state,
// the staged table pointers and the ballot/popcount refill.
#pragma once
#include "stev_device.cuh"

namespace stev {

template <int G, typename F>
__device__ __forceinline__ F group_sum(F v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, G);
  return v;
}

// Minimum of num/den over the group (den > 0; den == 0 encodes +inf), with a
// symmetric tie-break so that every lane keeps the same pair.
template <int G>
__device__ __forceinline__ void group_min_frac(double& num, double& den) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) {
    const double n2 = __shfl_xor_sync(0xffffffffu, num, o, G);
    const double d2 = __shfl_xor_sync(0xffffffffu, den, o, G);
    const double a = n2 * den, b = num * d2;
    const bool take = (a < b) || (a == b && (n2 < num || (n2 == num && d2 < den)));
    if (take) { num = n2; den = d2; }
  }
}

template <int G>
__device__ __forceinline__ bool group_any(bool v) {
  const unsigned b = __ballot_sync(0xffffffffu, v);
  const int base = (threadIdx.x & 31) & ~(G - 1);
  const unsigned m = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << base);
  return (b & m) != 0u;
}

struct CellState {
  long long cell;   // -1 when the group has no cell
  double T, P, t_rem;
  int it;
  int nhist;
  double lnT;       // mixed kernel: ln T kept up to date incrementally
  double dt;        // this cell's fluid time step t_f
  long long lc;     // index inside its batch
  int b;            // its batch (batched launches)
};

// Where cell c's arrays are: resolves batched launches by binary search over
// the batch offsets (every batch non-empty).
struct CellIO {
  const double* T;
  const double* P;
  const double* Y;
  double* T_out;
  double* Y_out;
  int* iters;
  unsigned char* status;
  double dt;
  long long n;   // cells in the batch (the Y stride of species-major input)
};

__device__ __forceinline__ CellIO cell_io(const Launch& L, int b) {
  CellIO io;
  if (L.nb > 0) {
    const BatchDesc& d = L.bdesc[b];
    io.T = d.T; io.P = d.P; io.Y = d.Y; io.T_out = d.T_out; io.Y_out = d.Y_out;
    io.iters = d.iters; io.status = d.status; io.dt = d.dt; io.n = d.n;
  } else {
    io.T = L.T; io.P = L.P; io.Y = L.Y; io.T_out = L.T_out; io.Y_out = L.Y_out;
    io.iters = L.iters; io.status = L.status; io.dt = L.dt; io.n = L.n_cells;
  }
  return io;
}

__device__ __forceinline__ int find_batch(const Launch& L, long long c) {
  if (L.nb <= 0) return 0;
  int lo = 0, hi = L.nb;  // boff[lo] <= c < boff[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (L.boff[mid] <= c) lo = mid; else hi = mid;
  }
  return lo;
}

struct Tables {
  const double* sp;
  const double* rx;
  const int4* ri;
  const int* gptr;
  const int* gent;
  const double* tw;
};

template <int G>
__device__ __forceinline__ float group_min(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o, G));
  return v;
}

// Refill (Sec. 2.4 variable load): every group whose cell is done sets one
// bit (its leader lane); the warp claims popc(bits) consecutive cell ids with
// one atomicAdd and each group takes base + (number of needy groups below
// it).  Returns the new cell id of this lane's group, or -1.  Warp-collective.
template <int G>
__device__ __forceinline__ long long refill(unsigned long long* counter, unsigned long long n,
                                            bool needs, bool& exhausted) {
  const int lane = threadIdx.x & 31;
  const int leader = lane & ~(G - 1);
  const unsigned need = __ballot_sync(0xffffffffu, (lane == leader) && needs);
  long long got = -1;
  if (need != 0u && !exhausted) {
    const unsigned cnt = __popc(need);
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(counter, (unsigned long long)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base + cnt >= n) exhausted = true;
    if (needs) {
      const unsigned long long c = base + __popc(need & ((1u << leader) - 1u));
      if (c < n) got = (long long)c;
    }
  }
  return got;
}

}  // namespace stev
