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
  double dt;        // this cell's fluid time step t_f
  double hcap;      // t_f * delta_max (Eq. 4's time cap)
  // mixed kernels: T and ln T as float pairs (hi + lo, ~2^-48 relative), and
  // the time cap as a float pair
  float Th, Tl, lnTh, lnTl, hcap_h, hcap_l;
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
  if (L.serve) {
    // slots are rewritten by the host between requests: read around L1
    const BatchDesc* d = &L.slots[b].d;
    io.T = (const double*)__ldcg((const long long*)&d->T);
    io.P = (const double*)__ldcg((const long long*)&d->P);
    io.Y = (const double*)__ldcg((const long long*)&d->Y);
    io.T_out = (double*)__ldcg((const long long*)&d->T_out);
    io.Y_out = (double*)__ldcg((const long long*)&d->Y_out);
    io.iters = (int*)__ldcg((const long long*)&d->iters);
    io.status = (unsigned char*)__ldcg((const long long*)&d->status);
    io.dt = __ldcg(&d->dt);
    io.n = __ldcg(&d->n);
  } else if (L.nb > 0) {
    const BatchDesc& d = L.bdesc[b];
    io.T = d.T; io.P = d.P; io.Y = d.Y; io.T_out = d.T_out; io.Y_out = d.Y_out;
    io.iters = d.iters; io.status = d.status; io.dt = d.dt; io.n = d.n;
  } else {
    io.T = L.T; io.P = L.P; io.Y = L.Y; io.T_out = L.T_out; io.Y_out = L.Y_out;
    io.iters = L.iters; io.status = L.status; io.dt = L.dt; io.n = L.n_cells;
  }
  return io;
}

// Bit pattern of a double as a signed integer: for values >= 0 (and +inf,
// NaN) the integers order like the values, and a negative value's pattern is
// negative, so range tests and min / max of such values need no FP64 unit.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ long long ld_acquire_s64(const long long* p) {
  long long v;
  asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Serving refill: lane 0 claims up to one id per needy group below
// `published` with a bounded compare-and-swap loop; needy groups take them in
// lane order.  `idle` (warp-uniform) is set when ids were wanted but none were
// ready, so that the caller can back off.
template <int G>
__device__ __forceinline__ long long serve_refill(const Launch& L, bool needs, bool& idle) {
  const int lane = threadIdx.x & 31;
  const int leader = lane & ~(G - 1);
  const unsigned need = __ballot_sync(0xffffffffu, (lane == leader) && needs);
  idle = false;
  if (need == 0u) return -1;
  const unsigned cnt = __popc(need);
  unsigned long long base = 0, got = 0;
  if (lane == 0 && *(volatile int*)&L.ctl->stop == 0 && *(volatile int*)&L.ctl->exiting == 0) {
    for (int attempt = 0; attempt < 64; ++attempt) {
      const unsigned long long pub = ld_acquire_u64(&L.ctl->published);
      const unsigned long long cur = *(volatile unsigned long long*)&L.ctl->claim;
      if (cur >= pub) break;
      const unsigned long long want = min((unsigned long long)cnt, pub - cur);
      if (atomicCAS(&L.ctl->claim, cur, cur + want) == cur) {
        base = cur;
        got = want;
        break;
      }
    }
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  got = __shfl_sync(0xffffffffu, got, 0);
  idle = got == 0;
  if (!needs) return -1;
  const unsigned rank = __popc(need & ((1u << leader) - 1u));
  return rank < got ? (long long)(base + rank) : -1;
}

// Serving: a warp with no cell.  Returns true when the warp should leave:
// on `stop`, once `exiting` is set, or when it finds every warp of the grid
// idle for idle_ns (it then sets `exiting`).  `committed` (warp-uniform) tells
// whether this warp counts itself in idle_warps; it counts itself out as soon
// as unclaimed work is visible, before it claims any.
__device__ __forceinline__ bool serve_idle(const Launch& L, unsigned long long& idle_since,
                                           bool& committed) {
  const int lane = threadIdx.x & 31;
  int leave = 0, comm = committed ? 1 : 0;
  if (lane == 0) {
    ServeCtl* ctl = L.ctl;
    const unsigned long long now = gtimer_ns();
    if (idle_since == 0) idle_since = now;
    if (*(volatile int*)&ctl->stop || *(volatile int*)&ctl->exiting) {
      leave = 1;
    } else if (*(volatile unsigned long long*)&ctl->claim < ld_acquire_u64(&ctl->published)) {
      if (comm) {
        atomicSub(&ctl->idle_warps, 1);
        comm = 0;
      }
      idle_since = now;
    } else {
      if (!comm && now - idle_since > (unsigned long long)L.idle_ns) {
        atomicAdd(&ctl->idle_warps, 1);
        comm = 1;
      }
      if (comm) {
        __threadfence();
        if (atomicAdd(&ctl->idle_warps, 0) >= L.serve_warps) {
          atomicExch(&ctl->exiting, 1);
          leave = 1;
        }
      }
    }
  }
  leave = __shfl_sync(0xffffffffu, leave, 0);
  committed = __shfl_sync(0xffffffffu, comm, 0) != 0;
  return leave != 0;
}

// Serving: the slot of claimed id c, by binary search over the newest serve_q
// sequence numbers.  Slots are retired in sequence order and only a retired
// slot is rewritten, so c's request (unfinished) is inside the window and its
// slot is stable.  A slot older than c's request reads as its old key (first
// id <= c) or as a newer request's key (other sequence number): both say
// "c lies beyond", which is right.  Returns -1 if the index would fall outside
// the request (never expected).
__device__ __forceinline__ int serve_find_slot(const Launch& L, long long c, long long& lc) {
  const long long hi0 = ld_acquire_s64(&L.ctl->pub_seq);
  long long lo = max(0LL, hi0 - L.serve_q + 1), hi = hi0;  // answer in [lo, hi]
  while (lo < hi) {
    const long long mid = (lo + hi + 1) >> 1;
    const unsigned long long key = __ldcg(&L.slots[(int)(mid % L.serve_q)].key);
    const bool beyond = (key & kServeSeqMask) != ((unsigned long long)mid & kServeSeqMask) ||
                        (long long)(key >> kServeSeqBits) <= c;
    if (beyond) lo = mid; else hi = mid - 1;
  }
  const int s = (int)(lo % L.serve_q);
  const unsigned long long key = __ldcg(&L.slots[s].key);
  lc = c - (long long)(key >> kServeSeqBits);
  const long long n = __ldcg(&L.slots[s].d.n);
  if ((key & kServeSeqMask) != ((unsigned long long)lo & kServeSeqMask) || lc < 0 || lc >= n) {
    atomicAdd(&L.ctl->dropped, 1);
    L.smail[L.serve_q] = -2;  // tell the host
    return -1;
  }
  return s;
}

// Serving: called by every lane of a group after it has written its share of
// a finished cell's outputs.  One lane counts the cell; the request's last
// cell posts the request's sequence number to the host mailbox.
template <int G>
__device__ __forceinline__ void serve_cell_done(const Launch& L, int b, long long n, int l) {
  const unsigned gmask = (G == 32) ? 0xffffffffu
                                   : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
  __threadfence();  // this lane's outputs before the count
  __syncwarp(gmask);
  if (l == 0) {
    ServeSlot* sl = L.slots + b;
    const unsigned long long prev = atomicAdd(&sl->done, 1ULL);
    if ((long long)prev + 1 == n) {
      __threadfence_system();
      L.smail[b] = (long long)__ldcg(&sl->key);
    }
  }
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
  const double* rg;   // general rate laws: [R][8] nu, order of the slots
  const double* gnu;  // general rate laws: [n_gather] nu
};

// C^a for a reaction order a: products for orders 1 and 2 (as elementary
// mass action evaluates them), pow otherwise (global rate laws, Eq. 28).
__device__ __forceinline__ double conc_pow(double c, double a) {
  if (a == 1.0) return c;
  if (a == 2.0) return c * c;
  return pow(c, a);
}

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
