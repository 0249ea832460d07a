// Mixed-precision STEV: rates in FP32; state, ln T, 1/T and the Gibbs terms
// of Eq. 30 in float-pair arithmetic on the FP32 pipe.
//
// Same structure as the FP64 kernel (a group of G lanes per cell, all cell
// state in shared memory, species-major gather, ballot/popcount refill).
// What changes is the arithmetic:
//   float pairs (hi + lo, about 48 significant bits, built with error-free
//         transformations: Knuth's TwoSum and FMA products): Y and T and
//         their forward Euler update (Eq. 18); ln T (updated by ln(1 + dT/T)
//         from its series, refreshed by the FP64 log every 256 steps) and 1/T;
//         each species' Gibbs term of Eq. 30, a compensated dot product of its
//         FP64 coefficients (split into float pairs on the host) with the
//         float-pair basis 1, ln T, 1/T, T, T^2, T^3, T^4; and the per-reaction
//         Gibbs difference dG/RT - dN ln(P_atm/RT) that sets K, summed from
//         those pairs with TwoSum, so that the exponent keeps no cancellation
//         loss before the single rounding to FP32 that the exponential takes
//         (error ~1e-11 in log2 K, against ~1e-6 relative in the FP32 rates);
//   FP64  t_rem and h (two instructions per step: which step ends at t_f is
//         decided exactly as in the FP64 path);
//   FP32  mixture, cp/R and H/RT (Eqs. 15-16), gamma and concentrations
//         (Eqs. 6-7), forward and reverse rate constants (exponentials on the
//         MUFU unit in base 2: k = 2^(log2 k)), rates of progress and rOF
//         (Eq. 14), production rates, dT/dt, the limiter (Eqs. 1-5) and the
//         ringing history and DFT test (Eqs. 8-13).
// B300's FP64 pipe runs at 1/75 of the FP32 rate, and a warp's FP64
// instruction costs it the same time whatever the number of active lanes, so
// per-cell scalars in FP64 (one cell per warp) would cost 32 lanes' worth.
#pragma once
#include "stev_common.cuh"
#include "stev_mlp.cuh"

namespace stev {

constexpr double kLog2e = 1.4426950408889634;

// Mechanism sizes and the rate-law kind: compile-time constants in a kernel
// built for one mechanism (STEV_SPEC_S, _R, _RREV, _GENERAL defined: loops of
// known trip count, table rows at immediate offsets), else the launch's.
#ifdef STEV_SPEC_S
__device__ __forceinline__ constexpr int mS(const Launch&) { return STEV_SPEC_S; }
__device__ __forceinline__ constexpr int mR(const Launch&) { return STEV_SPEC_R; }
__device__ __forceinline__ constexpr int mRrev(const Launch&) { return STEV_SPEC_RREV; }
__device__ __forceinline__ constexpr int mGeneral(const Launch&) { return STEV_SPEC_GENERAL; }
#else
__device__ __forceinline__ int mS(const Launch& L) { return L.S; }
__device__ __forceinline__ int mR(const Launch& L) { return L.R; }
__device__ __forceinline__ int mRrev(const Launch& L) { return L.Rrev; }
__device__ __forceinline__ int mGeneral(const Launch& L) { return L.general; }
#endif

// Running window sums of the damper (Eq. 9's D0 = |sum of the window| and the
// sum of |x| of its bound) held in registers for the first kWinRegs reactions
// of each lane, updated by the tap that enters and the tap that leaves and
// recomputed exactly once per window (every N steps), instead of re-summed
// from the 13 taps every step.  Only in a kernel compiled for a mechanism
// whose every reaction is elementary and reversible (history row = reaction),
// with 32-lane groups and the N = 13 window.
#if defined(STEV_SPEC_R) && defined(STEV_SPEC_RREV) && defined(STEV_SPEC_GENERAL)
constexpr bool kSpecAllRev = STEV_SPEC_R == STEV_SPEC_RREV && !STEV_SPEC_GENERAL;
constexpr int kSpecTrips32 = (STEV_SPEC_R + 31) / 32;  // reactions per lane, 32-lane groups
#else
constexpr bool kSpecAllRev = false;
constexpr int kSpecTrips32 = 1;
#endif
template <int G, int NT, bool MLP>
struct WinRegs {
  // four reactions per lane with the polynomial thermo; none with the
  // network, whose MMA fragments leave no registers for them (measured: with
  // them that kernel spills and gains 1%, the polynomial one gains 7%)
  static constexpr int cap = MLP ? 0 : 4;
  static constexpr int n =
      (kSpecAllRev && G == 32 && NT == 13) ? (kSpecTrips32 < cap ? kSpecTrips32 : cap) : 0;
};

__device__ __forceinline__ float ex2f(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Knuth's TwoSum: s + err == a + b exactly (round-to-nearest, no FMA needed).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& err) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// A float pair: the value h + l, |l| <= ulp(h).
struct FF {
  float h, l;
};

// Dekker's Fast2Sum: h + l == a + b exactly when |a| >= |b| (or a == 0).
__device__ __forceinline__ FF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// s + e of any magnitudes as a float pair.
__device__ __forceinline__ FF ff_norm(float s, float e) {
  FF r;
  two_sum(s, e, r.h, r.l);
  return r;
}

// x * y; the l * l term (2^-48 relative) is dropped.
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = fmaf(x.h, y.h, -p);
  e = fmaf(x.h, y.l, e);
  e = fmaf(x.l, y.h, e);
  return fast_two_sum(p, e);
}

// x + y
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  float s, t;
  two_sum(x.h, y.h, s, t);
  return fast_two_sum(s, t + (x.l + y.l));
}

// x + a * b for a float pair x, a float pair a and a float b (Eq. 18's update)
__device__ __forceinline__ FF ff_add_mul(FF x, FF a, float b) {
  const float p = __fmul_rn(a.h, b);
  float pe = fmaf(a.h, b, -p);
  pe = fmaf(a.l, b, pe);
  float s, t;
  two_sum(x.h, p, s, t);
  return fast_two_sum(s, t + (x.l + pe));
}

__device__ __forceinline__ FF ff_from_double(double x) {
  const float h = (float)x;
  return FF{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double ff_to_double(FF x) { return (double)x.h + (double)x.l; }

// (s, e) += c * b for a float-pair coefficient (ch, cl) and a float-pair
// basis value b: the product's rounding error by FMA, the sum's by TwoSum
// (the compensated dot product of Ogita, Rump and Oishi, 2005, with float-pair
// operands); s + e is the exact sum so far to ~2^-48 of the terms' magnitude.
__device__ __forceinline__ void dot2_term(float ch, float cl, FF b, float& s, float& e) {
  const float p = __fmul_rn(ch, b.h);
  float pe = fmaf(ch, b.h, -p);
  pe = fmaf(ch, b.l, pe);
  pe = fmaf(cl, b.h, pe);
  float t;
  two_sum(s, p, s, t);
  e += t + pe;
}

// ln(1 + u) for a float pair |u| <= 2^-7: u - u^2/2 + u^3 (1/3 - u/4 + u^2/5 -
// u^3/6 + u^4/7), u^2 exact by FMA; the truncated terms are below 2^-59 and
// the FP32 rounding of the u^3 part below 2^-46.
__device__ __forceinline__ FF ff_log1p_small(FF u) {
  const float q = __fmul_rn(u.h, u.h);
  float qe = fmaf(u.h, u.h, -q);
  qe = fmaf(2.0f * u.h, u.l, qe);
  const float c3 =
      q * u.h *
      fmaf(fmaf(fmaf(fmaf(u.h, 0.142857149f, -0.166666672f), u.h, 0.2f), u.h, -0.25f), u.h,
           0.333333343f);
  float s, t;
  two_sum(u.h, -0.5f * q, s, t);
  return fast_two_sum(s, t + (u.l + fmaf(-0.5f, qe, c3)));
}

// T below the float pair (sh, sl) (both exact pairs)
__device__ __forceinline__ bool ff_below(FF T, float sh, float sl) {
  return T.h < sh || (T.h == sh && T.l < sl);
}

struct TablesF {
  const float* spf;   // float species table [SF_ROWS][S]
  const float4* rxf;  // lg2 A, beta, Ea/R log2 e, dN
  const int4* ri;
  const int* gptr;
  const int* gent;
  const float* tw;    // float twiddles
  const float* rg;    // general rate laws: [R][8] nu, order of the slots
  const float* gnu;   // general rate laws: [n_gather] nu
};

// Adds nu * (g.x + g.y) to the sum s + e of a general reaction's exponent
// (g = (k, f) of gibbs_split): nu k and its rounding error by fma into s by
// TwoSum, nu f and the errors into e, so that s + e is exact but for the
// roundings of e (terms below a few units: ~2^-22 absolute).
__device__ __forceinline__ void pair_add_scaled(float nu, float2 g, float& s, float& e) {
  const float p = nu * g.x;
  const float pe = fmaf(nu, g.x, -p);
  float t;
  two_sum(s, p, s, t);
  e += t + fmaf(nu, g.y, pe);
}

// T inside the network's training range (on the pair's high part; the same
// test decides the request and its use)
__device__ __forceinline__ bool in_net_range(float Th) {
  return Th >= (float)kMlpTLow && Th <= (float)kMlpTHigh;
}

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float lg2f_approx(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// The reverse term kr C_p0 C_p1 of an elementary reaction (Eqs. 29-30):
// kr = kf 2^x with x = sum nu g2.  Each species' g2 is held as (k, f), k the
// integer nearest to it and f the rest (gibbs_split), so that the integer
// parts of the sum cancel exactly and only the fractions (|f| <= 1/2) are
// rounded: x before its one rounding is exact to a few 2^-25.
__device__ __forceinline__ float reverse_term(const float2* cG2, const float* cC, int a0, int a1,
                                              int p0, int p1, float lg2kf) {
  const float2 gp0 = cG2[p0], ga0 = cG2[a0], ga1 = cG2[a1], gp1 = cG2[p1];
  const float kx = (gp0.x - ga0.x) + (gp1.x - ga1.x);  // integers below 2^24: exact
  const float fx = (gp0.y - ga0.y) + (gp1.y - ga1.y);
  return ex2f(lg2kf + (kx + fx)) * cC[p0] * cC[p1];
}

// g2 = h + l (a float pair) as (k, f): k = rint(h), f = (h - k) + l, where
// h - k is exact (the fractional bits of h), so k + f = g2 to one rounding of
// a number below 1 in magnitude.
__device__ __forceinline__ float2 gibbs_split(FF g2) {
  const float k = rintf(g2.h);
  return make_float2(k, (g2.h - k) + g2.l);
}

// The stoichiometric coefficient of an elementary gather entry (gather_pack:
// reaction * 16 + nu + 8): nu = code - 8, formed as (2^23 + code) - (2^23 + 8)
// from the float bits, exact.
__device__ __forceinline__ float nu_of_code(int e) {
  return __int_as_float(0x4B000000 | (e & 15)) - 8388616.0f;
}

// Eq. 10's largest high-frequency |X_j|^2 (bins j = hi_first ...) of a full
// window hw[N] in storage order (|X_j| does not depend on the rotation),
// scaled by inv^2.  The twiddle rows of bin b are tw[b][0..N) = cos(-2 pi j
// k / N) and tw[b][N..2N) = sin(-2 pi j k / N); since cos(theta_{N-k}) =
// cos(theta_k) and sin(theta_{N-k}) = -sin(theta_k), taps k and N - k are
// paired: Re X_j = x_0 + sum_k (x_k + x_{N-k}) cos_k (+ the middle tap of an
// even N), Im X_j = sum_k (x_k - x_{N-k}) sin_k, k = 1 .. (N - 1) / 2.
template <int NT>
__device__ __forceinline__ float hi_bins_max2(const float* hw, int N, const float* tw, int n_bins,
                                              float inv) {
  float max2 = 0.0f;
  if constexpr (NT > 0 && (NT & 1)) {
    constexpr int kHalf = (NT - 1) / 2;
    float u[kHalf], v[kHalf];
#pragma unroll
    for (int k = 1; k <= kHalf; ++k) {
      const float a = hw[k], b = hw[NT - k];
      u[k - 1] = a + b;
      v[k - 1] = a - b;
    }
    const float x0 = hw[0];
#pragma unroll 1
    for (int bb = 0; bb < n_bins; ++bb) {
      const float* c = tw + bb * 2 * NT;
      float re = x0, im = 0.0f;
#pragma unroll
      for (int k = 1; k <= kHalf; ++k) {
        re = fmaf(u[k - 1], c[k], re);
        im = fmaf(v[k - 1], c[NT + k], im);
      }
      re *= inv;
      im *= inv;
      max2 = fmaxf(max2, fmaf(re, re, im * im));
    }
  } else {
    const int half = (N - 1) / 2;
    for (int bb = 0; bb < n_bins; ++bb) {
      const float* c = tw + bb * 2 * N;
      float re = hw[0], im = 0.0f;
      for (int k = 1; k <= half; ++k) {
        const float a = hw[k], b = hw[N - k];
        re = fmaf(a + b, c[k], re);
        im = fmaf(a - b, c[N + k], im);
      }
      if (!(N & 1)) re = fmaf(hw[N / 2], c[N / 2], re);
      re *= inv;
      im *= inv;
      max2 = fmaxf(max2, fmaf(re, re, im * im));
    }
  }
  return max2;
}

// MLP = true: cp/R (and, with L.mlp_h, H/RT) come from the thermo network
// (Sec. 3) whenever T is inside its training range; outside it, and for G/RT
// always, the NASA-7 polynomials are used.  The warp evaluates the network of
// all its cells at the start of the step (net_eval_cells: BF16 tensor-core
// MMAs with FP32 accumulation) into each cell's output row cOut, from which
// the thermo loop reads cp/R and H/R; net_buf holds the warp's activations.
//
// NT > 0: the DFT window N (Eq. 9) fixed at compile time (the taps unrolled);
// NT = 0: N = L.dft_n.  The history is reaction-major, N taps of a reaction
// contiguous at a stride of N rounded up to odd (lanes on consecutive
// reactions hit distinct banks).  A missing reactant or product slot points
// at species S, whose C is 1 and g2 is 0, so that products and Gibbs sums
// need no branch.
template <int G, bool MLP, int NT>
__device__ __forceinline__ int step_mixed(const Launch& L, const TablesF& tb, float* cYh,
                                          float* cYl, float2* cG2, float* cC, float* cH,
                                          float* cQ, float* cHist, float* cRof, float Pf, int l,
                                          CellState& st, float* netQ0, int cell_ld,
                                          float* win_s, float* win_a) {
  const int S = mS(L), R = mR(L), Rrev = mRrev(L);
  const int N = NT > 0 ? NT : L.dft_n;
  const int NP = N | 1;
  const FF T{st.Th, st.Tl};
  const FF lnT{st.lnTh, st.lnTl};
  const float Tf = T.h;
  const bool use_net = MLP && in_net_range(Tf);
  // the network's outputs for this cell, in its rate array until the rates
  // are computed
  const float* cOut = cQ + kNetOutOff;
  if (MLP && __any_sync(0xffffffffu, use_net))
    net_eval_cells<G>(L.mlp.frag, (Tf - kTMid) * (1.0f / kTHalf), netQ0, cell_ld, L.mlp_needed);
  // 1/T: the FP32 reciprocal r, then 1/T = r / (1 - e), e = 1 - T r exact to
  // ~2^-46 by FMA: lo = r (e + e^2)
  const float r0 = rcp_approx(Tf);
  float e0 = fmaf(-Tf, r0, 1.0f);
  e0 = fmaf(-T.l, r0, e0);
  const FF invT = fast_two_sum(r0, r0 * fmaf(e0, e0, e0));
  const float invTf = invT.h;
  const float lg2Tf = lg2f_approx(Tf);
  const FF T2 = ff_mul(T, T);
  const FF T3 = ff_mul(T2, T);
  const FF T4 = ff_mul(T2, T2);

  // mixture (FP32)
  float part = 0.0f;
  for (int i = l; i < S; i += G) part = fmaf(cYh[i], tb.spf[SF_INVW * S + i], part);
  const float sumYW = group_sum<G>(part);
  const float rho = Pf / ((float)kRu * Tf * sumYW);

  // thermo: cp/R, H/RT in FP32; the Gibbs term in log2 units with the
  // standard-state pressure of Eq. 30 folded in, g2 = (G/RT - ln(P_atm/RT))
  // log2 e, as a float pair (a reaction's sum of nu g2 is its whole exponent:
  // sum nu = dN carries the pressure term)
  float cpp = 0.0f;
  for (int i = l; i < S; i += G) {
    const float* f = tb.spf + i;  // row k of species i at f[k * S]
    const bool lo = ff_below(T, f[SF_SPLIT_H * S], f[SF_SPLIT_L * S]);
    const float* b = f + (lo ? SF_LOW : SF_HIGH) * S;
    const float* g = f + (lo ? SF_GLOW : SF_GHIGH) * S;
    const float Yi = cYh[i];
    if (!use_net) {
      const float cpR = fmaf(fmaf(fmaf(fmaf(b[BF_A4 * S], Tf, b[BF_A3 * S]), Tf, b[BF_A2 * S]),
                                  Tf, b[BF_A1 * S]), Tf, b[BF_A0 * S]);
      cpp = fmaf(Yi * cpR, f[SF_INVW * S], cpp);
    } else {
      cpp = fmaf(Yi * cOut[i], f[SF_INVW * S], cpp);  // cp/R from the network
    }
    if (!(use_net && L.mlp_h)) {
      const float hp = fmaf(fmaf(fmaf(b[BF_H4 * S], Tf, b[BF_H3 * S]), Tf, b[BF_H2 * S]), Tf,
                            b[BF_H1 * S]);
      cH[i] = fmaf(hp, Tf, b[BF_A0 * S]) + b[BF_A5 * S] * invTf;
    } else {
      cH[i] = cOut[S + i] * invTf;  // the network gives H/R
    }
    float gs = g[0], ge = g[S];
    dot2_term(g[2 * S], g[3 * S], lnT, gs, ge);
    dot2_term(g[4 * S], g[5 * S], invT, gs, ge);
    dot2_term(g[6 * S], g[7 * S], T, gs, ge);
    dot2_term(g[8 * S], g[9 * S], T2, gs, ge);
    dot2_term(g[10 * S], g[11 * S], T3, gs, ge);
    dot2_term(g[12 * S], g[13 * S], T4, gs, ge);
    cG2[i] = gibbs_split(ff_norm(gs, ge));
    const float y = fmaxf(Yi, 0.0f);
    const float ys = (L.alpha_f > 0.0f) ? y * __fdividef(y, L.alpha_f + y) : y;
    cC[i] = rho * ys * f[SF_INVW * S];
  }
  const float cpsum = group_sum<G>(cpp);
  __syncwarp();

  // rates of progress: kf = 2^(lg2 A + beta lg2 T - Ea/R log2e / T) (FP32);
  // kr = kf * 2^(x), x = (dG/RT - dN ln(P_atm/RT)) log2 e = sum nu g2, summed
  // exactly
  const int ktap = st.nhist % N;
  constexpr int kWin = WinRegs<G, NT, MLP>::n;
  if constexpr (kWin > 0) {
    // every reaction elementary and reversible, history row r = reaction r:
    // the tap that leaves the window (written N steps ago) comes off the
    // running sums here, before the slot takes this step's raw rate
#pragma unroll
    for (int j = 0; j < kSpecTrips32; ++j) {
      const int r = l + G * j;
      if (r >= R) break;
      const float4 rx = tb.rxf[r];
      const int4 ri = tb.ri[r];
      const int a0 = ri.x & 0xFF, a1 = (ri.x >> 8) & 0xFF;
      const int p0 = (ri.x >> 16) & 0xFF, p1 = (ri.x >> 24) & 0xFF;
      const float lg2kf = fmaf(rx.y, lg2Tf, rx.x) - rx.z * invTf;
      const float q = ex2f(lg2kf) * cC[a0] * cC[a1] - reverse_term(cG2, cC, a0, a1, p0, p1, lg2kf);
      float rof = 1.0f;
      if (L.dft_on) {
        float* slot = cHist + r * NP + ktap;
        if (j < kWin) {
          const float xo = *slot;
          win_s[j] -= xo;
          win_a[j] -= fabsf(xo);
        }
        *slot = q;
        rof = cRof[r];
      }
      cQ[r] = q * rof;
    }
  } else {
#pragma unroll 2  // two reactions per trip (measured)
  for (int r = l; r < R; r += G) {
    const float4 rx = tb.rxf[r];
    const int4 ri = tb.ri[r];
    const int a0 = ri.x & 0xFF, a1 = (ri.x >> 8) & 0xFF;
    const int p0 = (ri.x >> 16) & 0xFF, p1 = (ri.x >> 24) & 0xFF;
    const float lg2kf = fmaf(rx.y, lg2Tf, rx.x) - rx.z * invTf;
    if (mGeneral(L)) {
      // real stoichiometry and orders: C^a = 2^(a lg2 C); the exponent
      // x = sum nu g2 of Eq. 30 summed exactly with the products' errors
      // (an unused slot: species S, lg2 C = 0, order and nu 0)
      const float* rg = tb.rg + r * 8;
      float lq = fmaf(rg[4], lg2f_approx(cC[a0]), lg2kf);
      lq = fmaf(rg[5], lg2f_approx(cC[a1]), lq);
      float q = ex2f(lq), rof = 1.0f;
      if (ri.z) {
        float sx = 0.0f, e = 0.0f;
        pair_add_scaled(rg[2], cG2[p0], sx, e);
        pair_add_scaled(rg[0], cG2[a0], sx, e);
        pair_add_scaled(rg[1], cG2[a1], sx, e);
        pair_add_scaled(rg[3], cG2[p1], sx, e);
        float lr = fmaf(rg[6], lg2f_approx(cC[p0]), lg2kf + (sx + e));
        lr = fmaf(rg[7], lg2f_approx(cC[p1]), lr);
        q -= ex2f(lr);
        if (L.dft_on) {
          cHist[ri.w * NP + ktap] = q;
          rof = cRof[ri.w];
        }
      }
      cQ[r] = q * rof;
      continue;
    }
    float q = ex2f(lg2kf) * cC[a0] * cC[a1];
    float rof = 1.0f;
    if (ri.z) {
      q -= reverse_term(cG2, cC, a0, a1, p0, p1, lg2kf);
      if (L.dft_on) {
        cHist[ri.w * NP + ktap] = q;
        rof = cRof[ri.w];
      }
    }
    cQ[r] = q * rof;
  }
  }
  __syncwarp();

  // production rates, dY/dt, dT/dt terms and the limiter (FP32)
  const float invRho = 1.0f / rho;
  float hwp = 0.0f, tmin = __int_as_float(0x7f800000);  // +inf
  for (int i = l; i < S; i += G) {
    float wd = 0.0f;
    for (int k = tb.gptr[i]; k < tb.gptr[i + 1]; ++k) {
      const int e = tb.gent[k];
      wd = fmaf(mGeneral(L) ? tb.gnu[k] : nu_of_code(e), cQ[e >> 4], wd);
    }
    const float ri = tb.spf[SF_W * S + i] * wd * invRho;
    hwp = fmaf(cH[i], wd, hwp);
    cC[i] = ri;
    const float rstar = fmaxf(-ri, 1.0e-30f);
    const float Yi = cYh[i];
    const float ystar = (Yi < 1.0e-20f) ? 1.0f : 0.9f * Yi;
    tmin = fminf(tmin, __fdividef(fminf(L.y_step_max_f, ystar), rstar));
  }
  const float hw = group_sum<G>(hwp);
  tmin = group_min<G>(tmin);
  const float dTdt = -(Tf * hw) / (rho * cpsum);
  // h = min(tmin, t_f delta_max), the last step ends at t_f: decided in FP64
  // as in the FP64 path (all >= 0, so the comparisons run on the bit
  // patterns); h as a float pair for the update
  const long long hb = min(dbits((double)tmin), dbits(st.hcap));
  const bool last = hb >= dbits(st.t_rem);
  FF h;
  if (last)
    h = ff_from_double(st.t_rem);
  else if (hb == dbits(st.hcap))
    h = FF{st.hcap_h, st.hcap_l};
  else
    h = FF{tmin, 0.0f};
  st.t_rem = last ? 0.0 : st.t_rem - __longlong_as_double(hb);
  const float hf = h.h;

  // ringing detection and damping (Eqs. 8-13), FP32
  if (L.dft_on) {
    const bool full = (st.nhist + 1 >= N);
    const float tol_freq = L.tol_freq_f, tol_ring = L.tol_ring_f;
    const float r_fac = L.r_fac_f;
    // Eqs. 10-13 for a full window hw with sum s (storage order) and sum of
    // |x| a: the high bins only where D0 < Tol_freq and D0 < Tol_ring a
    // (every |X_j| <= a, so otherwise Eq. 10 cannot hold)
    auto next_rof = [&](const float* hw, float s, float a, float rof) -> float {
      const float D0 = fabsf(s);
      float rstar = r_fac;
      if (D0 < tol_freq && D0 < tol_ring * a) {
        const float inv = 1.0f / a;
        const float max2 = hi_bins_max2<NT>(hw, N, tb.tw, L.n_hi_bins, inv);
        const float d = D0 * inv;
        if (d * d < tol_ring * tol_ring * max2) rstar = L.inv_r_fac_f;
      }
      return fmaxf(fminf(rof * rstar, 1.0f), L.rof_min_f);
    };
    // the window sum (storage order) and sum of |x| in one pass
    auto window_sums = [&](const float* hw, float& s, float& a) {
      s = 0.0f;
      a = 0.0f;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        const float v = hw[m];
        s += v;
        a += fabsf(v);
      }
    };
    if constexpr (kWin > 0) {
      // exact sums once per window (the first full step and every N steps
      // after), running sums in between
      const bool refresh = (st.nhist + 1) % N == 0;
#pragma unroll
      for (int j = 0; j < kSpecTrips32; ++j) {
        const int w = l + G * j;
        if (w >= Rrev) break;
        float* hw = cHist + w * NP;
        const float x = hw[ktap] * hf;
        hw[ktap] = x;
        float rof = cRof[w];
        if (full) {
          float sw, aw;
          if (j < kWin && !refresh) {
            win_s[j] += x;
            win_a[j] += fabsf(x);
            sw = win_s[j];
            aw = win_a[j];
          } else {
            window_sums(hw, sw, aw);
            if (j < kWin) {
              win_s[j] = sw;
              win_a[j] = aw;
            }
          }
          rof = next_rof(hw, sw, aw, rof);
        } else {
          rof = fminf(rof * r_fac, 1.0f);
        }
        cRof[w] = rof;
      }
    } else {
      for (int w = l; w < Rrev; w += G) {
        float* hw = cHist + w * NP;
        const float x = hw[ktap] * hf;
        hw[ktap] = x;
        float rof = cRof[w];
        if (full) {
          float sw, aw;
          window_sums(hw, sw, aw);
          rof = next_rof(hw, sw, aw, rof);
        } else {
          rof = fminf(rof * r_fac, 1.0f);
        }
        cRof[w] = rof;
      }
    }
    st.nhist += 1;
  }

  // forward Euler (Eq. 18) in float pairs
  bool bad = false;
  for (int i = l; i < S; i += G) {
    const FF y = ff_add_mul(FF{cYh[i], cYl[i]}, h, cC[i]);
    cYh[i] = y.h;
    cYl[i] = y.l;
    bad = bad || !isfinite(y.h);
  }
  const float pT = __fmul_rn(h.h, dTdt);
  float peT = fmaf(h.h, dTdt, -pT);
  peT = fmaf(h.l, dTdt, peT);
  float sT, tT;
  two_sum(T.h, pT, sT, tT);
  const FF Tn = fast_two_sum(sT, tT + (T.l + peT));
  st.Th = Tn.h;
  st.Tl = Tn.l;
  st.it += 1;
  // ln T for the next step: ln T' = ln T + ln(1 + u), u = (T' - T)/T =
  // h dT/dt / T, from the series while |u| <= 2^-7; the FP64 log every 256
  // steps and on larger changes keeps the accumulated rounding below ~1e-12
  const FF u = ff_mul(FF{pT, peT}, invT);
  FF lnTn;
  if (fabsf(u.h) <= 0x1p-7f && (st.it & 255) != 0)
    lnTn = ff_add(lnT, ff_log1p_small(u));
  else
    lnTn = ff_from_double(log(ff_to_double(Tn)));
  st.lnTh = lnTn.h;
  st.lnTl = lnTn.l;
  bad = group_any<G>(bad) || !isfinite(Tn.h);
  __syncwarp();
  if (bad) return 2;
  if (ff_below(Tn, 200.0f, 0.0f) || Tn.h > 6000.0f || (Tn.h == 6000.0f && Tn.l > 0.0f)) return 3;
  if (last) return 0;
  if (st.it >= L.max_iters) return 1;
  return -1;
}

// Shared-memory pointers of one resident cell of the mixed kernels.
struct MixedCell {
  float2* G2;
  float* Yh;  // Y as float pairs: high parts (the FP32 view of Y) ...
  float* Yl;  // ... and low parts
  float* C;
  float* H;
  float* Q;
  float* Hist;
  float* Rof;
};

// net: the cell of a network kernel (its rate array also holds the network's
// activations and outputs, mixed_q_len).
__device__ __forceinline__ MixedCell mixed_cell(const Launch& L, unsigned char* base,
                                                bool net) {
  MixedCell c;
  c.G2 = reinterpret_cast<float2*>(base);  // S + 1 (the unused-slot entry)
  c.Yh = reinterpret_cast<float*>(c.G2 + mS(L) + 1);
  c.Yl = c.Yh + mS(L);
  c.C = c.Yl + mS(L);                        // S + 1
  c.H = c.C + mS(L) + 1;
  c.Q = c.H + mS(L);
  c.Hist = c.Q + mixed_q_len(mS(L), mR(L), net);  // [Rrev][N | 1]
  c.Rof = c.Hist + (L.dft_n | 1) * mRrev(L);
  return c;
}

// Zeroes a cell block's Y and sets the unused-slot entries (C = 1, g2 = 0).
template <int G>
__device__ __forceinline__ void init_mixed_cell(const Launch& L, const MixedCell& cs, int l) {
  for (int i = l; i < mS(L); i += G) {
    cs.Yh[i] = 0.0f;
    cs.Yl[i] = 0.0f;
  }
  if (l == 0) {
    cs.C[mS(L)] = 1.0f;
    cs.G2[mS(L)] = make_float2(0.0f, 0.0f);
  }
  __syncwarp();
}

// Stages the mechanism tables of the mixed kernels in shared memory.
__device__ __forceinline__ TablesF stage_tables_mixed(const Launch& L, unsigned char* smem_raw) {
  const int S = mS(L), R = mR(L);
  float4* s_rxf = reinterpret_cast<float4*>(smem_raw);
  int4* s_ri = reinterpret_cast<int4*>(s_rxf + R);
  float* s_spf = reinterpret_cast<float*>(s_ri + R);
  float* s_tw = s_spf + S * SF_ROWS;
  int* s_gptr = reinterpret_cast<int*>(s_tw + L.n_hi_bins * 2 * L.dft_n);
  int* s_gent = s_gptr + S + 1;
  for (int t = threadIdx.x; t < R; t += blockDim.x) s_rxf[t] = L.rx_tab_f[t];
  for (int t = threadIdx.x; t < R; t += blockDim.x) s_ri[t] = L.rx_idx_m[t];
  for (int t = threadIdx.x; t < S * SF_ROWS; t += blockDim.x) s_spf[t] = L.sp_tab_f[t];
  for (int t = threadIdx.x; t < L.n_hi_bins * 2 * L.dft_n; t += blockDim.x) s_tw[t] = L.dft_tw_f[t];
  for (int t = threadIdx.x; t <= S; t += blockDim.x) s_gptr[t] = L.g_ptr[t];
  for (int t = threadIdx.x; t < L.n_gather; t += blockDim.x) s_gent[t] = L.g_ent[t];
  float* s_rg = nullptr;
  float* s_gnu = nullptr;
  if (mGeneral(L)) {  // after the 16-byte-aligned base tables
    s_rg = reinterpret_cast<float*>(smem_raw + table_smem_bytes_mixed(S, R, L.n_gather,
                                                                      L.n_hi_bins, L.dft_n, 0));
    s_gnu = s_rg + R * 8;
    for (int t = threadIdx.x; t < R * 8; t += blockDim.x) s_rg[t] = L.rg_tab_f[t];
    for (int t = threadIdx.x; t < L.n_gather; t += blockDim.x) s_gnu[t] = L.g_nu_f[t];
  }
  __syncthreads();
  return TablesF{s_spf, s_rxf, s_ri, s_gptr, s_gent, s_tw, s_rg, s_gnu};
}

__device__ __forceinline__ void set_mixed_scalars(CellState& st) {
  const FF T = ff_from_double(st.T);
  const FF lnT = ff_from_double(log(st.T));
  const FF hc = ff_from_double(st.hcap);
  st.Th = T.h;
  st.Tl = T.l;
  st.lnTh = lnT.h;
  st.lnTl = lnT.l;
  st.hcap_h = hc.h;
  st.hcap_l = hc.l;
}

__device__ __forceinline__ CellState idle_cell_state() {
  CellState st;
  st.cell = -1;
  st.T = 1000.0;
  st.P = kPatm;
  st.t_rem = 1.0;
  st.dt = 1.0;
  st.hcap = 0.01;
  st.lc = 0;
  st.b = 0;
  st.it = 0;
  st.nhist = 0;
  set_mixed_scalars(st);
  return st;
}

// Claims cell c for the group: finds its batch or request and loads its state.
template <int G>
__device__ __forceinline__ void load_mixed_cell(const Launch& L, long long c, int l,
                                                MixedCell& cs, CellState& st, float& Pf) {
  if (L.serve) {
    st.b = serve_find_slot(L, c, st.lc);
    if (st.b < 0) {  // dropped: counted in ctl->dropped
      st.b = 0;
      return;
    }
  } else {
    st.b = find_batch(L, c);
    st.lc = L.nb > 0 ? c - L.boff[st.b] : c;
  }
  const int S = mS(L);
  const CellIO io = cell_io(L, st.b);
  const long long lc = st.lc;
  st.cell = c;
  st.T = __ldcg(io.T + lc);  // L1 bypass: serving reuses these addresses
  st.P = __ldcg(io.P + lc);
  st.dt = io.dt;
  st.hcap = io.dt * L.delta_max;
  st.t_rem = io.dt;
  st.it = 0;
  st.nhist = 0;
  set_mixed_scalars(st);
  Pf = (float)st.P;
  for (int i = l; i < S; i += G) {
    const double y = L.y_soa ? __ldcg(io.Y + (long long)i * io.n + lc) : __ldcg(io.Y + lc * S + i);
    const FF yf = ff_from_double(y);
    cs.Yh[i] = yf.h;
    cs.Yl[i] = yf.l;
  }
  for (int w = l; w < mRrev(L); w += G) cs.Rof[w] = 1.0f;
}

// Writes a finished cell's outputs and frees the group.
template <int G>
__device__ __forceinline__ void store_mixed_cell(const Launch& L, int l, MixedCell& cs,
                                                 CellState& st, int outcome) {
  const int S = mS(L);
  const CellIO io = cell_io(L, st.b);
  const long long c = st.lc;
  if (l == 0) {
    io.T_out[c] = ff_to_double(FF{st.Th, st.Tl});
    io.iters[c] = st.it;
    io.status[c] = (unsigned char)outcome;
  }
  if (L.y_soa)
    for (int i = l; i < S; i += G) io.Y_out[(long long)i * io.n + c] = ff_to_double(FF{cs.Yh[i], cs.Yl[i]});
  else
    for (int i = l; i < S; i += G) io.Y_out[c * S + i] = ff_to_double(FF{cs.Yh[i], cs.Yl[i]});
  if (L.serve) serve_cell_done<G>(L, st.b, io.n, l);
  st.cell = -1;
}

// The mixed-precision persistent kernels' body: lane groups of G lanes, one
// cell each, refilled in place (Sec. 2.4); MLP: with the thermo network
// evaluated by each warp for its cells inside the step (Sec. 3).
// Shared memory: tables | cells (blockDim / G blocks of cell_bytes).
template <int G, int NT, bool MLP>
__device__ __forceinline__ void mixed_kernel_body(const Launch& L, unsigned char* smem_raw) {
  const int S = mS(L);
  const TablesF tb = stage_tables_mixed(L, smem_raw);

  const int group = threadIdx.x / G;
  const int l = threadIdx.x % G;
  const size_t tables = table_smem_bytes_mixed(S, mR(L), L.n_gather, L.n_hi_bins, L.dft_n, mGeneral(L));
  const size_t cell_bytes = cell_smem_bytes_mixed(S, mR(L), mRrev(L), L.dft_n, MLP);
  MixedCell cs = mixed_cell(L, smem_raw + tables + (size_t)group * cell_bytes, MLP);
  init_mixed_cell<G>(L, cs, l);
  // the network's scratch of the warp's first cell (the others follow at
  // cell_bytes strides)
  const int warp = threadIdx.x >> 5;
  float* net_q0 = mixed_cell(L, smem_raw + tables + (size_t)(warp * (32 / G)) * cell_bytes, MLP).Q;
  const int cell_ld = (int)(cell_bytes / sizeof(float));
  // the damper's running window sums (WinRegs; unused elsewhere)
  constexpr int kWin = WinRegs<G, NT, MLP>::n;
  float win_s[kWin > 0 ? kWin : 1], win_a[kWin > 0 ? kWin : 1];
#pragma unroll
  for (int j = 0; j < (kWin > 0 ? kWin : 1); ++j) win_s[j] = win_a[j] = 0.0f;

  const unsigned long long n = (unsigned long long)L.n_cells;
  CellState st = idle_cell_state();
  float Pf = (float)kPatm;
  unsigned long long idle_since = 0;  // serving: when this warp last ran out of work
  bool idle_committed = false;        // serving: counted in ctl->idle_warps
  unsigned idle_sleep = 1000u;        // serving: ns between looks while idle
  int serve_skip = 0;                 // serving: steps before the next look
  bool exhausted = false;
  while (true) {
    long long c = -1;
    if (!L.serve) {
      c = refill<G>(L.counter, n, st.cell < 0, exhausted);
    } else if (serve_skip > 0) {
      --serve_skip;  // nothing was ready recently: look again in a few steps
    } else if (idle_committed) {
      // counted idle: the idle path counts the warp out before it claims
    } else {
      bool none_ready;
      c = serve_refill<G>(L, st.cell < 0, none_ready);
      if (none_ready) serve_skip = 32;
    }
    if (c >= 0) load_mixed_cell<G>(L, c, l, cs, st, Pf);
    __syncwarp();
    if (!__any_sync(0xffffffffu, st.cell >= 0)) {
      if (!L.serve) break;
      // serving: wait for published work; bounded by stop and the grid-wide idle exit
      if (serve_idle(L, idle_since, idle_committed)) break;
      __nanosleep(idle_sleep);
      idle_sleep = min(2u * idle_sleep, 32000u);
      serve_skip = 0;
      continue;
    }
    idle_since = 0;
    idle_sleep = 1000u;
    const int outcome = step_mixed<G, MLP, NT>(L, tb, cs.Yh, cs.Yl, cs.G2, cs.C, cs.H, cs.Q,
                                               cs.Hist, cs.Rof, Pf, l, st, net_q0, cell_ld,
                                               win_s, win_a);
    if (st.cell >= 0 && outcome >= 0) store_mixed_cell<G>(L, l, cs, st, outcome);
  }
}

// Mixed-precision persistent kernel, NASA-7 thermo.
template <int G, int NT>
__global__ void __launch_bounds__(kMaxBlockMixed, 1) stev_mixed_kernel(Launch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  mixed_kernel_body<G, NT, false>(L, smem_raw);
}

// Mixed-precision persistent kernel with the thermo network (Sec. 3): cp/R
// (and with L.mlp_h H/RT) from the network, evaluated on the tensor cores by
// each warp for its own cells at the start of every step.
template <int G, int NT>
__global__ void __launch_bounds__(kMaxBlockMixed, 1) stev_mixed_net_kernel(Launch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  mixed_kernel_body<G, NT, true>(L, smem_raw);
}

}  // namespace stev
