// Plain FP64 STEV: the persistent, compacting step kernel.
//
// A group of G lanes (G = 8, 16 or 32, chosen per mechanism) integrates one
// cell at a time.  Lanes split the species (i = lane, lane+G, ...) and the
// reactions (r = lane, lane+G, ...) of their cell.  Every piece of a resident
// cell's state lives in shared memory: Y, the gamma-stabilised
// concentrations, G/RT, H/RT, the effective rates of progress, the N-value
// ringing history of every reversible reaction (Eq. 8) and rOF (Eqs. 11-13),
// so a step touches global memory only to read the mechanism once per CTA and
// to load/store whole cells.  Group-wide sums and the limiter's minimum are
// xor-butterfly shuffles, which leave bit-identical results in every lane.
//
// Production rates are gathered species-major: lane i sums nu_ir q_r over
// the reactions of species i in ascending r, the order of the oracle's
// reaction-major scatter, with no atomics.
//
// Variable load (Sec. 2.4): a group whose cell reaches t_f writes it out and
// takes the next cell.  The warp gathers the groups that need work with
// __ballot_sync (one bit per group leader), claims that many consecutive cell
// ids with a single atomicAdd and hands them out by the popcount of the lower
// groups.  Groups left without work once the queue is empty keep stepping a
// dead state (no memory writes) so that the warp's shuffles stay convergent;
// the warp exits when none of its groups holds a cell.  The kernel has no
// waits: every loop is bounded by the mechanism size or max_iters.
#pragma once
#include "stev_common.cuh"

namespace stev {

// One STEV iteration of one cell by its group (Secs. 2.1-2.3, Eq. 18).
// Returns -1 to continue, else the STEV_CELL_* outcome.
template <int G, int kWin>
__device__ __forceinline__ int step_fp64(const Launch& L, const Tables& tb, double* cY, double* cC,
                                         double* cG, double* cH, double* cQ, double* cHist,
                                         double* cRof, int l, CellState& st, double* win_s,
                                         double* win_a) {
  const int S = L.S, R = L.R, Rrev = L.Rrev, N = L.dft_n;
  const double T = st.T;
  const double lnT = log(T);
  const double invT = 1.0 / T;

  // mixture: sum Y/W and ideal-gas density
  double part = 0.0;
  for (int i = l; i < S; i += G) part = fma(cY[i], tb.sp[SP_INVW * S + i], part);
  const double sumYW = group_sum<G>(part);
  const double rho = st.P / (kRu * T * sumYW);

  // thermo (Eqs. 15-16, G/RT) and gamma-stabilised concentrations (Eqs. 6-7)
  double cpp = 0.0;
  for (int i = l; i < S; i += G) {
    const double* sp = tb.sp + i;  // row k of species i at sp[k * S]
    const double* b = sp + (T < sp[SP_TSPLIT * S] ? SP_LOW : SP_HIGH) * S;
    const double Yi = cY[i];
    const double cpR = fma(fma(fma(fma(b[B_A4 * S], T, b[B_A3 * S]), T, b[B_A2 * S]), T,
                               b[B_A1 * S]), T, b[B_A0 * S]);
    const double hp = fma(fma(fma(b[B_H4 * S], T, b[B_H3 * S]), T, b[B_H2 * S]), T, b[B_H1 * S]);
    cH[i] = fma(hp, T, b[B_A0 * S]) + b[B_A5 * S] * invT;
    const double gp = fma(fma(fma(b[B_G4 * S], T, b[B_G3 * S]), T, b[B_G2 * S]), T, b[B_H1 * S]);
    cG[i] = fma(b[B_A0 * S], 1.0 - lnT, fma(b[B_A5 * S], invT, -b[B_A6 * S])) - gp * T;
    cpp = fma(Yi * cpR, sp[SP_INVW * S], cpp);
    const double y = fmax(Yi, 0.0);
    const double ys = (L.alpha > 0.0) ? y * (y / (L.alpha + y)) : y;
    cC[i] = rho * ys * sp[SP_INVW * S];
  }
  const double cpsum = group_sum<G>(cpp);
  __syncwarp();

  // rates of progress (Eqs. 29-30 in log form) and effective rates (Eq. 14)
  const double lnPref = L.ln_patm_over_ru - lnT;  // ln(P_atm / (R T))
  const int ktap = st.nhist % N;
  for (int r = l; r < R; r += G) {
    const double* rx = tb.rx + r * RX_STRIDE;
    const int4 ri = tb.ri[r];
    const int a0 = ri.x & 0xFF, a1 = (ri.x >> 8) & 0xFF;
    const int p0 = (ri.x >> 16) & 0xFF, p1 = (ri.x >> 24) & 0xFF;
    const double lnkf = fma(rx[RX_BETA], lnT, rx[RX_LNA]) - rx[RX_EAR] * invT;
    double q, rof = 1.0;
    if (L.general) {
      // real stoichiometry and orders: slots hold distinct species with their
      // nu (rg[0..3]) and rate-law order (rg[4..7])
      const double* rg = tb.rg + r * 8;
      q = exp(lnkf) * conc_pow(cC[a0], rg[4]);
      if (a1 != kNone) q *= conc_pow(cC[a1], rg[5]);
      if (ri.z) {
        double dG = fma(rg[2], cG[p0], rg[0] * cG[a0]);
        if (a1 != kNone) dG = fma(rg[1], cG[a1], dG);
        if (p1 != kNone) dG = fma(rg[3], cG[p1], dG);
        double rev = exp(fma(-rx[RX_DN], lnPref, lnkf + dG)) * conc_pow(cC[p0], rg[6]);
        if (p1 != kNone) rev *= conc_pow(cC[p1], rg[7]);
        q -= rev;
        if (L.dft_on) {
          cHist[ktap * Rrev + ri.w] = q;
          rof = cRof[ri.w];
        }
      }
      cQ[r] = q * rof;
      continue;
    }
    q = exp(lnkf) * cC[a0];
    if (a1 != kNone) q *= cC[a1];
    if (ri.z) {
      // dG/RT = sum nu G/RT;  ln kr = ln kf - ln K,  ln K = dN ln(P_atm/RT) - dG/RT
      double dG = cG[p0] - cG[a0];
      if (a1 != kNone) dG -= cG[a1];
      if (p1 != kNone) dG += cG[p1];
      double rev = exp(fma(-rx[RX_DN], lnPref, lnkf + dG)) * cC[p0];
      if (p1 != kNone) rev *= cC[p1];
      q -= rev;
      if (L.dft_on) {
        cHist[ktap * Rrev + ri.w] = q;  // raw rate; times h once h is known (Eq. 8)
        rof = cRof[ri.w];
      }
    }
    cQ[r] = q * rof;
  }
  __syncwarp();

  // production rates, dY/dt, adiabatic dT/dt terms and the limiter (Eqs. 1-5)
  const double invRho = 1.0 / rho;
  double hwp = 0.0, num = 1.0, den = 0.0;
  for (int i = l; i < S; i += G) {
    double wd = 0.0;
    for (int k = tb.gptr[i]; k < tb.gptr[i + 1]; ++k) {
      const int e = tb.gent[k];
      wd = fma(L.general ? tb.gnu[k] : kNuOf[e & 15], cQ[e >> 4], wd);
    }
    const double ri = tb.sp[SP_W * S + i] * wd * invRho;
    hwp = fma(cH[i], wd, hwp);
    cC[i] = ri;  // concentrations are no longer needed: keep dY/dt here
    const double rstar = fmax(-ri, 1.0e-30);
    const double Yi = cY[i];
    const double ystar = (Yi < 1.0e-20) ? 1.0 : 0.9 * Yi;
    const double nn = fmin(L.y_step_max, ystar);
    if (den == 0.0 || nn * den < num * rstar) { num = nn; den = rstar; }
  }
  const double hw = group_sum<G>(hwp);
  group_min_frac<G>(num, den);
  const double dTdt = -(T * hw) / (rho * cpsum);
  double h = fmin(num / den, st.dt * L.delta_max);
  const bool last = (h >= st.t_rem);
  if (last) h = st.t_rem;

  // DFT ringing detection and damping (Eqs. 8-13) on reversible reactions.
  // Eq. 9's D0 = |sum of the window| and the sum of |x| of Eq. 10's bound:
  // for a lane's first kWin rows kept as running sums in registers (the tap
  // that leaves at the next step, still in its slot now, comes off them after
  // this step's decision, the new tap goes on at the next step), recomputed
  // from the N taps once per window (the first full step and every N steps
  // after), so their drift stays within a window's roundings; elsewhere summed
  // directly from the taps in storage order.
  if (L.dft_on) {
    const bool full = (st.nhist + 1 >= N);
    const bool refresh = (st.nhist + 1) % N == 0;
    const int knext = (ktap + 1) % N;
    auto damp = [&](int w, bool running, double& ws, double& wa) {
      const double x = cHist[ktap * Rrev + w] * h;
      cHist[ktap * Rrev + w] = x;
      double rof = cRof[w];
      if (full) {
        double s = 0.0, a = 0.0;
        bool have_a = false;
        if (running && !refresh) {
          s = ws + x;
          a = wa + fabs(x);
          have_a = true;
        } else {
          for (int m = 0; m < N; ++m) s += cHist[m * Rrev + w];  // storage order, as Eq. 9's sum
        }
        const double D0 = fabs(s);
        double rstar = L.r_fac;
        if (D0 < L.tol_freq) {  // only then can Eq. 12 damp
          // every |X_j| <= sum |x_m|: a window with D0 >= Tol_ring sum|x_m|
          // cannot ring (Eq. 10), so its high bins are not needed
          if (!have_a) {
            for (int m = 0; m < N; ++m) a += fabs(cHist[m * Rrev + w]);
            have_a = true;
          }
          if (D0 < L.tol_ring * a) {
            // D0 < Tol_ring max|X_j|, compared as squares in units of sum|x_m|
            // (every scaled magnitude is <= 1, so the squares cannot underflow)
            const double inv = 1.0 / a;
            // taps m and N - m paired: cos is even and sin odd in m about
            // N / 2 (tw[b] = cos, sin of -2 pi j m / N), so Re X_j = x_0 +
            // sum (x_m + x_{N-m}) cos_m (+ an even N's middle tap) and Im X_j
            // = sum (x_m - x_{N-m}) sin_m, m = 1 .. (N - 1) / 2
            double max2 = 0.0;
            const double* xw = cHist + w;
            const int half = (N - 1) / 2;
            for (int bb = 0; bb < L.n_hi_bins; ++bb) {
              const double* c = tb.tw + bb * 2 * N;
              double re = xw[0], im = 0.0;
              for (int m = 1; m <= half; ++m) {
                const double xa = xw[m * Rrev], xb = xw[(N - m) * Rrev];
                re = fma(xa + xb, c[m], re);
                im = fma(xa - xb, c[N + m], im);
              }
              if (!(N & 1)) re = fma(xw[(N / 2) * Rrev], c[N / 2], re);
              re *= inv;
              im *= inv;
              max2 = fmax(max2, fma(re, re, im * im));
            }
            const double d = D0 * inv;
            if (d * d < L.tol_ring * L.tol_ring * max2) rstar = 1.0 / L.r_fac;
          }
        }
        rof = fmax(fmin(rof * rstar, 1.0), L.rof_min);
        if (running) {
          if (!have_a)
            for (int m = 0; m < N; ++m) a += fabs(cHist[m * Rrev + w]);
          const double xl = cHist[knext * Rrev + w];  // leaves the window next step
          ws = s - xl;
          wa = a - fabs(xl);
        }
      } else {
        rof = fmin(rof * L.r_fac, 1.0);
      }
      cRof[w] = rof;
    };
    double unused_s = 0.0, unused_a = 0.0;
#pragma unroll
    for (int j = 0; j < kWin; ++j) {
      const int w = l + G * j;
      if (w < Rrev) damp(w, true, win_s[j], win_a[j]);
    }
    for (int w = l + G * kWin; w < Rrev; w += G) damp(w, false, unused_s, unused_a);
    st.nhist += 1;
  }

  // forward Euler (Eq. 18)
  bool bad = false;
  for (int i = l; i < S; i += G) {
    const double y = fma(h, cC[i], cY[i]);
    cY[i] = y;
    bad = bad || !isfinite(y);
  }
  st.T = fma(h, dTdt, T);
  st.t_rem -= h;
  st.it += 1;
  bad = group_any<G>(bad) || !isfinite(st.T);
  __syncwarp();
  if (bad) return 2;                           // STEV_CELL_NONFINITE
  if (st.T < 200.0 || st.T > 6000.0) return 3;  // STEV_CELL_TRANGE
  if (last) return 0;                          // STEV_CELL_OK
  if (st.it >= L.max_iters) return 1;          // STEV_CELL_MAXITER
  return -1;
}

// ---------------------------------------------------------- persistent kernel
// Reversible reactions per lane whose damper window sums are kept running in
// registers (step_fp64): the first five of each lane with 32-lane groups,
// whose cells (19 KB each on 32/150) leave at most 12 per CTA, so the block
// bound of 384 threads gives the registers (170 per thread) for them.
template <int G>
struct Fp64Win {
  static constexpr int n = G == 32 ? 5 : 0;
  static constexpr int block = G == 32 ? 384 : kMaxBlock;
};

template <int G>
__global__ void __launch_bounds__(Fp64Win<G>::block, 1) stev_fp64_kernel(Launch L) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int S = L.S, R = L.R;
  // stage the mechanism tables once per CTA
  double* s_sp = reinterpret_cast<double*>(smem_raw);
  double* s_rx = s_sp + S * SP_STRIDE;
  int4* s_ri = reinterpret_cast<int4*>(s_rx + R * RX_STRIDE);
  double* s_tw = reinterpret_cast<double*>(s_ri + R);
  int* s_gptr = reinterpret_cast<int*>(s_tw + L.n_hi_bins * 2 * L.dft_n);
  int* s_gent = s_gptr + S + 1;
  // species table transposed to [row][S] in shared memory: lane i reading
  // species i then walks consecutive banks (species-major rows 256 bytes apart
  // put every lane on the same bank)
  for (int t = threadIdx.x; t < S * SP_STRIDE; t += blockDim.x)
    s_sp[(t % SP_STRIDE) * S + t / SP_STRIDE] = L.sp_tab[t];
  for (int t = threadIdx.x; t < R * RX_STRIDE; t += blockDim.x) s_rx[t] = L.rx_tab[t];
  for (int t = threadIdx.x; t < R; t += blockDim.x) s_ri[t] = L.rx_idx[t];
  for (int t = threadIdx.x; t < L.n_hi_bins * 2 * L.dft_n; t += blockDim.x) s_tw[t] = L.dft_tw[t];
  for (int t = threadIdx.x; t <= S; t += blockDim.x) s_gptr[t] = L.g_ptr[t];
  for (int t = threadIdx.x; t < L.n_gather; t += blockDim.x) s_gent[t] = L.g_ent[t];
  double* s_rg = nullptr;
  double* s_gnu = nullptr;
  if (L.general) {  // after the 16-byte-aligned base tables
    s_rg = reinterpret_cast<double*>(smem_raw + table_smem_bytes(S, R, L.n_gather, L.n_hi_bins,
                                                                 L.dft_n, 0));
    s_gnu = s_rg + R * 8;
    for (int t = threadIdx.x; t < R * 8; t += blockDim.x) s_rg[t] = L.rg_tab[t];
    for (int t = threadIdx.x; t < L.n_gather; t += blockDim.x) s_gnu[t] = L.g_nu[t];
  }
  __syncthreads();
  const Tables tb{s_sp, s_rx, s_ri, s_gptr, s_gent, s_tw, s_rg, s_gnu};

  // this group's cell area
  const int group = threadIdx.x / G;
  const int l = threadIdx.x % G;
  const size_t tables = table_smem_bytes(S, R, L.n_gather, L.n_hi_bins, L.dft_n, L.general);
  const size_t cell_bytes = cell_smem_bytes_fp64(S, R, L.Rrev, L.dft_n);
  double* cY = reinterpret_cast<double*>(smem_raw + tables + (size_t)group * cell_bytes);
  double* cC = cY + S;
  double* cG = cC + S;
  double* cH = cG + S;
  double* cQ = cH + S;
  double* cHist = cQ + R;
  double* cRof = cHist + L.dft_n * L.Rrev;
  for (int i = l; i < S; i += G) cY[i] = 0.0;

  const unsigned long long n = (unsigned long long)L.n_cells;
  CellState st;
  st.cell = -1;
  st.T = 1000.0;
  st.P = kPatm;
  st.t_rem = 1.0;
  st.dt = 1.0;
  st.lc = 0;
  st.b = 0;
  st.it = 0;
  st.nhist = 0;
  unsigned long long idle_since = 0;  // serving: when this warp last ran out of work
  bool idle_committed = false;        // serving: counted in ctl->idle_warps
  unsigned idle_sleep = 1000u;        // serving: ns between looks while idle
  int serve_skip = 0;                 // serving: steps before the next look
  bool exhausted = false;  // warp-uniform
  // the damper's running window sums (Fp64Win; rewritten at a cell's first
  // full window before they are read)
  constexpr int kWin = Fp64Win<G>::n;
  double win_s[kWin > 0 ? kWin : 1], win_a[kWin > 0 ? kWin : 1];
#pragma unroll
  for (int j = 0; j < (kWin > 0 ? kWin : 1); ++j) win_s[j] = win_a[j] = 0.0;
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
    if (c >= 0 && L.serve) {
      st.b = serve_find_slot(L, c, st.lc);
      if (st.b < 0) {  // dropped: counted in ctl->dropped
        st.b = 0;
        c = -1;
      }
    } else if (c >= 0) {
      st.b = find_batch(L, c);
      st.lc = L.nb > 0 ? c - L.boff[st.b] : c;
    }
    if (c >= 0) {
      const CellIO io = cell_io(L, st.b);
      const long long lc = st.lc;
      st.cell = c;
      st.T = __ldcg(io.T + lc);  // L1 bypass: serving reuses these addresses
      st.P = __ldcg(io.P + lc);
      st.dt = io.dt;
      st.t_rem = io.dt;
      st.it = 0;
      st.nhist = 0;
      if (L.y_soa)
        for (int i = l; i < S; i += G) cY[i] = __ldcg(io.Y + (long long)i * io.n + lc);
      else
        for (int i = l; i < S; i += G) cY[i] = __ldcg(io.Y + lc * S + i);
      for (int w = l; w < L.Rrev; w += G) cRof[w] = 1.0;  // Eq. 11
    }
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
    const int outcome = step_fp64<G, Fp64Win<G>::n>(L, tb, cY, cC, cG, cH, cQ, cHist, cRof, l, st,
                                                    win_s, win_a);
    if (st.cell >= 0 && outcome >= 0) {
      const CellIO io = cell_io(L, st.b);
      const long long c = st.lc;
      if (l == 0) {
        io.T_out[c] = st.T;
        io.iters[c] = st.it;
        io.status[c] = (unsigned char)outcome;
      }
      if (L.y_soa)
        for (int i = l; i < S; i += G) io.Y_out[(long long)i * io.n + c] = cY[i];
      else
        for (int i = l; i < S; i += G) io.Y_out[c * S + i] = cY[i];
      if (L.serve) serve_cell_done<G>(L, st.b, io.n, l);
      st.cell = -1;
    }
  }
}

}  // namespace stev
