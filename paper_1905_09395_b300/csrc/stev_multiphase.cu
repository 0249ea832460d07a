// STEV on the paper's multiphase (gas-solid) coal gasification cells: Sec.
// 7.2, reactions 31-41 with the rate laws of Eqs. 42-56 and Table 2's
// constants, integrated by the same method as the single-phase path: the
// limiter of Eqs. 1-5, the ringing damper of Eqs. 8-14 on the reversible
// water-gas shift, forward Euler (Eq. 18), each cell to its own end (Sec.
// 2.4).  FP64 throughout.
//
// A cell is a record of 24 doubles: gas mass fractions of O2 CO CO2 CH4 H2
// H2O H2S C3H6 HCN C2H4 C2H6 Tar SO3 N2 (14), solid mass fractions of CV
// (volatile matter) CC (fixed carbon) CM (moisture) CA (ash) (4), T_g, T_s
// (K), eps_s, rho_s (kg/m^3, the solid material density), d_p (m), P (Pa):
// with eps_g = 1 - eps_s and rho_g, the 26 variables per cell the paper
// counts.  What the kernel integrates, and why (the paper prints the
// kinetics, not the cell model around them):
//   - reactions 31-41 are molar; Tar's molecular weight is the one that
//     balances Eq. 37, CV's the one that balances Eq. 31; CC is carbon, CM
//     water, CA inert;
//   - each printed rate is a rate of progress in kmol/m^3/s (SI: Table 2's
//     A_WGS = 1/101325 Pa makes A_WGS P the pressure in atm);
//   - the state is the species' partial densities (kg per m^3 of cell), so
//     mass is conserved exactly by the reactions; eps_s follows the solid's
//     mass at constant rho_s, rho_g the gas's mass in eps_g; P is held;
//   - the phase temperatures are held over the step (no phase energy
//     equations or pseudo-species thermochemistry are given), so each rate's
//     Arrhenius factor and the WGS pressure factor are evaluated once per
//     cell;
//   - gamma (Eq. 7) where the rate laws print it, on max(X, 0), with its
//     limit at alpha = 0; fractional powers of max(X, 0);
//   - the limiter takes the 18 mass fractions and their rates of change in
//     their phase.
// One thread per cell (18 species, 11 reactions: the cell fits in
// registers); the WGS ringing history in shared memory, [tap][thread].
#include <cuda_runtime.h>

#include <cmath>

#include "../../include/stev.h"
#include "stev_internal.h"

namespace stev {
namespace mp {

constexpr int kThreads = 128;
constexpr int kNG = 14, kNSp = 18, kNIn = 24;
constexpr int kMaxN = 32;  // DFT window (options.dft_n <= 32)
enum { iO2, iCO, iCO2, iCH4, iH2, iH2O, iH2S, iC3H6, iHCN, iC2H4, iC2H6, iTAR, iSO3, iN2,
       iCV, iCC, iCM, iCA };

// molecular weights (kg/kmol) and their reciprocals, set by the host
struct Weights {
  double w[kNSp];
  double inv[kNSp];
};

struct Params {
  long long n;
  const double* in;
  double* out;
  double* rho_g;
  int* iters;
  unsigned char* status;
  double dt;
  double y_step_max, delta_max, alpha, tol_ring, tol_freq, r_fac, rof_min;
  int dft_n, dft_hi_first, max_iters, dft_on;
  double tw_c[kMaxN / 2 + 1][kMaxN], tw_s[kMaxN / 2 + 1][kMaxN];  // cos, sin of -2 pi j m / N
  Weights mw;
};

// Table 2
constexpr double kApyro = 5.39808917197452e-1, kEpyro = 2.02305749338465e3;
constexpr double kAwgs = 9.86923266716013e-6, kFPwgs = 3.94769306686405e-8;
constexpr double kKFwgs = 2.87480073925354e0, kEFwgs = 8.42570940582151e3;
constexpr double kKRwgs = 1.08482987533646e2, kERwgs = 1.23814194058215e4;
constexpr double kThG4 = -1.74119074065241e0, kThG3 = 6.75755882493237e-1,
                 kThG2 = 2.42994500814316e-1, kThG1 = 1.80861879808380e-1,
                 kThG0 = -1.37554327457087e-1;
constexpr double kThC4 = -1.71305029851856e0, kThC3 = 1.02332704517333e0,
                 kThC2 = -2.12046897502992e-1, kThC1 = -4.34614630452274e-3,
                 kThC0 = 1.00829969505805e-2;
constexpr double kAstg = 3.64422300238124e-5, kFPstg = 2.58573895879595e-7,
                 kEstg = 4.27760404137599e3;
constexpr double kAcg = 1.21674169495915e1, kFPcg = 2.57586972612879e-6,
                 kEcg = 1.76136636997835e4;
constexpr double kAmeg = 1.66401967700346e-8, kEmeg = 9.15910512388742e3;
constexpr double kBetaC = 4.7741935483871e-1;
constexpr double kAcox = 2.16444452624815e1, kEcox = 1.43928313687756e4;
constexpr double kAtox = 2.59900518618807e6, kEtox = 1.50981378963261e4;
constexpr double kAcoox = 7.91515800843217e9, kEcoox = 2.01288244766506e4;
constexpr double kAhox = 1.67426958313306e11, kEhox = 1.50966183574879e4;
constexpr double kAmeox = 1.34383699737932e9, kEmeox = 2.43558776167472e4;
constexpr double kAmr = 1.0061447769396e-1;
constexpr double kRu = 8314.462618;  // J/(kmol K)

__device__ __forceinline__ double gam(double x, double alpha) {
  const double y = fmax(x, 0.0);
  return alpha > 0.0 ? y / (alpha + y) : (y > 0.0 ? 1.0 : 0.0);
}
__device__ __forceinline__ double ppow(double x, double a) { return pow(fmax(x, 0.0), a); }
// the rate laws' half-integer and quarter powers by square roots (a pow costs
// an exp and a log on the FP64 pipe)
__device__ __forceinline__ double psqrt(double x) { return sqrt(fmax(x, 0.0)); }
__device__ __forceinline__ double pqrt(double x) { return sqrt(sqrt(fmax(x, 0.0))); }

// Per-cell constants: the Arrhenius factors at the held temperatures, the WGS
// pressure factor.
struct CellConst {
  double kpyro, kwgs_f, kwgs_r, wgs_p, kstg, kcg, kmeg, kcox, ktox, kcoox, khox, kmeox;
  double rho_s, dp, P;
};

// Eqs. 42-56 at partial densities c: raw rates of progress r[11].
__device__ __forceinline__ void rates(const Params& L, const CellConst& k, const double* c,
                                      double* X, double* r) {
  double mg = 0.0, ms = 0.0;
#pragma unroll
  for (int i = 0; i < kNG; ++i) mg += c[i];
#pragma unroll
  for (int i = kNG; i < kNSp; ++i) ms += c[i];
  const double img = 1.0 / mg, ims = 1.0 / ms;
  double inv_mw = 0.0;
#pragma unroll
  for (int i = 0; i < kNG; ++i) {
    X[i] = c[i] * img;
    inv_mw = fma(X[i], L.mw.inv[i], inv_mw);
  }
#pragma unroll
  for (int i = kNG; i < kNSp; ++i) X[i] = c[i] * ims;
  const double es = ms / k.rho_s, eg = 1.0 - es, rg = mg / eg, mwg = 1.0 / inv_mw;
  const double al = L.alpha;
  const double ratio = X[iCA] > 0.0 ? X[iCC] / X[iCA] : (X[iCC] > 0.0 ? INFINITY : 0.0);
  const double th = fmax(0.0, fmin(1.0, kBetaC * ratio));  // Eq. 44
  const double ph = 1.0 - th;                               // Eq. 45
  const double ph2 = ph * ph, ph3 = ph2 * ph, ph4 = ph3 * ph, ph5 = ph4 * ph;
  const double aG = ph5 + kThG4 * ph4 + kThG3 * ph3 + kThG2 * ph2 + kThG1 * th + kThG0;  // Eq. 46
  const double aC = ph5 + kThC4 * ph4 + kThC3 * ph3 + kThC2 * ph2 + kThC1 * th + kThC0;
  const double solid_cc = es * k.rho_s * X[iCC] * gam(X[iCC], al);
  const double pw = mwg * k.P;  // P / (mole fraction / mass fraction) scale
  r[0] = k.kpyro * es * k.rho_s * X[iCV] * gam(X[iCV], al);                            // Eq. 42
  r[1] = eg * es * k.rho_s * k.wgs_p *                                                  // Eq. 43
         (k.kwgs_f * X[iCO] * X[iH2O] * gam(X[iCO], al) * gam(X[iH2O], al) -
          k.kwgs_r * X[iCO2] * X[iH2] * gam(X[iCO2], al) * gam(X[iH2], al));
  r[2] = k.kstg * aG * solid_cc * ppow(pw * X[iH2O] / 18.01530, 0.98) /                // Eq. 47
         (1.0 + kFPstg * (pw * X[iH2] / 2.01588));
  r[3] = k.kcg * aG * solid_cc * ppow(pw * X[iCO2] / 44.00980, 0.56) /                 // Eq. 48
         (1.0 + kFPcg * (pw * X[iCO] / 28.01040));
  r[4] = k.kmeg * aG * solid_cc * (pw * X[iH2] / 2.01588);                              // Eq. 49
  r[5] = aC * k.kcox * gam(X[iO2], al) * gam(X[iCC], al) *                              // Eq. 50
         ppow(pw * X[iO2] / 31.9988, 0.73) * es / k.dp;
  const double rg_h = sqrt(rg), rg_q = sqrt(rg_h);
  const double rg175 = rg * rg_h * rg_q, rg15 = rg * rg_h;
  const double o2_q = pqrt(X[iO2]), o2_h = psqrt(X[iO2]);
  r[6] = k.ktox * eg * rg175 * (fmax(X[iO2], 0.0) * o2_h) * pqrt(X[iTAR]) *              // Eq. 52
         gam(X[iO2], al) * gam(X[iTAR], al);
  r[7] = k.kcoox * eg * rg175 * o2_q * X[iCO] * psqrt(X[iH2O]) *                         // Eq. 53
         gam(X[iO2], al) * gam(X[iCO], al);
  r[8] = k.khox * eg * rg * rg * X[iO2] * X[iH2] * gam(X[iO2], al) * gam(X[iH2], al);   // Eq. 54
  r[9] = k.kmeox * eg * rg15 * ppow(X[iO2], 1.3) * ppow(X[iCH4], 0.2) *                  // Eq. 55
         gam(X[iO2], al) * gam(X[iCH4], al);
  r[10] = kAmr * gam(X[iCM], al) * es / k.dp;                                            // Eq. 56
}

// Molar production of each species from the rates of progress q (reactions
// 31-41, written out: reactants negative).
__device__ __forceinline__ void production(const double* q, double* wd) {
  wd[iCV] = -q[0];
  wd[iCO] = 0.242057 * q[0] - q[1] + q[2] + 2.0 * q[3] - q[7];
  wd[iCO2] = 0.0987274 * q[0] + q[1] - q[3] + q[5] + 25.1144 * q[6] + q[7] + q[9];
  wd[iCH4] = 0.229174 * q[0] + q[4] - q[9];
  wd[iH2] = 0.0852648 * q[0] + q[1] + q[2] - 2.0 * q[4] - q[8];
  wd[iH2O] = 0.198778 * q[0] - q[1] - q[2] + 11.9133 * q[6] + q[8] + 2.0 * q[9] + q[10];
  wd[iH2S] = 0.0112077 * q[0];
  wd[iC3H6] = 0.024509 * q[0];
  wd[iHCN] = 0.0266777 * q[0];
  wd[iC2H4] = 0.0473162 * q[0];
  wd[iC2H6] = 0.008257 * q[0];
  wd[iTAR] = 0.02146 * q[0] - q[6];
  wd[iSO3] = 0.0881788 * q[6];
  wd[iN2] = 0.543006 * q[6];
  wd[iO2] = -q[5] - 28.6409 * q[6] - 0.5 * q[7] - 0.5 * q[8] - 2.0 * q[9];
  wd[iCC] = -q[2] - q[3] - q[4] - q[5];
  wd[iCM] = -q[10];
  wd[iCA] = 0.0;
}

__global__ void __launch_bounds__(kThreads) stev_mp_kernel(const Params L) {
  __shared__ double hist_s[kMaxN][kThreads];
  const long long cell = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= L.n) return;
  const double* in = L.in + cell * kNIn;
  const double* w = L.mw.w;
  const double Tg = in[18], Ts = in[19];
  CellConst k;
  k.rho_s = in[21];
  k.dp = in[22];
  k.P = in[23];
  k.kpyro = kApyro * exp(-kEpyro / Ts);
  k.kwgs_f = kKFwgs * exp(-kEFwgs / Tg);
  k.kwgs_r = kKRwgs * exp(-kERwgs / Tg);
  k.wgs_p = pow(kAwgs * k.P, -kFPwgs * k.P + 0.5);
  k.kstg = kAstg * exp(-kEstg / Ts);
  k.kcg = kAcg * exp(-kEcg / Ts);
  k.kmeg = kAmeg * exp(-kEmeg / Ts);
  k.kcox = kAcox * exp(-kEcox / (0.5 * Tg + 0.5 * Ts));  // Eq. 51: T_film
  k.ktox = kAtox * exp(-kEtox / Tg);
  k.kcoox = kAcoox * exp(-kEcoox / Tg);
  k.khox = kAhox * exp(-kEhox / Tg);
  k.kmeox = kAmeox * exp(-kEmeox / Tg);
  // initial partial densities: rho_g from the ideal gas law
  double c[kNSp];
  double inv_mw = 0.0;
#pragma unroll
  for (int i = 0; i < kNG; ++i) inv_mw += in[i] / w[i];  // once per cell
  const double rg0 = k.P / (inv_mw * kRu * Tg);
  const double es0 = in[20];
#pragma unroll
  for (int i = 0; i < kNG; ++i) c[i] = (1.0 - es0) * rg0 * in[i];
#pragma unroll
  for (int i = kNG; i < kNSp; ++i) c[i] = es0 * k.rho_s * in[i];

  const int N = L.dft_n;
  double* hist = &hist_s[0][threadIdx.x];  // tap m at hist[m * kThreads]
  double rOF = 1.0, t_rem = L.dt;
  const double hcap = L.dt * L.delta_max;
  long long nhist = 0;
  int it = 0, status = STEV_CELL_OK;
  double X[kNSp], r[11], wd[kNSp];
  while (true) {
    rates(L, k, c, X, r);
    const double r_wgs = r[1];
    r[1] *= rOF;  // Eq. 14
    production(r, wd);
    double dmg = 0.0, dms = 0.0;
#pragma unroll
    for (int i = 0; i < kNSp; ++i) {
      wd[i] *= w[i];  // dc_i/dt, kg/m^3/s
      if (i < kNG) dmg += wd[i]; else dms += wd[i];
    }
    double mg = 0.0, ms = 0.0;
#pragma unroll
    for (int i = 0; i < kNG; ++i) mg += c[i];
#pragma unroll
    for (int i = kNG; i < kNSp; ++i) ms += c[i];
    // Eqs. 1-5 on the phase mass fractions
    double tstar = INFINITY;
    const double img = 1.0 / mg, ims = 1.0 / ms;
#pragma unroll
    for (int i = 0; i < kNSp; ++i) {
      const double iM = i < kNG ? img : ims, dM = i < kNG ? dmg : dms;
      const double dX = (wd[i] - X[i] * dM) * iM;
      const double rstar = fmax(-dX, 1.0e-30);
      const double ystar = (X[i] < 1.0e-20) ? 1.0 : 0.9 * X[i];
      tstar = fmin(tstar, fmin(L.y_step_max, ystar) / rstar);
    }
    double h = fmin(tstar, hcap);
    const bool last = h >= t_rem;
    if (last) h = t_rem;
    if (L.dft_on) {
      const int m0 = (int)(nhist % N);
      hist[m0 * kThreads] = r_wgs * h;  // Eq. 8
      if (nhist + 1 >= N) {
        double re = 0.0;
        for (int m = 0; m < N; ++m) re += hist[m * kThreads];
        const double D0 = fabs(re);
        double maxhf = 0.0;
        for (int j = L.dft_hi_first; j <= N / 2; ++j) {
          double a = 0.0, b = 0.0;
          for (int m = 0; m < N; ++m) {
            const double x = hist[m * kThreads];
            a = fma(x, L.tw_c[j][m], a);
            b = fma(x, L.tw_s[j][m], b);
          }
          maxhf = fmax(maxhf, hypot(a, b));
        }
        const bool ring = D0 < L.tol_ring * maxhf, eq = D0 < L.tol_freq;  // Eqs. 10-12
        rOF = fmax(fmin(rOF * (ring && eq ? 1.0 / L.r_fac : L.r_fac), 1.0), L.rof_min);
      } else {
        rOF = fmin(rOF * L.r_fac, 1.0);
      }
      ++nhist;
    }
    bool finite = true;
#pragma unroll
    for (int i = 0; i < kNSp; ++i) {
      c[i] = fma(h, wd[i], c[i]);  // Eq. 18
      finite = finite && isfinite(c[i]);
    }
    t_rem -= h;
    ++it;
    if (!finite) { status = STEV_CELL_NONFINITE; break; }
    if (last) break;
    if (it >= L.max_iters) { status = STEV_CELL_MAXITER; break; }
  }
  double mg = 0.0, ms = 0.0;
#pragma unroll
  for (int i = 0; i < kNG; ++i) mg += c[i];
#pragma unroll
  for (int i = kNG; i < kNSp; ++i) ms += c[i];
  double* out = L.out + cell * kNIn;
#pragma unroll
  for (int i = 0; i < kNG; ++i) out[i] = c[i] / mg;
#pragma unroll
  for (int i = kNG; i < kNSp; ++i) out[i] = c[i] / ms;
  const double es = ms / k.rho_s;
  out[18] = Tg;
  out[19] = Ts;
  out[20] = es;
  out[21] = k.rho_s;
  out[22] = k.dp;
  out[23] = k.P;
  if (L.rho_g) L.rho_g[cell] = mg / (1.0 - es);
  L.iters[cell] = it;
  L.status[cell] = (unsigned char)status;
}

// Molecular weights (C 12.011, H 1.00794, O 15.9994 as Eqs. 47-50's
// divisors imply; N, S standard); Tar balancing Eq. 37, CV Eq. 31.
static Weights weights() {
  const double C = 12.011, H = 1.00794, O = 15.9994, Nn = 14.0067, S = 32.065;
  Weights m{};
  double* w = m.w;
  w[iO2] = 2 * O;
  w[iCO] = C + O;
  w[iCO2] = C + 2 * O;
  w[iCH4] = C + 4 * H;
  w[iH2] = 2 * H;
  w[iH2O] = 2 * H + O;
  w[iH2S] = 2 * H + S;
  w[iC3H6] = 3 * C + 6 * H;
  w[iHCN] = H + C + Nn;
  w[iC2H4] = 2 * C + 4 * H;
  w[iC2H6] = 2 * C + 6 * H;
  w[iSO3] = S + 3 * O;
  w[iN2] = 2 * Nn;
  w[iCC] = C;
  w[iCM] = w[iH2O];
  w[iCA] = 60.0843;
  w[iTAR] = 25.1144 * w[iCO2] + 11.9133 * w[iH2O] + 0.0881788 * w[iSO3] + 0.543006 * w[iN2] -
            28.6409 * w[iO2];
  w[iCV] = 0.242057 * w[iCO] + 0.0987274 * w[iCO2] + 0.229174 * w[iCH4] + 0.0852648 * w[iH2] +
           0.198778 * w[iH2O] + 0.0112077 * w[iH2S] + 0.024509 * w[iC3H6] +
           0.0266777 * w[iHCN] + 0.0473162 * w[iC2H4] + 0.008257 * w[iC2H6] +
           0.02146 * w[iTAR];
  for (int i = 0; i < kNSp; ++i) m.inv[i] = 1.0 / w[i];
  return m;
}

}  // namespace mp
}  // namespace stev

extern "C" stev_status stev_mp_solve(long n_cells, const double* cells, double dt_cfd,
                                     const stev_options* opt, double* cells_out, double* rho_g,
                                     int* iters, unsigned char* cell_status, void* stream) {
  using namespace stev;
  host::clear_error();
  if (n_cells < 0) return host::fail(STEV_EINVAL, "n_cells < 0");
  if (!(dt_cfd > 0.0) || !std::isfinite(dt_cfd)) return host::fail(STEV_EINVAL, "dt_cfd must be finite and > 0");
  if (n_cells == 0) return STEV_OK;
  if (!cells || !cells_out || !iters || !cell_status) return host::fail(STEV_EINVAL, "NULL array");
  stev_options o;
  stev_default_options(&o);
  if (opt) o = *opt;
  if (!(o.y_step_max > 0.0) || !(o.delta_max > 0.0 && o.delta_max <= 1.0) || !(o.alpha >= 0.0) ||
      o.dft_n < 2 || o.dft_n > mp::kMaxN || o.dft_hi_first < 1 || o.dft_hi_first > o.dft_n / 2 ||
      !(o.r_fac > 0.0) || !(o.rof_min > 0.0 && o.rof_min <= 1.0) || o.max_iters < 1)
    return host::fail(STEV_EINVAL, "options out of range");
  mp::Params L{};
  L.n = n_cells;
  L.in = cells;
  L.out = cells_out;
  L.rho_g = rho_g;
  L.iters = iters;
  L.status = cell_status;
  L.dt = dt_cfd;
  L.y_step_max = o.y_step_max;
  L.delta_max = o.delta_max;
  L.alpha = o.alpha;
  L.tol_ring = o.tol_ring;
  L.tol_freq = o.tol_freq;
  L.r_fac = o.r_fac;
  L.rof_min = o.rof_min;
  L.dft_n = o.dft_n;
  L.dft_hi_first = o.dft_hi_first;
  L.max_iters = o.max_iters;
  L.dft_on = o.dft_on;
  for (int j = 0; j <= o.dft_n / 2; ++j)
    for (int m = 0; m < o.dft_n; ++m) {
      const double a = -2.0 * M_PI * (double)j * (double)m / (double)o.dft_n;
      L.tw_c[j][m] = std::cos(a);
      L.tw_s[j][m] = std::sin(a);
    }
  L.mw = mp::weights();
  const unsigned blocks = (unsigned)((n_cells + mp::kThreads - 1) / mp::kThreads);
  mp::stev_mp_kernel<<<blocks, mp::kThreads, 0, (cudaStream_t)stream>>>(L);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return host::fail(STEV_ECUDA, "multiphase kernel: %s", cudaGetErrorString(e));
  return STEV_OK;
}
