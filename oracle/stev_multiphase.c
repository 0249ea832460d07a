/*
 * Plain FP64 CPU oracle of STEV on the paper's multiphase (gas-solid) coal
 * gasification cells: Sec. 7.2, Eqs. 31-56, Table 2 of Buchheit et al.,
 * arXiv:1905.09395.
 *
 * TEST INFRASTRUCTURE ONLY, like stev_oracle.c: nothing in the product path
 * calls, links or executes it, and it shares no code, header, table or
 * constant with the CUDA path.
 *
 * The cell (26 variables, as the paper counts them): gas mass fractions of
 * O2 CO CO2 CH4 H2 H2O H2S C3H6 HCN C2H4 C2H6 Tar SO3 N2 (14), solid mass
 * fractions of CV (volatile matter), CC (fixed carbon), CM (moisture), CA
 * (ash) (4), the gas and solid temperatures T_g, T_s, the volume fractions
 * eps_g = 1 - eps_s and eps_s, the phase densities rho_g and rho_s, the
 * particle diameter d_p and the pressure P.
 *
 * What each function follows:
 *   mp_rates        Eqs. 42-56 (rates of progress of reactions 31-41), with
 *                   gamma of Eq. 7 where the rate laws print it, Eqs. 44-46
 *                   (annealing factors), Eq. 51 (film temperature), and
 *                   Eq. 14 (the damped rate of the reversible WGS);
 *   mp_step_size    Sec. 2.1 Eqs. 1-5 on the 18 mass fractions;
 *   mp_solve_cell   Sec. 2.3 Eqs. 8-14 (ringing history and damper of the
 *                   reversible WGS), Eq. 18 (forward Euler on the species'
 *                   partial densities), Sec. 2.4 (each cell to its own end).
 *
 * Readings where the paper is silent (the same as the single-phase oracle's
 * where they overlap):
 *   - reactions 31-41 are molar; the pseudo-species' molecular weights are
 *     those that balance them: Tar's from Eq. 37, CV's from Eq. 31 (with
 *     Tar's); CC is carbon, CM is water (Eq. 41 moves it to the gas), CA is
 *     inert;
 *   - every rate printed in Eqs. 42-56 is a rate of progress in kmol/m^3/s
 *     (SI; Table 2's A_WGS = 1/101325 Pa turns P in Pa into atm); a species
 *     changes by MW_i * sum_r nu_ir r_r kg/m^3/s;
 *   - the integrated state is the species' partial densities c_i (kg per m^3
 *     of cell): the gas phase holds c_0..c_13, the solid c_14..c_17; each
 *     phase's mass fractions are its c_i over its total; rho_s is the
 *     material density (constant), so eps_s = (solid total) / rho_s, eps_g =
 *     1 - eps_s and rho_g = (gas total) / eps_g; rho_g starts from the ideal
 *     gas law at (P, T_g, MW_g); P is held over the step;
 *   - the phase temperatures are held over the chemistry step (the paper
 *     prints no phase energy equations and no thermochemistry for CV, CC, CM,
 *     CA or Tar);
 *   - gamma (Eq. 7) acts on max(X, 0); alpha = 0 takes its limit (1 for X > 0,
 *     0 otherwise);
 *   - fractional powers act on max(X, 0); ratio X_CC / X_CA of Eq. 44 with
 *     X_CA <= 0 is read as +inf (theta = 1) when X_CC > 0, else 0; Eq. 46's
 *     theta_1 term multiplies theta (vartheta) as printed;
 *   - the limiter (Eqs. 1-5) takes the 18 mass fractions and their rates of
 *     change within their phase, dX_i/dt = (dc_i/dt - X_i dM/dt) / M with M
 *     the phase's total;
 *   - the ringing history (Eq. 8) stores the raw WGS rate times h.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define MP_NG 14
#define MP_NS 4
#define MP_NSP 18
#define MP_NR 11
#define MP_NIN 24  /* per-cell input record: X_g[14] X_s[4] T_g T_s eps_s rho_s d_p P */
#define MP_RU 8314.462618  /* J/(kmol K) */

/* conditioning probe: every rate constant A scaled (default exactly 1) */
#ifndef ORACLE_MP_A_SCALE
#define ORACLE_MP_A_SCALE 1.0
#endif

enum { O2, CO, CO2, CH4, H2, H2O, H2S, C3H6, HCN, C2H4, C2H6, TAR, SO3, N2,
       CV, CC, CM, CA };
enum { PYRO, WGS, STG, CG, MEG, COX, TOX, COOX, HOX, MEOX, MR };

/* atomic weights (kg/kmol) as Eqs. 47-50's divisors imply (C 12.011,
 * H 1.00794, O 15.9994), N and S standard */
#define AW_C 12.011
#define AW_H 1.00794
#define AW_O 15.9994
#define AW_N 14.0067
#define AW_S 32.065

typedef struct {
  double mw[MP_NSP];
  double nu[MP_NR][MP_NSP];  /* molar stoichiometry, reactants < 0 */
} mp_tables;

typedef struct {
  double y_step_max, delta_max, alpha;
  int dft_n, dft_hi_first;
  double tol_ring, tol_freq, r_fac, rof_min;
  int max_iters, dft_on;
} mp_opts;

enum { MP_CELL_OK = 0, MP_CELL_MAXITER = 1, MP_CELL_NONFINITE = 2 };

/* Table 2 */
static const double A_PYRO = 5.39808917197452e-1, EA_PYRO = 2.02305749338465e3;
static const double A_WGS = 9.86923266716013e-6, FP_WGS = 3.94769306686405e-8;
static const double KF_WGS = 2.87480073925354e0, EAF_WGS = 8.42570940582151e3;
static const double KR_WGS = 1.08482987533646e2, EAR_WGS = 1.23814194058215e4;
static const double TH_G[5] = {-1.37554327457087e-1, 1.80861879808380e-1, 2.42994500814316e-1,
                               6.75755882493237e-1, -1.74119074065241e0}; /* theta_0..theta_4 */
static const double TH_C[5] = {1.00829969505805e-2, -4.34614630452274e-3, -2.12046897502992e-1,
                               1.02332704517333e0, -1.71305029851856e0};
static const double A_STG = 3.64422300238124e-5, FP_STG = 2.58573895879595e-7;
static const double EA_STG = 4.27760404137599e3;
static const double A_CG = 1.21674169495915e1, FP_CG = 2.57586972612879e-6;
static const double EA_CG = 1.76136636997835e4;
static const double A_MEG = 1.66401967700346e-8, EA_MEG = 9.15910512388742e3;
static const double BETA_C = 4.7741935483871e-1;
static const double A_COX = 2.16444452624815e1, EA_COX = 1.43928313687756e4;
static const double A_TOX = 2.59900518618807e6, EA_TOX = 1.50981378963261e4;
static const double A_COOX = 7.91515800843217e9, EA_COOX = 2.01288244766506e4;
static const double A_HOX = 1.67426958313306e11, EA_HOX = 1.50966183574879e4;
static const double A_MEOX = 1.34383699737932e9, EA_MEOX = 2.43558776167472e4;
static const double A_MR = 1.0061447769396e-1;

/* Molecular weights and stoichiometry of reactions 31-41. */
void mp_tables_init(mp_tables *t) {
  memset(t, 0, sizeof *t);
  double *w = t->mw;
  w[O2] = 2 * AW_O;
  w[CO] = AW_C + AW_O;
  w[CO2] = AW_C + 2 * AW_O;
  w[CH4] = AW_C + 4 * AW_H;
  w[H2] = 2 * AW_H;
  w[H2O] = 2 * AW_H + AW_O;
  w[H2S] = 2 * AW_H + AW_S;
  w[C3H6] = 3 * AW_C + 6 * AW_H;
  w[HCN] = AW_H + AW_C + AW_N;
  w[C2H4] = 2 * AW_C + 4 * AW_H;
  w[C2H6] = 2 * AW_C + 6 * AW_H;
  w[SO3] = AW_S + 3 * AW_O;
  w[N2] = 2 * AW_N;
  w[CC] = AW_C;
  w[CM] = w[H2O];
  w[CA] = 60.0843;  /* inert: its value changes nothing */
  /* Eq. 37 fixes Tar */
  w[TAR] = 25.1144 * w[CO2] + 11.9133 * w[H2O] + 0.0881788 * w[SO3] + 0.543006 * w[N2] -
           28.6409 * w[O2];
  /* Eq. 31 */
  double (*nu)[MP_NSP] = t->nu;
  nu[PYRO][CV] = -1.0;
  nu[PYRO][CO] = 0.242057;
  nu[PYRO][CO2] = 0.0987274;
  nu[PYRO][CH4] = 0.229174;
  nu[PYRO][H2] = 0.0852648;
  nu[PYRO][H2O] = 0.198778;
  nu[PYRO][H2S] = 0.0112077;
  nu[PYRO][C3H6] = 0.024509;
  nu[PYRO][HCN] = 0.0266777;
  nu[PYRO][C2H4] = 0.0473162;
  nu[PYRO][C2H6] = 0.008257;
  nu[PYRO][TAR] = 0.02146;
  double mcv = 0.0;
  for (int i = 0; i < MP_NSP; ++i)
    if (i != CV) mcv += nu[PYRO][i] * w[i];
  w[CV] = mcv;
  /* Eqs. 32-41 */
  nu[WGS][CO] = -1; nu[WGS][H2O] = -1; nu[WGS][CO2] = 1; nu[WGS][H2] = 1;
  nu[STG][CC] = -1; nu[STG][H2O] = -1; nu[STG][CO] = 1; nu[STG][H2] = 1;
  nu[CG][CC] = -1; nu[CG][CO2] = -1; nu[CG][CO] = 2;
  nu[MEG][CC] = -1; nu[MEG][H2] = -2; nu[MEG][CH4] = 1;
  nu[COX][CC] = -1; nu[COX][O2] = -1; nu[COX][CO2] = 1;
  nu[TOX][TAR] = -1; nu[TOX][O2] = -28.6409; nu[TOX][CO2] = 25.1144; nu[TOX][H2O] = 11.9133;
  nu[TOX][SO3] = 0.0881788; nu[TOX][N2] = 0.543006;
  nu[COOX][CO] = -1; nu[COOX][O2] = -0.5; nu[COOX][CO2] = 1;
  nu[HOX][H2] = -1; nu[HOX][O2] = -0.5; nu[HOX][H2O] = 1;
  nu[MEOX][CH4] = -1; nu[MEOX][O2] = -2; nu[MEOX][CO2] = 1; nu[MEOX][H2O] = 2;
  nu[MR][CM] = -1; nu[MR][H2O] = 1;
}

/* Eq. 7 on max(X, 0); alpha = 0 is its limit: 1 for X > 0, else 0 (a rate
 * law that prints gamma(X) still stops when X is exhausted) */
static double gam(double x, double alpha) {
  double y = x > 0.0 ? x : 0.0;
  if (alpha > 0.0) return y / (alpha + y);
  return y > 0.0 ? 1.0 : 0.0;
}
static double ppow(double x, double a) { return pow(x > 0.0 ? x : 0.0, a); }

/* Phase quantities from the partial densities c[18] (and rho_s):
 * X[18] (each phase's mass fractions), eps_g, eps_s, rho_g, MW_g. */
void mp_phase(const mp_tables *t, const double *c, double rho_s, double *X, double *eps_g,
              double *eps_s, double *rho_g, double *mw_g) {
  double mg = 0.0, ms = 0.0;
  for (int i = 0; i < MP_NG; ++i) mg += c[i];
  for (int i = MP_NG; i < MP_NSP; ++i) ms += c[i];
  for (int i = 0; i < MP_NG; ++i) X[i] = c[i] / mg;
  for (int i = MP_NG; i < MP_NSP; ++i) X[i] = c[i] / ms;
  *eps_s = ms / rho_s;
  *eps_g = 1.0 - *eps_s;
  *rho_g = mg / *eps_g;
  double inv = 0.0;
  for (int i = 0; i < MP_NG; ++i) inv += X[i] / t->mw[i];
  *mw_g = 1.0 / inv;
}

/* Eqs. 42-56: raw rates of progress r[11] (kmol/m^3/s; WGS net, undamped). */
void mp_rates(const mp_tables *t, const mp_opts *o, const double *c, double Tg, double Ts,
              double rho_s, double dp, double P, double *r) {
  double X[MP_NSP], eg, es, rg, mwg;
  mp_phase(t, c, rho_s, X, &eg, &es, &rg, &mwg);
  const double al = o->alpha;
  const double Tfilm = 0.5 * Tg + 0.5 * Ts;                                 /* Eq. 51 */
  /* Eqs. 44-46 */
  double ratio;
  if (X[CA] > 0.0) ratio = X[CC] / X[CA];
  else ratio = X[CC] > 0.0 ? INFINITY : 0.0;
  const double th = fmax(0.0, fmin(1.0, BETA_C * ratio));                 /* Eq. 44 */
  const double ph = 1.0 - th;                                             /* Eq. 45 */
  const double aG = pow(ph, 5) + TH_G[4] * pow(ph, 4) + TH_G[3] * pow(ph, 3) +
                    TH_G[2] * pow(ph, 2) + TH_G[1] * th + TH_G[0];        /* Eq. 46 */
  const double aC = pow(ph, 5) + TH_C[4] * pow(ph, 4) + TH_C[3] * pow(ph, 3) +
                    TH_C[2] * pow(ph, 2) + TH_C[1] * th + TH_C[0];
  const double s = ORACLE_MP_A_SCALE;
  r[PYRO] = s * A_PYRO * es * rho_s * X[CV] * gam(X[CV], al) * exp(-EA_PYRO / Ts);  /* Eq. 42 */
  r[WGS] = s * eg * es * rho_s * pow(A_WGS * P, -FP_WGS * P + 0.5) *               /* Eq. 43 */
           (KF_WGS * X[CO] * X[H2O] * gam(X[CO], al) * gam(X[H2O], al) * exp(-EAF_WGS / Tg) -
            KR_WGS * X[CO2] * X[H2] * gam(X[CO2], al) * gam(X[H2], al) * exp(-EAR_WGS / Tg));
  r[STG] = s * A_STG * aG * es * rho_s * X[CC] * gam(X[CC], al) *                    /* Eq. 47 */
           ppow(mwg * P * X[H2O] / 18.01530, 0.98) /
           (1.0 + FP_STG * (mwg * P * X[H2] / 2.01588)) * exp(-EA_STG / Ts);
  r[CG] = s * A_CG * aG * es * rho_s * X[CC] * gam(X[CC], al) *                      /* Eq. 48 */
          ppow(mwg * P * X[CO2] / 44.00980, 0.56) /
          (1.0 + FP_CG * (mwg * P * X[CO] / 28.01040)) * exp(-EA_CG / Ts);
  r[MEG] = s * A_MEG * aG * es * rho_s * X[CC] * gam(X[CC], al) *                    /* Eq. 49 */
           (mwg * P * X[H2] / 2.01588) * exp(-EA_MEG / Ts);
  r[COX] = s * aC * A_COX * gam(X[O2], al) * gam(X[CC], al) * exp(-EA_COX / Tfilm) * /* Eq. 50 */
           ppow(mwg * P * X[O2] / 31.9988, 0.73) * es / dp;
  r[TOX] = s * A_TOX * exp(-EA_TOX / Tg) * eg * pow(rg, 1.75) * ppow(X[O2], 1.5) *   /* Eq. 52 */
           ppow(X[TAR], 0.25) * gam(X[O2], al) * gam(X[TAR], al);
  r[COOX] = s * A_COOX * exp(-EA_COOX / Tg) * eg * pow(rg, 1.75) * ppow(X[O2], 0.25) * /* Eq. 53 */
            X[CO] * ppow(X[H2O], 0.5) * gam(X[O2], al) * gam(X[CO], al);
  r[HOX] = s * A_HOX * exp(-EA_HOX / Tg) * eg * rg * rg * X[O2] * X[H2] *             /* Eq. 54 */
           gam(X[O2], al) * gam(X[H2], al);
  r[MEOX] = s * A_MEOX * exp(-EA_MEOX / Tg) * eg * pow(rg, 1.5) * ppow(X[O2], 1.3) *  /* Eq. 55 */
            ppow(X[CH4], 0.2) * gam(X[O2], al) * gam(X[CH4], al);
  r[MR] = s * A_MR * gam(X[CM], al) * es / dp;                                     /* Eq. 56 */
}

/* dc_i/dt = MW_i sum_r nu_ir q_r, q = r with the WGS damped (Eq. 14), and each
 * phase's mass-fraction rates dX_i/dt (for the limiter). */
static void mp_derivs(const mp_tables *t, const double *c, const double *q, double *dc,
                      double *dX) {
  for (int i = 0; i < MP_NSP; ++i) {
    double w = 0.0;
    for (int k = 0; k < MP_NR; ++k) w += t->nu[k][i] * q[k];
    dc[i] = t->mw[i] * w;
  }
  double mg = 0.0, ms = 0.0, dmg = 0.0, dms = 0.0;
  for (int i = 0; i < MP_NG; ++i) { mg += c[i]; dmg += dc[i]; }
  for (int i = MP_NG; i < MP_NSP; ++i) { ms += c[i]; dms += dc[i]; }
  for (int i = 0; i < MP_NG; ++i) dX[i] = (dc[i] - (c[i] / mg) * dmg) / mg;
  for (int i = MP_NG; i < MP_NSP; ++i) dX[i] = (dc[i] - (c[i] / ms) * dms) / ms;
}

/* Eqs. 1-5 */
static double mp_step_size(const double *X, const double *dX, double t_f, const mp_opts *o) {
  double tstar = INFINITY;
  for (int i = 0; i < MP_NSP; ++i) {
    double rstar = fmax(-dX[i], 1.0e-30);
    double ystar = (X[i] < 1.0e-20) ? 1.0 : 0.9 * X[i];
    double cand = fmin(o->y_step_max, ystar) / rstar;
    if (cand < tstar) tstar = cand;
  }
  return fmin(tstar, t_f * o->delta_max);
}

/* Eq. 9 */
static double mp_dft_mag(const double *x, int N, int j) {
  double re = 0.0, im = 0.0;
  for (int k = 0; k < N; ++k) {
    double ang = -2.0 * 3.14159265358979323846 * (double)j * (double)k / (double)N;
    re += x[k] * cos(ang);
    im += x[k] * sin(ang);
  }
  return j == 0 ? fabs(re) : hypot(re, im);
}

/* Initial partial densities from an input record (X_g, X_s, T_g, T_s, eps_s,
 * rho_s, d_p, P): rho_g from the ideal gas law. */
void mp_initial(const mp_tables *t, const double *in, double *c) {
  double inv = 0.0;
  for (int i = 0; i < MP_NG; ++i) inv += in[i] / t->mw[i];
  const double mwg = 1.0 / inv, Tg = in[18], es = in[20], rs = in[21], P = in[23];
  const double rg = P * mwg / (MP_RU * Tg);
  for (int i = 0; i < MP_NG; ++i) c[i] = (1.0 - es) * rg * in[i];
  for (int i = MP_NG; i < MP_NSP; ++i) c[i] = es * rs * in[i];
}

/* One cell over t_f = dt (Sec. 2.4).  out: the record with the new X_g, X_s
 * and eps_s (T_g, T_s, rho_s, d_p, P unchanged); rho_g_out (nullable) the
 * final gas density. */
int mp_solve_cell(const mp_tables *t, const mp_opts *o, const double *in, double dt,
                  double *out, double *rho_g_out, int *iters_out) {
  const double Tg = in[18], Ts = in[19], rs = in[21], dp = in[22], P = in[23];
  const int N = o->dft_n;
  double c[MP_NSP], r[MP_NR], q[MP_NR], dc[MP_NSP], dX[MP_NSP], X[MP_NSP];
  double hist[64] = {0.0};
  double rOF = 1.0, t_rem = dt;
  long nhist = 0;
  int it = 0, status = MP_CELL_OK;
  mp_initial(t, in, c);
  for (;;) {
    mp_rates(t, o, c, Tg, Ts, rs, dp, P, r);
    for (int k = 0; k < MP_NR; ++k) q[k] = r[k];
    q[WGS] = r[WGS] * rOF;                                          /* Eq. 14 */
    mp_derivs(t, c, q, dc, dX);
    double eg, es, rg, mwg;
    mp_phase(t, c, rs, X, &eg, &es, &rg, &mwg);
    double h = mp_step_size(X, dX, dt, o);
    int last = (h >= t_rem);
    if (last) h = t_rem;
    if (o->dft_on) {
      hist[nhist % N] = r[WGS] * h;                                 /* Eq. 8 */
      if (nhist + 1 >= N) {
        double D0 = mp_dft_mag(hist, N, 0), maxhf = 0.0;
        for (int j = o->dft_hi_first; j <= N / 2; ++j) {
          double d = mp_dft_mag(hist, N, j);
          if (d > maxhf) maxhf = d;
        }
        int ring = D0 < o->tol_ring * maxhf, eq = D0 < o->tol_freq;  /* Eqs. 10-12 */
        rOF = fmax(fmin(rOF * (ring && eq ? 1.0 / o->r_fac : o->r_fac), 1.0), o->rof_min);
      } else {
        rOF = fmin(rOF * o->r_fac, 1.0);
      }
      ++nhist;
    }
    for (int i = 0; i < MP_NSP; ++i) c[i] += h * dc[i];             /* Eq. 18 */
    t_rem -= h;
    ++it;
    int finite = 1;
    for (int i = 0; i < MP_NSP; ++i) finite = finite && isfinite(c[i]);
    if (!finite) { status = MP_CELL_NONFINITE; break; }
    if (last) break;
    if (it >= o->max_iters) { status = MP_CELL_MAXITER; break; }
  }
  double eg, es, rg, mwg;
  mp_phase(t, c, rs, X, &eg, &es, &rg, &mwg);
  memcpy(out, in, sizeof(double) * MP_NIN);
  for (int i = 0; i < MP_NSP; ++i) out[i] = X[i];
  out[20] = es;
  if (rho_g_out) *rho_g_out = rg;
  *iters_out = it;
  return status;
}

/* ---------------------------------------------------- many cells, threads */
typedef struct {
  const mp_tables *t; const mp_opts *o;
  long n, start, stride;
  const double *in; double dt;
  double *out, *rho_g; int *iters; unsigned char *status;
} mp_job;

static void *mp_worker(void *arg) {
  mp_job *j = (mp_job *)arg;
  for (long c = j->start; c < j->n; c += j->stride) {
    int it = 0;
    int st = mp_solve_cell(j->t, j->o, j->in + (size_t)c * MP_NIN, j->dt,
                           j->out + (size_t)c * MP_NIN, j->rho_g + c, &it);
    j->iters[c] = it;
    j->status[c] = (unsigned char)st;
  }
  return NULL;
}

void mp_solve(const mp_opts *o, long n_cells, const double *in, double dt, double *out,
              double *rho_g, int *iters, unsigned char *status, int n_threads) {
  mp_tables t;
  mp_tables_init(&t);
  if (n_threads < 1) n_threads = 1;
  pthread_t *th = malloc(sizeof(pthread_t) * n_threads);
  mp_job *jobs = malloc(sizeof(mp_job) * n_threads);
  for (int k = 0; k < n_threads; ++k) {
    mp_job j = {&t, o, n_cells, k, n_threads, in, dt, out, rho_g, iters, status};
    jobs[k] = j;
    pthread_create(&th[k], NULL, mp_worker, &jobs[k]);
  }
  for (int k = 0; k < n_threads; ++k) pthread_join(th[k], NULL);
  free(th); free(jobs);
}

/* The tables and one evaluation of the rates, for the tests. */
void mp_get_tables(double *mw, double *nu) {
  mp_tables t;
  mp_tables_init(&t);
  memcpy(mw, t.mw, sizeof t.mw);
  memcpy(nu, t.nu, sizeof t.nu);
}
void mp_eval_rates(const mp_opts *o, const double *c, double Tg, double Ts, double rho_s,
                   double dp, double P, double *r) {
  mp_tables t;
  mp_tables_init(&t);
  mp_rates(&t, o, c, Tg, Ts, rho_s, dp, P, r);
}
void mp_initial_state(const double *in, double *c) {
  mp_tables t;
  mp_tables_init(&t);
  mp_initial(&t, in, c);
}
