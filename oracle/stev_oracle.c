/*
 * Plain FP64 CPU oracle of the STEV solver (Buchheit et al., "STEV: A
 * Stabilized Explicit Variable-Load Solver with Machine Learning Acceleration
 * for the Rapid Solution of Stiff Chemical Kinetics", arXiv:1905.09395).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file: it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can compare the CUDA path against a slow,
 * obviously correct restatement of the method.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * One cell at a time, every quantity in double precision, loops in the
 * paper's order.  What each function follows:
 *   oracle_thermo      Sec. 3, Eqs. 15-16 (cp/R, H/RT) and the standard
 *                      NASA-7 entropy form S/R (needed by dG of Eq. 30).
 *   oracle_rates       Sec. 2.2 Eqs. 6-7 (gamma stabilisation), Sec. 7.1
 *                      Eqs. 28-30 (mass action or the real orders of global
 *                      rate laws, Arrhenius, K from dG),
 *                      Eq. 14 (effective rate), Sec. 3 / Eq. 17 (the ODE
 *                      right-hand side including adiabatic temperature).
 *   oracle_step_size   Sec. 2.1 Eqs. 1-5.
 *   oracle_dft_mag     Sec. 2.3 Eq. 9 (plain O(N) sum per bin).
 *   oracle_ring_update Sec. 2.3 Eqs. 10-13.
 *   oracle_solve_cell  Sec. 2.4 (variable load: each cell stops at its own
 *                      iteration) and Eq. 18 (forward Euler).
 *
 * Readings where the paper is silent (all are parameters):
 *   - y_i, r_i are mass fractions and dY/dt (1/s);  "y << 1e-20" is y < 1e-20.
 *   - gamma acts on max(Y,0) in both mass-action products; the limiter uses raw Y.
 *   - the ringing history stores the raw (undamped) net rate times h.
 *   - order within a step: rates (with rOF_t) -> h -> history -> rOF_{t+1} -> Euler.
 *   - the last step is clamped to the remaining time with an explicit flag.
 *   - no ringing test before the N-value window is full (rOF stays 1).
 *   - DFT bins 0 and dft_hi_first..floor(N/2); Eq. 10 in multiply form;
 *     a window whose high-frequency maximum is 0 is not ringing.
 *   - rOF is kept >= rof_min so that it stays positive (Sec. 2.3: 0 < rOF <= 1).
 *   - temperature equation: adiabatic, constant pressure, ideal gas.
 *   - K uses a standard-state pressure of 1 atm (Eq. 30).
 *   - a cell whose T leaves [200, 6000] K stops with status TRANGE.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_RU 8.314462618      /* J/(mol K) */
#define ORACLE_PATM 101325.0       /* Pa, the 1 atm of Eq. 30 */
#define ORACLE_PI 3.14159265358979323846

/* Conditioning probes: the test suite also builds this file with kf scaled by
 * 1 +- 1 ulp, or K scaled by 1 +- 64 ulp (the rounding error of dG/RT, a sum
 * of terms up to ~64 in size, is of that order), to measure how far a cell's
 * result moves under a rounding-size change of its rates.  The default build
 * multiplies by exactly 1.0. */
#ifndef ORACLE_KF_SCALE
#define ORACLE_KF_SCALE 1.0
#endif
#ifndef ORACLE_K_SCALE
#define ORACLE_K_SCALE 1.0
#endif
/* Single-precision probes: round every concentration (ORACLE_ROUND32_C) or
 * every net rate of progress (ORACLE_ROUND32_Q) to the nearest float. */
#ifdef ORACLE_ROUND32_C
#define ORACLE_C(x) ((double)(float)(x))
#else
#define ORACLE_C(x) (x)
#endif
/* Single-precision noise probe (ORACLE_Q_NOISE = a): every reverse term of
 * a net rate times (1 + a xi), xi in [-1, 1) from a hash (the splitmix64
 * finaliser) of the cell's rate-evaluation count, the reaction index and
 * ORACLE_Q_NOISE_SEED, so that no equilibrium cancels exactly, as none does
 * with FP32 rates.  The uniform scalings above move an exact fixed point
 * without making it inexact, so they cannot show a cell whose stability
 * rests on exact cancellation. */
#ifdef ORACLE_Q_NOISE
#include <stdint.h>
#ifndef ORACLE_Q_NOISE_SEED
#define ORACLE_Q_NOISE_SEED 1
#endif
static _Thread_local uint64_t oracle_noise_calls;  /* reset per cell solve */
static double oracle_noise(int r) {
  uint64_t x = oracle_noise_calls * 0xD1B54A32D192ED03ULL;
  x ^= (uint64_t)(r + 1) * 0x9E3779B97F4A7C15ULL + (uint64_t)ORACLE_Q_NOISE_SEED;
  x ^= x >> 30;
  x *= 0xBF58476D1CE4E5B9ULL;
  x ^= x >> 27;
  x *= 0x94D049BB133111EBULL;
  x ^= x >> 31;
  return (double)(x >> 11) * 0x1p-52 - 1.0;
}
#define ORACLE_REV(x, r) ((x) * (1.0 + ORACLE_Q_NOISE * oracle_noise(r)))
#define ORACLE_NOISE_NEXT() (++oracle_noise_calls)
#define ORACLE_NOISE_RESET() (oracle_noise_calls = 0)
#else
#define ORACLE_REV(x, r) (x)
#define ORACLE_NOISE_NEXT() ((void)0)
#define ORACLE_NOISE_RESET() ((void)0)
#endif
#ifdef ORACLE_ROUND32_Q
#define ORACLE_Q(x) ((double)(float)(x))
#else
#define ORACLE_Q(x) (x)
#endif

typedef struct {
  int n_species, n_reactions;
  const double *mol_weight;          /* [S] kg/mol */
  const double *nasa7;               /* [S][2][7] */
  const double *t_range;             /* [S][3] low, split, high */
  const int *rxn_ptr;                /* [R+1] */
  const int *rxn_species;            /* [nnz] */
  const double *rxn_nu;              /* [nnz] */
  const double *A, *beta, *Ea;       /* [R] SI, J/mol */
  const unsigned char *reversible;   /* [R] */
  const double *rxn_order;           /* [nnz] or NULL: the entry's order in the forward
                                        (nu < 0) or reverse (nu > 0) rate; NULL = |nu| */
} oracle_mech;

typedef struct {
  double y_step_max;   /* Y_step^max, Eq. 3 */
  double delta_max;    /* delta^max, Eq. 4 */
  double alpha;        /* Eq. 7; 0 disables the stabilisation */
  int dft_n;           /* N, length of the stored history, Eq. 8 */
  int dft_hi_first;    /* n, first high-frequency bin, Eq. 10 */
  double tol_ring;     /* Tol_ring, Eq. 12 */
  double tol_freq;     /* Tol_freq, Eq. 12 (mol/m^3) */
  double r_fac;        /* r_fac, Eq. 12 */
  double rof_min;      /* lower clamp keeping rOF > 0 */
  int max_iters;       /* per-cell iteration cap */
  int dft_on;          /* 0 disables Sec. 2.3 entirely */
} oracle_opts;

enum { ORACLE_CELL_OK = 0, ORACLE_CELL_MAXITER = 1, ORACLE_CELL_NONFINITE = 2,
       ORACLE_CELL_TRANGE = 3 };

/* ---------------------------------------------------------------- thermo */
/* Eq. 15: Cp/R;  Eq. 16: H/RT;  S/R = a1 lnT + a2 T + a3 T^2/2 + a4 T^3/3
 * + a5 T^4/4 + a7.  Range: T < T_split -> low coefficients, else high. */
void oracle_thermo(const oracle_mech *m, double T, double *cpR, double *hRT, double *sR) {
  for (int i = 0; i < m->n_species; ++i) {
    int hi = (T < m->t_range[3 * i + 1]) ? 0 : 1;
    const double *a = m->nasa7 + (2 * i + hi) * 7;
    double T2 = T * T, T3 = T2 * T, T4 = T3 * T;
    cpR[i] = a[0] + a[1] * T + a[2] * T2 + a[3] * T3 + a[4] * T4;
    hRT[i] = a[0] + a[1] * T / 2.0 + a[2] * T2 / 3.0 + a[3] * T3 / 4.0 + a[4] * T4 / 5.0 + a[5] / T;
    sR[i] = a[0] * log(T) + a[1] * T + a[2] * T2 / 2.0 + a[3] * T3 / 3.0 + a[4] * T4 / 4.0 + a[6];
  }
}

/* Conditioning probe of the real-order powers (default: exactly 1.0): pow
 * results may differ between math libraries by a few ulp. */
#ifndef ORACLE_POW_SCALE
#define ORACLE_POW_SCALE 1.0
#endif

static double int_power(double x, double nu) {
  /* C^a: repeated products for the integer orders of elementary reactions,
   * pow for the real orders of global rate laws (Eqs. 28-29). */
  int n = (int)nu;
  if ((double)n != nu) return pow(x, nu) * ORACLE_POW_SCALE;
  double p = 1.0;
  for (int k = 0; k < n; ++k) p *= x;
  return p;
}

/* Order of CSR entry k in its rate law: the given order, else |nu|. */
static double entry_order(const oracle_mech *m, int k) {
  return m->rxn_order ? m->rxn_order[k] : fabs(m->rxn_nu[k]);
}

/* ----------------------------------------------------------------- rates */
/* Right-hand side of Eq. 17 for one cell.
 * Outputs (any may be NULL except dTdt):
 *   qraw[R]  net raw rate of progress per reaction (mol/m^3/s), before rOF
 *   wdot[S]  molar production rates with the effective rates of Eq. 14
 *   dYdt[S]  dY/dt (1/s);  *dTdt (K/s) */
void oracle_rates(const oracle_mech *m, const oracle_opts *o, double T, double P,
                  const double *Y, const double *rOF, double *qraw, double *wdot,
                  double *dYdt, double *dTdt) {
  const int S = m->n_species, R = m->n_reactions;
  double *cpR = malloc(sizeof(double) * S), *hRT = malloc(sizeof(double) * S);
  double *sR = malloc(sizeof(double) * S), *C = malloc(sizeof(double) * S);
  double *w = malloc(sizeof(double) * S), *q = malloc(sizeof(double) * R);

  ORACLE_NOISE_NEXT();
  /* mixture molar mass and ideal-gas density */
  double inv_wbar = 0.0;
  for (int i = 0; i < S; ++i) inv_wbar += Y[i] / m->mol_weight[i];
  double wbar = 1.0 / inv_wbar;
  double rho = P * wbar / (ORACLE_RU * T);

  oracle_thermo(m, T, cpR, hRT, sR);

  /* Eqs. 6-7: y** = y * gamma(y), gamma = y/(alpha+y), on max(Y,0) */
  for (int i = 0; i < S; ++i) {
    double y = Y[i] > 0.0 ? Y[i] : 0.0;
    double ystar2 = (o->alpha > 0.0) ? y * (y / (o->alpha + y)) : y;
    C[i] = ORACLE_C(rho * ystar2 / m->mol_weight[i]);
  }

  /* Eqs. 29-30: kf = A T^beta exp(-Ea/RT);
   * K = (1 atm / RT)^dN exp(-dG/RT), dG/RT = sum nu (H/RT - S/R); kr = kf/K */
  for (int r = 0; r < R; ++r) {
    double kf = m->A[r] * pow(T, m->beta[r]) * exp(-m->Ea[r] / (ORACLE_RU * T)) * ORACLE_KF_SCALE;
    double fwd = kf, rev = 0.0;
    for (int k = m->rxn_ptr[r]; k < m->rxn_ptr[r + 1]; ++k) {
      double nu = m->rxn_nu[k];
      if (nu < 0.0) fwd *= int_power(C[m->rxn_species[k]], entry_order(m, k));
    }
    if (m->reversible[r]) {
      double dG = 0.0, dN = 0.0;
      for (int k = m->rxn_ptr[r]; k < m->rxn_ptr[r + 1]; ++k) {
        int s = m->rxn_species[k];
        dG += m->rxn_nu[k] * (hRT[s] - sR[s]);
        dN += m->rxn_nu[k];
      }
      double K = pow(ORACLE_PATM / (ORACLE_RU * T), dN) * exp(-dG) * ORACLE_K_SCALE;
      double kr = kf / K;
      rev = kr;
      for (int k = m->rxn_ptr[r]; k < m->rxn_ptr[r + 1]; ++k) {
        double nu = m->rxn_nu[k];
        if (nu > 0.0) rev *= int_power(C[m->rxn_species[k]], entry_order(m, k));
      }
    }
    q[r] = ORACLE_Q(fwd - ORACLE_REV(rev, r));
  }

  /* Eq. 14 effective rates, production rates in ascending reaction order */
  for (int i = 0; i < S; ++i) w[i] = 0.0;
  for (int r = 0; r < R; ++r) {
    double qe = m->reversible[r] ? q[r] * rOF[r] : q[r];
    for (int k = m->rxn_ptr[r]; k < m->rxn_ptr[r + 1]; ++k)
      w[m->rxn_species[k]] += m->rxn_nu[k] * qe;
  }

  /* species and adiabatic constant-pressure temperature equations */
  double cp = 0.0, hw = 0.0;
  for (int i = 0; i < S; ++i) cp += Y[i] * cpR[i] / m->mol_weight[i];
  cp *= ORACLE_RU;                                   /* J/(kg K) */
  for (int i = 0; i < S; ++i) hw += hRT[i] * w[i];
  *dTdt = -(ORACLE_RU * T * hw) / (rho * cp);
  for (int i = 0; i < S; ++i) {
    if (dYdt) dYdt[i] = m->mol_weight[i] * w[i] / rho;
    if (wdot) wdot[i] = w[i];
  }
  if (qraw)
    for (int r = 0; r < R; ++r) qraw[r] = q[r];
  free(cpR); free(hRT); free(sR); free(C); free(w); free(q);
}

/* ---------------------------------------------------------- step size */
/* Eqs. 1-5: r*_i = max(-r_i, 1e-30);  y*_i = 1 if y_i < 1e-20 else 0.9 y_i;
 * t* = min_i min(Y_step^max, y*_i)/r*_i;  dt_max = t_f delta^max;
 * h = min(t*, dt_max). */
double oracle_step_size(int S, const double *Y, const double *dYdt, double t_f,
                        double y_step_max, double delta_max) {
  double tstar = INFINITY;
  for (int i = 0; i < S; ++i) {
    double rstar = fmax(-dYdt[i], 1.0e-30);
    double ystar = (Y[i] < 1.0e-20) ? 1.0 : 0.9 * Y[i];
    double cand = fmin(y_step_max, ystar) / rstar;
    if (cand < tstar) tstar = cand;
  }
  double dtmax = t_f * delta_max;
  return fmin(tstar, dtmax);
}

/* ------------------------------------------------------------------ DFT */
/* Eq. 9: magnitude of bin j of the N-point DFT of x (any rotation of the
 * window gives the same magnitudes). */
double oracle_dft_mag(const double *x, int N, int j) {
  double re = 0.0, im = 0.0;
  for (int k = 0; k < N; ++k) {
    double ang = -2.0 * ORACLE_PI * (double)j * (double)k / (double)N;
    re += x[k] * cos(ang);
    im += x[k] * sin(ang);
  }
  if (j == 0) return fabs(re);
  return hypot(re, im);
}

/* Eqs. 10-13 for one reversible reaction whose window x[N] is full:
 * ringing  <=> D0 < Tol_ring * max_{n<=j<=N/2} D_j   (f_ring < Tol_ring)
 * equilib. <=> D0 < Tol_freq
 * rOF_{t+1} = min(rOF_t * rOF*, 1), rOF* = 1/r_fac if both, else r_fac. */
double oracle_ring_update(const double *x, int N, int hi_first, double rOF,
                          double tol_ring, double tol_freq, double r_fac, double rof_min) {
  double D0 = oracle_dft_mag(x, N, 0);
  double maxhf = 0.0;
  for (int j = hi_first; j <= N / 2; ++j) {
    double d = oracle_dft_mag(x, N, j);
    if (d > maxhf) maxhf = d;
  }
  int ringing = (D0 < tol_ring * maxhf);
  int at_eq = (D0 < tol_freq);
  double rstar = (ringing && at_eq) ? 1.0 / r_fac : r_fac;
  double next = fmin(rOF * rstar, 1.0);
  return fmax(next, rof_min);
}

/* ------------------------------------------------------------ one cell */
/* Integrates one cell from (T0, P, Y0) over t_f = dt with the STEV scheme.
 * If trace_cap > 0, per-step records are written before each Euler update:
 * trace_h[it], trace_T[it], trace_Y[it][S] (state the step starts from). */
int oracle_solve_cell_trace(const oracle_mech *m, const oracle_opts *o, double T0, double P,
                            const double *Y0, double dt, double *T_out, double *Y_out,
                            int *iters_out, int trace_cap, double *trace_h, double *trace_T,
                            double *trace_Y) {
  const int S = m->n_species, R = m->n_reactions, N = o->dft_n;
  double *Y = malloc(sizeof(double) * S), *dYdt = malloc(sizeof(double) * S);
  double *rOF = malloc(sizeof(double) * R), *qraw = malloc(sizeof(double) * R);
  double *hist = calloc((size_t)R * (size_t)(N > 0 ? N : 1), sizeof(double));
  for (int i = 0; i < S; ++i) Y[i] = Y0[i];
  for (int r = 0; r < R; ++r) rOF[r] = 1.0;                 /* Eq. 11 */
  double T = T0, t_rem = dt, dTdt = 0.0;
  long nhist = 0;
  ORACLE_NOISE_RESET();
  int it = 0, status = ORACLE_CELL_OK;
  for (;;) {
    oracle_rates(m, o, T, P, Y, rOF, qraw, NULL, dYdt, &dTdt);
    double h = oracle_step_size(S, Y, dYdt, dt, o->y_step_max, o->delta_max);
    int last = (h >= t_rem);
    if (last) h = t_rem;
    if (trace_cap > 0 && it < trace_cap) {
      trace_h[it] = h;
      trace_T[it] = T;
      for (int i = 0; i < S; ++i) trace_Y[(size_t)it * S + i] = Y[i];
    }
    if (o->dft_on) {
      for (int r = 0; r < R; ++r) {
        if (!m->reversible[r]) continue;
        double *x = hist + (size_t)r * N;
        x[nhist % N] = qraw[r] * h;                          /* Eq. 8 */
        if (nhist + 1 >= N)
          rOF[r] = oracle_ring_update(x, N, o->dft_hi_first, rOF[r], o->tol_ring,
                                      o->tol_freq, o->r_fac, o->rof_min);
        else
          rOF[r] = fmin(rOF[r] * o->r_fac, 1.0);
      }
      ++nhist;
    }
    for (int i = 0; i < S; ++i) Y[i] += h * dYdt[i];       /* Eq. 18 */
    T += h * dTdt;
    t_rem -= h;
    ++it;
    int finite = isfinite(T);
    for (int i = 0; i < S; ++i) finite = finite && isfinite(Y[i]);
    if (!finite) { status = ORACLE_CELL_NONFINITE; break; }
    if (T < 200.0 || T > 6000.0) { status = ORACLE_CELL_TRANGE; break; }
    if (last) break;
    if (it >= o->max_iters) { status = ORACLE_CELL_MAXITER; break; }
  }
  *T_out = T;
  for (int i = 0; i < S; ++i) Y_out[i] = Y[i];
  *iters_out = it;
  free(Y); free(dYdt); free(rOF); free(qraw); free(hist);
  return status;
}

int oracle_solve_cell(const oracle_mech *m, const oracle_opts *o, double T0, double P,
                      const double *Y0, double dt, double *T_out, double *Y_out, int *iters_out) {
  return oracle_solve_cell_trace(m, o, T0, P, Y0, dt, T_out, Y_out, iters_out, 0, NULL, NULL, NULL);
}

/* ---------------------------------------------------- many cells, threads */
typedef struct {
  const oracle_mech *m; const oracle_opts *o;
  long n, start, stride;
  const double *T, *P, *Y; double dt;
  double *T_out, *Y_out; int *iters; unsigned char *status;
} oracle_job;

static void *oracle_worker(void *arg) {
  oracle_job *j = (oracle_job *)arg;
  const int S = j->m->n_species;
  for (long c = j->start; c < j->n; c += j->stride) {
    int it = 0;
    int st = oracle_solve_cell(j->m, j->o, j->T[c], j->P[c], j->Y + (size_t)c * S, j->dt,
                               j->T_out + c, j->Y_out + (size_t)c * S, &it);
    j->iters[c] = it;
    j->status[c] = (unsigned char)st;
  }
  return NULL;
}

/* Cells are independent (Sec. 2.4); threads take every n_threads-th cell. */
void oracle_solve(const oracle_mech *m, const oracle_opts *o, long n_cells, const double *T,
                  const double *P, const double *Y, double dt, double *T_out, double *Y_out,
                  int *iters, unsigned char *status, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  pthread_t *th = malloc(sizeof(pthread_t) * n_threads);
  oracle_job *jobs = malloc(sizeof(oracle_job) * n_threads);
  for (int t = 0; t < n_threads; ++t) {
    oracle_job j = {m, o, n_cells, t, n_threads, T, P, Y, dt, T_out, Y_out, iters, status};
    jobs[t] = j;
    pthread_create(&th[t], NULL, oracle_worker, &jobs[t]);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  free(th); free(jobs);
}
