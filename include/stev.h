/*
 * stev.h - C ABI of the B300 STEV stiff-chemistry integrator.
 *
 * STEV (Buchheit et al., arXiv:1905.09395) integrates the chemical source
 * terms of many independent CFD cells over one fluid time step t_f with
 * forward Euler (Eq. 18), each cell on its own step size (Sec. 2.1, Eqs. 1-5),
 * small-species damping of the rate laws (Sec. 2.2, Eqs. 6-7), a DFT ringing
 * damper on reversible reactions (Sec. 2.3, Eqs. 8-14), and variable loading:
 * a cell leaves the workload the iteration it reaches t_f (Sec. 2.4).
 *
 * Conventions for every entry point below:
 *   - SI units: Pa, K, kg/mol, J/mol, mol/m^3, s.  Mass fractions Y.
 *   - Cell arrays passed to stev_solve / stev_solve_soa are DEVICE pointers
 *     owned by the caller; stev_solve_host takes HOST pointers.  Mechanism
 *     tables passed to stev_mechanism_create are HOST pointers, copied.
 *   - Calls are asynchronous on `cuda_stream` (NULL = legacy default stream)
 *     unless stated otherwise; completion is observed through the stream.
 *   - A mechanism owns its device tables and a work counter; at most one
 *     solve may be in flight per mechanism at a time.
 *   - Errors are returned as stev_status; stev_last_error() gives a message
 *     (thread-local).  Per-cell outcomes go to the cell_status array.
 */
#ifndef STEV_H
#define STEV_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stev_mechanism stev_mechanism; /* opaque */

typedef enum {
  STEV_OK = 0,
  STEV_EINVAL = 1,       /* bad argument or mechanism table */
  STEV_ENOMEM = 2,       /* device or host allocation failed */
  STEV_ECUDA = 3,        /* a CUDA call failed (message has the CUDA error) */
  STEV_ETIMEOUT = 4,     /* a bounded wait gave up */
  STEV_EUNBALANCED = 5,  /* a reaction does not conserve mass */
  STEV_EINCOMPLETE = 6   /* the solver did not finish every cell */
} stev_status;

/* per-cell outcome written to cell_status[] */
enum {
  STEV_CELL_OK = 0,         /* reached t_f */
  STEV_CELL_MAXITER = 1,    /* stopped at options.max_iters iterations */
  STEV_CELL_NONFINITE = 2,  /* Y or T became NaN/Inf; state at that step */
  STEV_CELL_TRANGE = 3      /* T left [200, 6000] K; state at that step */
};

/* options.precision.  FP64: every quantity in IEEE double (the oracle's
 * arithmetic).  MIXED: rates, limiter and ringing test in FP32 (base-2 MUFU
 * exponentials); Y, T, ln T, 1/T and the species' Gibbs terms of Eq. 30 as
 * float pairs (about 48 significant bits) on the FP32 pipe; h and t_rem in
 * double.  Results of MIXED meet 1e-4 in Y and 0.5 K against FP64 on cells
 * that are well-conditioned at single-precision rounding. */
enum { STEV_FP64 = 0, STEV_MIXED = 1 };
/* options.thermo: where the mixed path takes species properties from.
 * POLY: NASA-7 polynomials.  MLP: cp/R from the thermo network, H/RT and G/RT
 * from the polynomials.  MLP_CPH: cp/R and H/RT from the network.  G/RT (the
 * equilibrium constants of Eq. 30) always comes from the polynomials, at
 * FP64-grade precision. */
enum { STEV_THERMO_POLY = 0, STEV_THERMO_MLP = 1, STEV_THERMO_MLP_CPH = 2 };

/* Solver parameters.  The paper names them but gives values for few; the
 * defaults (stev_default_options) are the readings listed beside each. */
typedef struct {
  double y_step_max;  /* Y_step^max, Eq. 3: max mass-fraction consumption per step (1e-3) */
  double delta_max;   /* delta^max, Eq. 4: h <= t_f * delta_max (0.01) */
  double alpha;       /* Eq. 7 species limit factor; 0 disables (1e-5) */
  int dft_n;          /* N, stored history length per reversible reaction, Sec. 2.3 (13) */
  int dft_hi_first;   /* n, first high-frequency bin of Eq. 10 (4) */
  double tol_ring;    /* Tol_ring, Eq. 12 (0.5) */
  double tol_freq;    /* Tol_freq, Eq. 12, mol/m^3 (1e-6) */
  double r_fac;       /* r_fac, Eq. 12, > 1 (2) */
  double rof_min;     /* lower clamp keeping rOF > 0 (1e-30) */
  int max_iters;      /* per-cell iteration cap (200000) */
  int precision;      /* STEV_FP64 or STEV_MIXED */
  int thermo;         /* STEV_THERMO_POLY, _MLP or _MLP_CPH (POLY) */
  int dft_on;         /* 0 disables the Sec. 2.3 damper (1) */
  int lanes_per_cell; /* lanes that share one cell: 8, 16 or 32; 0 = chosen per
                         mechanism and precision (0) */
  int specialize;     /* mixed precision: 1 compiles the solver kernel for this
                         mechanism at run time (NVRTC; its sizes and rate-law
                         kind as constants), about a second at creation or
                         when the options change; 0 uses the generic kernel
                         (0).  Needs the csrc directory beside the library and
                         CUDA's headers. */
} stev_options;

/* Fills *opt with the defaults above.  Never fails for a non-NULL opt. */
void stev_default_options(stev_options *opt);

/* Builds a mechanism from host tables and stages them on the current device.
 *   n_species   S, 1..64;  n_reactions R, 1..512.
 *   mol_weight  [S] kg/mol, > 0.
 *   nasa7       [S][2][7] NASA-7 coefficients, low range then high range
 *               (Sec. 3, Eqs. 15-16; a6 enthalpy and a7 entropy constants).
 *   t_range     [S][3] T_low, T_split, T_high: T < T_split uses the low block.
 *   rxn_ptr     [R+1] CSR row pointers into rxn_species / rxn_nu.
 *   rxn_species [nnz] species index of each entry.
 *   rxn_nu      [nnz] stoichiometric coefficient: < 0 reactant, > 0 product.
 *               Reactions must be elementary: integer orders with at most two
 *               molecules on each side (Sec. 4), each species at most once
 *               (stev_mechanism_create_orders takes global rate laws).
 *   A, beta, Ea [R] Arrhenius k = A T^beta exp(-Ea/(R T)) (Eq. 29 form), SI.
 *   reversible  [R] nonzero: reverse rate kf/K with K from Eq. 30.
 *   opt         NULL for the defaults.
 * Returns STEV_EINVAL for sizes out of range, non-finite or negative A,
 * non-positive molar masses, bad indices or orders; STEV_EUNBALANCED when
 * |sum nu W| > 1e-12 sum |nu W| for a reaction; STEV_ECUDA / STEV_ENOMEM on
 * device failures.  On success *out owns the mechanism (free with
 * stev_destroy).  Synchronous. */
stev_status stev_mechanism_create(int n_species, int n_reactions, const double *mol_weight,
                                  const double *nasa7, const double *t_range,
                                  const int *rxn_ptr, const int *rxn_species,
                                  const double *rxn_nu, const double *A, const double *beta,
                                  const double *Ea, const unsigned char *reversible,
                                  const stev_options *opt, stev_mechanism **out);

/* As stev_mechanism_create, for global rate laws such as the paper's BFER
 * methane mechanism (Sec. 7.1, Eqs. 26-29): stoichiometric coefficients may be
 * any nonzero real (e.g. 1.5 O2), and rxn_order [nnz] (nullable) gives each
 * entry's order in its rate law, > 0: the forward rate kf prod C^order over
 * the reactant entries (nu < 0), the reverse rate kf/K prod C^order over the
 * product entries (nu > 0).  NULL orders mean |nu| (mass action).  A reaction
 * then has at most two distinct reactant and two distinct product species;
 * K (Eq. 30) uses dN = sum nu.  Mechanisms whose every |nu| is 1 or 2 with
 * orders |nu| take the same path as stev_mechanism_create.  Errors as
 * stev_mechanism_create, plus STEV_EINVAL for an order <= 0. */
stev_status stev_mechanism_create_orders(int n_species, int n_reactions, const double *mol_weight,
                                         const double *nasa7, const double *t_range,
                                         const int *rxn_ptr, const int *rxn_species,
                                         const double *rxn_nu, const double *rxn_order,
                                         const double *A, const double *beta, const double *Ea,
                                         const unsigned char *reversible, const stev_options *opt,
                                         stev_mechanism **out);

/* Replaces the solver options of a mechanism (validated as in create). */
stev_status stev_mechanism_set_options(stev_mechanism *mech, const stev_options *opt);

/* Reads back the options in force. */
stev_status stev_mechanism_get_options(const stev_mechanism *mech, stev_options *opt);

/* Integrates n_cells independent cells over t_f = dt_cfd (Secs. 2.1-2.4).
 *   T, P        [n_cells] initial temperature (K) and pressure (Pa), device.
 *   Y           [n_cells][S] initial mass fractions (cell-major), device.
 *   T_out, Y_out final state, same layouts; Y_out == Y and T_out == T are allowed.
 *   iters       [n_cells] int32 iterations taken by each cell.
 *   cell_status [n_cells] STEV_CELL_* per cell.
 * n_cells == 0 is a no-op.  Returns STEV_EINVAL for NULL arrays with
 * n_cells > 0, dt_cfd <= 0 or non-finite.  Asynchronous on cuda_stream. */
stev_status stev_solve(stev_mechanism *mech, long n_cells, const double *T, const double *P,
                       const double *Y, double dt_cfd, double *T_out, double *Y_out,
                       int *iters, unsigned char *cell_status, void *cuda_stream);

/* As stev_solve, but Y and Y_out are species-major [S][n_cells] (structure of
 * arrays), for callers that keep their state that way.  The solver stages a
 * whole cell per lane group, so its loads here are strided by n_cells; the
 * cell-major layout of stev_solve is the coalesced one. */
stev_status stev_solve_soa(stev_mechanism *mech, long n_cells, const double *T, const double *P,
                           const double *Y_soa, double dt_cfd, double *T_out, double *Y_out_soa,
                           int *iters, unsigned char *cell_status, void *cuda_stream);

/* Integrates n_batches independent batches of cells in ONE persistent launch
 * (Sec. 2.4's variable load across all of them): batch b has n_cells[b]
 * cells, its own fluid time step dt[b] and its own DEVICE arrays T[b], P[b],
 * Y[b] ([n][S]), T_out[b], Y_out[b], iters[b], cell_status[b]; the pointer
 * arrays and n_cells, dt are HOST arrays.  Batches of 0 cells are skipped.
 * Each cell's result equals the one stev_solve gives it.  The batch table is
 * copied to a device buffer the mechanism owns (grown when n_batches grows).
 * Asynchronous on cuda_stream. */
stev_status stev_solve_batched(stev_mechanism *mech, int n_batches, const long *n_cells,
                               const double *const *T, const double *const *P,
                               const double *const *Y, const double *dt, double *const *T_out,
                               double *const *Y_out, int *const *iters,
                               unsigned char *const *cell_status, void *cuda_stream);

/* As stev_solve with HOST arrays: copies the inputs to the device, solves and
 * copies the results back on cuda_stream, then waits for the stream.
 * Device buffers are owned by the mechanism and reused across calls. */
stev_status stev_solve_host(stev_mechanism *mech, long n_cells, const double *T, const double *P,
                            const double *Y, double dt_cfd, double *T_out, double *Y_out,
                            int *iters, unsigned char *cell_status, void *cuda_stream);

/* As stev_solve_host, but allocates nothing.  For callers that may not allocate
 * device memory when they solve: a CFD code whose device memory belongs to its
 * own pool allocator and budget, a real-time or callback context where
 * cudaMalloc's implicit synchronisation is not acceptable, or a process that
 * must not grow its device footprint after start-up.  (The paper has no
 * counterpart; it is a property of this library's interface.)
 *   Staging goes through one fixed 16 MiB device array in the library, shared
 *   by every call and held by every GPU that loads the library until exit.
 *   A call needs  256 + align(8n)*2 + align(8nS) + align(8n) + align(8nS)
 *   + align(4n) + align(n)  bytes (align = round up to 256); larger n_cells
 *   are rejected with STEV_EINVAL and a message giving the largest n that
 *   fits (about 31,000 cells at S = 32).
 *   The first call on a device looks up the array's device address (a one-off
 *   set-up); make that first call before any stream capture.  The address is
 *   kept for the life of the process: like every mechanism's device buffers,
 *   it is invalid after cudaDeviceReset, so do not call this entry point on a
 *   device after resetting it.
 *   The array keeps the previous call's contents; the work counter is cleared
 *   on every call.  Calls whose GPU work overlaps (different streams, host
 *   threads) race on the array: serialise them.
 *   No cudaMalloc, cudaFree or other allocating routine is called.  Blocks
 *   until the results are in the host arrays. */
stev_status stev_solve_host_noalloc(stev_mechanism *mech, long n_cells, const double *T,
                                    const double *P, const double *Y, double dt_cfd,
                                    double *T_out, double *Y_out, int *iters,
                                    unsigned char *cell_status, void *cuda_stream);

/* ---- multiphase coal gasification cells (Sec. 7.2: reactions 31-41, rate laws
 * Eqs. 42-56, Table 2) integrated by STEV (Eqs. 1-5, 8-14, 18), FP64.
 *   cells      [n_cells][24] DEVICE records: gas mass fractions of O2 CO CO2
 *              CH4 H2 H2O H2S C3H6 HCN C2H4 C2H6 Tar SO3 N2 (14), solid mass
 *              fractions of CV (volatile matter) CC (fixed carbon) CM
 *              (moisture) CA (ash) (4), T_g, T_s (K), eps_s (solid volume
 *              fraction), rho_s (solid material density, kg/m^3), d_p
 *              (particle diameter, m), P (Pa).  With eps_g = 1 - eps_s and
 *              rho_g (the ideal gas law at P, T_g and the gas's molar mass)
 *              these are the paper's 26 variables per cell.
 *   dt_cfd     the fluid step t_f (s).
 *   opt        NULL = defaults; y_step_max, delta_max, alpha, dft_n,
 *              dft_hi_first, tol_ring, tol_freq, r_fac, rof_min, max_iters and
 *              dft_on are used (precision, thermo, lanes and specialize are
 *              not: the path is FP64).
 *   cells_out  [n_cells][24] DEVICE: the records after t_f: new mass
 *              fractions and eps_s; T_g, T_s, rho_s, d_p, P as given (the
 *              phase temperatures are held over the chemistry step: the
 *              paper prints no phase energy equations).  May equal cells.
 *   rho_g      [n_cells] DEVICE (nullable): the final gas density.
 *   iters, cell_status [n_cells] DEVICE, as stev_solve.
 * The species' partial densities are integrated (mass is conserved by the
 * reactions, read as molar with Tar's and CV's molecular weights balancing
 * Eqs. 37 and 31, rates of progress in kmol/m^3/s); eps_s follows the solid's
 * mass at constant rho_s.  Asynchronous on cuda_stream. */
stev_status stev_mp_solve(long n_cells, const double *cells, double dt_cfd,
                          const stev_options *opt, double *cells_out, double *rho_g, int *iters,
                          unsigned char *cell_status, void *cuda_stream);

/* ---- thermo network (Sec. 3: a small neural network of temperature stands in
 * for the NASA-7 species properties; Figs. 2-3).  The library's network is
 * t = (T - 1650)/1350, a1 = tanh(W1 t + b1), a2 = tanh(W2 a1 + b2) (64 each),
 * y = W3 a2 + b3 (3S standardised outputs: cp/R of every species, then H/R
 * in kelvin (H/RT times T, smooth over the range), then S/R; value =
 * y * std + mean).  Parameters are one flat float array:
 * W1[64], b1[64], W2[64][64], b2[64], W3[3S][64], b3[3S] (rows = outputs). */

/* Number of network parameters of this mechanism (64*64 + 67*3S + 192). */
long stev_mlp_num_params(const stev_mechanism *mech);

/* Trains the network on the GPU with the library's own kernels: targets are
 * the NASA-7 polynomials at the given HOST temperatures (FP64, stored FP32,
 * standardised per output), FP32 forward/backward, Adam (beta 0.9/0.999)
 * over minibatches of `batch` samples in sample order for `epochs` epochs,
 * the step size decaying from lr to lr/100 along a cosine, weights
 * initialised Xavier-uniform from splitmix64(seed).  Gradients are summed
 * over 64-sample tiles in a fixed order, so the same inputs train the same
 * network bit for bit.  loss_per_epoch (host, nullable) receives each epoch's
 * mean squared error in standardised units.  Afterwards inference uses BF16
 * copies of W2, W3 (BF16 tensor-core MMAs with FP32 accumulation, inside the
 * solver step for the cells of each warp).  Synchronous. */
stev_status stev_mlp_train(stev_mechanism *mech, const double *T_samples, long n_samples,
                           int epochs, int batch, float lr, unsigned long long seed,
                           float *loss_per_epoch);

/* Trains the network with Levenberg-Marquardt, the optimizer Sec. 3 uses:
 * each iteration takes the next `batch` samples (consecutive windows of the
 * HOST sample array), forms the Jacobian J of the batch's standardised
 * outputs with respect to every parameter (FP32, stored transposed) and the
 * residuals r, then J^T J (stev_gram_tf32: TF32 tensor-core products, FP32
 * accumulation) and J^T r (FP32), and solves
 * (J^T J + lambda diag(J^T J) + 1e-12 I) d = J^T r by Jacobi-preconditioned
 * conjugate gradients (stev_damped_cg: until the residual has fallen by 1e-3
 * or 400 steps, an inexact Levenberg-Marquardt step); every step runs in the
 * library's own kernels.  The step p - d is kept if it lowers the batch's mean
 * squared error (then lambda /= 3), else lambda *= 2 and the solve is
 * repeated, at most 8 times.  init: 0 =
 * Xavier-uniform weights from splitmix64(seed) and fresh output statistics;
 * 1 = continue from the current network and its statistics (e.g. after
 * stev_mlp_train).  lambda0 > 0: the starting damping.  loss_per_iter
 * (HOST, nullable) receives each iteration's batch loss after its step, in
 * standardised units.  The Jacobian takes batch * 3S * n_params * 4 bytes of
 * device memory (at most 8 GB).  Synchronous. */
stev_status stev_mlp_train_lm(stev_mechanism *mech, const double *T_samples, long n_samples,
                              int iterations, int batch, double lambda0, int init,
                              unsigned long long seed, float *loss_per_iter);

/* The Jacobian the Levenberg-Marquardt trainer forms: d(standardised output o
 * at sample s) / d(parameter p) for parameters `params` (HOST) at n <= 4096
 * HOST temperatures; J (HOST) receives [n * 3S][n_params], row s * 3S + o.
 * Synchronous. */
stev_status stev_mlp_jacobian(stev_mechanism *mech, const float *params, const double *T,
                              long n, float *J);

/* ---- the Levenberg-Marquardt trainer's linear algebra (Sec. 3), on the
 * library's own kernels.  DEVICE pointers; synchronous (the stream is
 * synchronised before returning). */

/* G = X X^T for X [n][ldx] row-major FP32 (the first k values of each row
 * used): n x n, full (both triangles), row stride ldg >= n.  The products are
 * taken on the tensor cores in TF32 (inputs rounded to 10-bit mantissas, as
 * the hardware's TF32 mode does) and accumulated in FP32 (the Gauss-Newton
 * matrix of the trainer; a 128 x 256 tile per CTA, operands staged by TMA).
 * X must be 16-byte aligned, ldx >= k a multiple of 4.  The call is
 * synchronous (it reads back the kernel's error flag, allocated from the
 * stream's memory pool).  STEV_EINVAL on bad sizes; STEV_ETIMEOUT if a wait of
 * the kernel's pipeline ran out (never expected; the kernel then stops and G
 * is incomplete). */
stev_status stev_gram_tf32(long n, long k, const float *X, long ldx, float *G, long ldg,
                           void *cuda_stream);

/* Solves (A + lambda diag(A) + eps I) x = b for symmetric A [n][lda] (FP32,
 * row-major, both triangles) by conjugate gradients with the Jacobi
 * preconditioner diag(A)(1 + lambda) + eps: from x = 0 until the residual
 * norm has fallen by rtol, or max_iters steps, or a direction of non-positive
 * curvature (then the current x is returned).  *iters (HOST, nullable)
 * receives the steps taken.  Dot products are reduced in FP64 in a fixed
 * order (the same inputs give the same x).  Work arrays are allocated and
 * freed inside. */
stev_status stev_damped_cg(long n, const float *A, long lda, const float *b, double lambda,
                           double eps, float *x, int max_iters, double rtol, int *iters,
                           void *cuda_stream);

/* Sets / reads the network parameters (HOST arrays) and the per-output mean and
 * standard deviation ([3S] each) used to undo the standardisation. */
stev_status stev_mlp_set_params(stev_mechanism *mech, const float *params, long n_params,
                                const float *mean, const float *stdv);
stev_status stev_mlp_get_params(const stev_mechanism *mech, float *params, long n_params,
                                float *mean, float *stdv);

/* Mean-squared error of the network with parameters `params` on n samples
 * (HOST: T [n], standardised targets [n][3S]) and its gradient (HOST,
 * [n_params]), computed by the training kernel (FP32).  Synchronous. */
stev_status stev_mlp_loss_grad(stev_mechanism *mech, const float *params, const double *T,
                               const float *target, long n, float *grad, double *loss);

/* Evaluates the trained network (BF16 tensor-core MMAs, FP32 accumulation) at
 * n DEVICE temperatures; props (DEVICE) receives [n][3S] values (cp/R, H/RT,
 * S/R) in the order above.  Asynchronous on cuda_stream. */
stev_status stev_mlp_eval(stev_mechanism *mech, const double *T, long n, float *props,
                          void *cuda_stream);

/* ---- serving: continuous batching of solve requests.
 * Requests (independent cell batches, each with its own t_f, from concurrent
 * CFD steps) arrive over time.  A server keeps one persistent kernel per
 * mechanism resident on its own share of the SMs and feeds it requests as
 * they are admitted: a cell slot freed by a finished cell takes the next
 * cell of the oldest unfinished request (the variable loading of Sec. 2.4,
 * across requests).  Each cell's result is the one stev_solve gives it.
 *
 * Admission is first-come first-served by device memory: a request needs
 *   2*align(8n) + align(8nS) + align(4n) + align(n)   bytes (align = 256)
 * of the server's arena (allocated once, at creation, to mem_budget bytes;
 * nothing is allocated while serving), and one of queue_len slots of its
 * mechanism.  A worker thread in the library makes every CUDA call of the
 * server: input copies, launches, completion polling (a host-mapped mailbox
 * written by each request's last cell) and result copies, on streams of its
 * own.  While a server holds a mechanism, do not change the mechanism's
 * options or network, and do not destroy it. */
typedef struct stev_server stev_server; /* opaque */

typedef struct {
  long long id;    /* from stev_server_submit */
  int mechanism;   /* index into the server's mechanism list */
  int status;      /* STEV_OK: results are in the host arrays;
                      STEV_EINCOMPLETE: cancelled by stev_server_destroy */
  long n_cells;
  long cells_done; /* cells solved: n_cells when finished; for a cancelled
                      request, those whose results were written on the device
                      before the kernels stopped (not copied back) */
  double t_submit; /* seconds on the server clock (stev_server_clock): submitted, */
  double t_admit;  /*   admitted (arena range reserved, copies queued), */
  double t_done;   /*   results copied to the host arrays */
} stev_request_info;

typedef struct {
  long long submitted, admitted, completed, cancelled;
  long long cells_completed;
  size_t resident_bytes;       /* arena bytes held by admitted, unfinished requests */
  size_t peak_resident_bytes;
  size_t budget_bytes;
  long long kernel_launches;   /* persistent-kernel (re)launches */
} stev_server_stats;

/* Creates a server for n_mechs mechanisms (all on the current device).
 * sm_share[i] (HOST, nullable = even split) is the number of SMs whose single
 * CTA runs mechanism i's kernel; the shares may add up to at most the SM
 * count.  mem_budget: bytes of the device arena.  queue_len: request slots per
 * mechanism (0 = 1024).  Errors: STEV_EINVAL (bad arguments, a mechanism with
 * thermo = MLP and no trained network), STEV_ENOMEM (the arena), STEV_ECUDA. */
stev_status stev_server_create(stev_mechanism *const *mechs, int n_mechs, const int *sm_share,
                               size_t mem_budget, int queue_len, stev_server **out);

/* Queues a request of n_cells cells of mechanism `mech` (HOST arrays, layouts
 * as for stev_solve; pinned memory makes the copies asynchronous).  The arrays
 * must stay valid and untouched until the request is reported by
 * stev_server_poll.  Returns at once; *request_id (nullable) gets the id.
 * Errors: STEV_EINVAL for bad arguments or a request larger than the whole
 * budget; the error of a failed server. */
stev_status stev_server_submit(stev_server *srv, int mech, long n_cells, double dt_cfd,
                               const double *T, const double *P, const double *Y,
                               double *T_out, double *Y_out, int *iters,
                               unsigned char *cell_status, long long *request_id);

/* Moves up to max_done finished requests into done[] (HOST), oldest first,
 * waiting up to timeout_s seconds for the first one if none is ready.
 * *n_done gets the count.  Returns the server's error if its worker failed. */
stev_status stev_server_poll(stev_server *srv, stev_request_info *done, int max_done,
                             int *n_done, double timeout_s);

/* Copies the server's counters into *stats. */
stev_status stev_server_get_stats(stev_server *srv, stev_server_stats *stats);

/* Seconds since the server was created (the clock of stev_request_info). */
double stev_server_clock(const stev_server *srv);

/* Stops the server: no more submissions; kernels finish the cells they hold,
 * claim no more and leave.  Requests whose cells all finished get their
 * results; the rest are reported STEV_EINCOMPLETE with their cells_done.
 * Every report stays readable with stev_server_poll until destroy.  Waits at
 * most timeout_s (<= 0: 30 s) for the kernels to leave; STEV_ETIMEOUT if they
 * did not.  Calling it again returns the first call's outcome. */
stev_status stev_server_stop(stev_server *srv, double timeout_s);

/* Stops the server if needed (as stev_server_stop) and frees it; unread
 * reports are lost.  If the kernels did not leave in time (STEV_ETIMEOUT) the
 * device buffers are not freed.  NULL is a no-op. */
stev_status stev_server_destroy(stev_server *srv, double timeout_s);

/* Cell-steps of this mechanism's network solves that took the polynomials
 * because the network's answer did not arrive in time.  Each warp now
 * evaluates the network for its own cells inside the step (no wait), so this
 * stays 0; kept for callers of earlier versions.  Synchronous; -1 if the
 * device read fails. */
long long stev_mlp_stalls(const stev_mechanism *mech);

/* Number of resident solver slots (cells in flight) of the persistent kernel
 * on the current device for this mechanism and its options. */
long stev_resident_slots(const stev_mechanism *mech);

/* 1 if this mechanism's solves run a kernel specialised for it
 * (options.specialize with mixed precision), 0 if the generic kernel. */
int stev_is_specialized(const stev_mechanism *mech);

/* Compiles (NVRTC, for sm_103a) the mixed-precision kernel specialised for
 * these sizes without loading it: no GPU is needed.  general: real orders or
 * stoichiometry; lanes_per_cell: 8, 16 or 32 (network: 1 for the kernel with
 * the thermo network, any lane group); dft_n:
 * 13 selects the unrolled window, any other value the run-time one.  NVRTC's
 * log is copied into log[log_len] (may be NULL).  STEV_EINVAL for sizes out
 * of range, STEV_ECUDA if the compilation fails (its log in
 * stev_last_error()). */
stev_status stev_spec_compile_check(int n_species, int n_reactions, int n_reversible,
                                    int general, int lanes_per_cell, int dft_n, int network,
                                    char *log, size_t log_len);

/* Frees a mechanism and everything it owns.  NULL is a no-op.  Waits for
 * outstanding work of the mechanism to finish. */
void stev_destroy(stev_mechanism *mech);

/* Message of the last error on this host thread ("" if none). */
const char *stev_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* STEV_H */
