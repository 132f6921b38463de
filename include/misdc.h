/*
 * misdc.h — C ABI of the GB300 (sm_103a) concurrent MISDC library.
 *
 * The library advances the constant-density species/enthalpy
 * advection-diffusion-reaction system of Hamon, Day & Minion
 * (arXiv:1801.01201, Sec. 2) with the spectral deferred correction sweeps of
 * Sec. 3: serial MISDC (eqs. update_equation_misdc_discrete_form_D/R),
 * MISDCQ (eqs. update_equation_misdcq_discrete_form_D/R) and the concurrent
 * CISDCQ-nu (eqs. update_equation_amisdcq_discrete_form_D and _R_alt, lags
 * initial_lagged_values_A/D/R, steps I1-I4 and S1-S7 of Sec. 3.3). In CISDCQ
 * the diffusion step at node m+1 and the reaction step at node m run on two
 * CUDA streams (the two "processors" of the pipelining of Sec. 3.2.2).
 *
 * Conventions (all entry points):
 *  - Arrays are FP64 and laid out field-major: a state is [N+1][cells] with
 *    Y_1..Y_N then the mass-specific enthalpy h (J/kg, formation included);
 *    cells are x-fastest, then y, then z. Grids are periodic.
 *  - "device" pointers are CUDA device (or managed) memory owned by the
 *    caller; the library never frees them. "host" pointers are read during the
 *    call only. The library owns its internal buffers (freed by
 *    misdc_destroy).
 *  - Calls taking a stream are stream-ordered on it (NULL = legacy default
 *    stream) and do not synchronise unless stated. A stream-ordered call that
 *    fails inside a kernel reports it through misdc_get_stats().status.
 *  - Every call returns a misdc_status; on error misdc_last_error() gives a
 *    thread-local message. No C++ exception crosses the ABI. A handle is used
 *    by one host thread at a time.
 *  - Units are SI (kg, m, s, mol, K, J).
 */
#ifndef MISDC_H
#define MISDC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MISDC_OK = 0,
  MISDC_E_INVALID = 1,   /* bad argument or size                               */
  MISDC_E_CUDA = 2,      /* a CUDA runtime call failed                         */
  MISDC_E_NEWTON = 3,    /* a reaction Newton solve hit its iteration limit    */
  MISDC_E_MG = 4,        /* a diffusion solve missed its residual tolerance    */
  MISDC_E_TIMEOUT = 5,   /* a bounded device wait gave up                      */
  MISDC_E_NAN = 6,       /* non-finite value in a solve                        */
  MISDC_E_OOM = 7,       /* device allocation failed                           */
  MISDC_E_TDIAG = 8      /* temperature outside [50, 6000] K while diagnosing  */
} misdc_status;

typedef enum {
  MISDC_SCHEME_MISDC = 0,    /* node-to-node MISDC (backward/forward Euler)     */
  MISDC_SCHEME_MISDCQ = 1,   /* serial MISDC with LU-trick weights              */
  MISDC_SCHEME_CISDCQ = 2    /* concurrent implicit SDCQ with nu nested iters   */
} misdc_scheme;

typedef enum { MISDC_PREC_FP64 = 0, MISDC_PREC_MIXED = 1 } misdc_precision;

/* Mechanism (host arrays, copied at create). Mass-action kinetics:
 * k_f = A T^beta exp(-Ea/(R T)), k_r = k_f/K_c,
 * K_c = exp(-sum_i nu_i g_i/(R T)) (p_ref/(R T))^{sum_i nu_i}, where g_i from the
 * NASA-7 polynomial (one temperature range) and nu = nu_r - nu_f.
 * Each reaction may have at most 3 reactant and 3 product molecules (counting
 * multiplicity). Diffusivities: D_i(T) = D0_i (T/T_ref)^theta_exp for species
 * and lambda/(rho cp) = alpha0 (T/T_ref)^theta_exp for enthalpy. */
typedef struct misdc_mech_desc {
  int n_species;          /* N, 1..63                                  */
  int n_reactions;        /* R, 1..1024                                */
  const double *W;        /* [N] molar mass, kg/mol                    */
  const double *nasa7;    /* [N][7] a1..a7                             */
  const double *A;        /* [R] SI pre-exponential factor             */
  const double *beta;     /* [R] temperature exponent                  */
  const double *Ea;       /* [R] activation energy, J/mol              */
  const int *nu_f;        /* [R][N] reactant stoichiometric coefficients */
  const int *nu_r;        /* [R][N] product stoichiometric coefficients  */
  const double *D0;       /* [N] species diffusivity at T_ref, m^2/s   */
  double alpha0;          /* thermal diffusivity at T_ref, m^2/s       */
  double T_ref, theta_exp, p_ref;
} misdc_mech_desc;

/* Periodic uniform grid: dim 1..3, nx*ny*nz cells (ny = nz = 1 in 1D). */
typedef struct misdc_grid_desc {
  int dim, nx, ny, nz;
  double dx;
} misdc_grid_desc;

typedef struct misdc_opts {
  int n_nodes;            /* M+1 Gauss-Lobatto nodes, 2..9             */
  int n_sweeps;           /* sweeps per time step, >= 1                */
  int nu;                 /* nested iterations (CISDCQ), >= 1          */
  int scheme;             /* misdc_scheme                              */
  int precision;          /* misdc_precision                           */
  int dominant_species;   /* i0: closed by Y_i0 = 1 - sum of the others */
  double rho;             /* constant density, kg/m^3                  */
  double newton_rtol;     /* stop once max|dY| <= rtol, |dT| <= rtol T  */
  int newton_maxit;       /* iteration limit per cell                  */
  double lin_rtol;        /* diffusion solve: relative residual target  */
  int mg_levels;          /* 0 or 1: Chebyshev-accelerated Jacobi alone; > 1: multigrid
                             V-cycles on that many levels (fewer where an extent turns
                             odd), FP32 coarse levels in mixed precision              */
  int two_streams;        /* 1: D and R stages on separate streams     */
  int use_graph;          /* 1: capture the step in a CUDA graph       */
  int profile;            /* 1: time every Newton and diffusion-solve launch with CUDA events */
  int rates_mma;          /* 1: production rates (Sec. 2, omega-dot) contract diag(W) nu^T q
                             on the FP64 tensor cores (mma m8n8k4) instead of the sparse
                             FMA sum; the same values up to FP64 summation order     */
  double nu_eta;          /* > 0 (CISDCQ, nu > 2): adaptive nested iterations. The paper
                             asks for such a rule as future work (Sec. 4, 5); this one
                             runs iterations 0 and 1 of every sweep, then iteration l+1
                             only while delta_l > nu_eta delta_0 and delta_l <
                             nu_rho_stall delta_{l-1}, delta_l being the largest
                             field-relative max-norm change of the node states made by
                             iteration l (iteration 0: against sweep k); nu is the cap.
                             Captured steps decide on the device (IF graph nodes);
                             eager steps read the decision on the host.           */
  double nu_rho_stall;    /* the contraction bound of that rule (> 0 when nu_eta > 0) */
  int lanes;              /* CISDCQ on two streams: stream pairs for the nested
                             iterations, 1..min(nu, 4). With lanes > 1, iteration l
                             runs its diffusion and reaction steps on pair l mod lanes,
                             so iteration l+1 starts at a node as soon as iteration l
                             has passed the next one (the pipelining of up to 2 nu
                             tasks of Sec. 3.2.2, Fig. 2); results are bitwise those of
                             one pair. Each further pair has its own stage buffers.
                             Multigrid solves, the learned guess and the adaptive rule
                             use one pair. Default 1. */
  int lin_rounds;         /* mixed precision, Chebyshev diffusion solve: FP64-residual
                             refinement rounds around the FP32 inner solves (each
                             reduces the residual by about 1e-6); 0: 3 rounds      */
} misdc_opts;

typedef struct misdc_stats {
  long long newton_solves;      /* cell solves since the last reset      */
  long long newton_iters;       /* Newton iterations summed over cells   */
  long long newton_fail;        /* cells that failed                     */
  int newton_max;               /* most iterations taken by one cell     */
  int status;                   /* misdc_status of the device work       */
  long long lin_sweeps;         /* smoother sweeps per field, summed     */
  double lin_resid_max;         /* largest relative residual seen        */
  long long kernel_launches;    /* library kernels launched by misdc_step */
  long long surrogate_used;     /* cells whose Newton started from the learned guess */
  long long surrogate_rejected; /* learned guesses the residual test rejected */
  long long newton_fp64_fallbacks; /* mixed precision: solves restarted with FP64
                                      Newton after the mixed iteration failed */
  long long newton_jacobians;   /* Jacobian assemblies (every iteration in FP64 mode;
                                   mixed precision reuses factors between them) */
  long long newton_lu_fp64;     /* of which factorised in FP64 (the rest in FP32) */
  long long newton_certified;   /* mixed precision: solves whose guess a kept factor
                                   certified from the stored reaction term alone
                                   (counted as one iteration, no rate evaluated) */
  long long nested_iterations;  /* CISDCQ nested iterations run, summed over sweeps */
  long long newton_stored_steps; /* mixed precision: uncertified solves whose first
                                    chord step came from the stored reaction term
                                    (iteration 1 without a rate evaluation) */
  long long newton_floor_stops;  /* exact (FP64) Newton solves that stopped on the
                                    round-off-floor test: step d <= 1e-8 that no longer
                                    halves, while still above newton_rtol */
  long long newton_chord_cells;  /* mixed precision: uncertified solves finished by the
                                    thread-per-cell chord pass (stored first step, then
                                    chord iterations through the kept inverse) */
} misdc_stats;

typedef struct misdc_solver misdc_solver;

/* Fill misdc_opts with defaults: 3 nodes, 4 sweeps, nu = 2, CISDCQ, FP64,
 * newton_rtol 1e-12, newton_maxit 50, lin_rtol 1e-14, two streams, graph. */
void misdc_default_opts(misdc_opts *opts);

/* Create a solver. face_vel: device [3][cells] (only the first dim rows are
 * read), the velocity normal to the low face of each cell along x, y, z; it
 * should be discretely divergence free. The array is copied. */
misdc_status misdc_create(const misdc_mech_desc *mech, const misdc_grid_desc *grid,
                          const misdc_opts *opts, const double *face_vel,
                          misdc_solver **out);
void misdc_destroy(misdc_solver *s);

/* Advance n_steps time steps of size dt (Sec. 3.3, I1-I4 and S1-S7).
 * state: device [N+1][cells] in/out. T: device [cells] in/out temperature
 * (input used as the first guess of the temperature diagnosis; may be NULL).
 * Stream-ordered. */
misdc_status misdc_step(misdc_solver *s, double *state, double *T, double dt,
                        int n_steps, void *stream);

/* Same with HOST state/T buffers: copies in, steps, copies out, and waits for
 * the stream (the end-to-end path). */
misdc_status misdc_step_host(misdc_solver *s, double *state_host, double *T_host,
                             double dt, int n_steps, void *stream);

/* Read and reset the accumulated statistics (synchronises the device). */
misdc_status misdc_get_stats(misdc_solver *s, misdc_stats *stats, int reset);

/* With opts.profile = 1: device time of the reaction-Newton launches and of the
 * diffusion solves of the most recent time step, measured with CUDA events on
 * the streams they run on (synchronises the device). Outputs may be NULL. */
misdc_status misdc_stage_times(misdc_solver *s, double *newton_ms, int *newton_launches,
                               double *diffusion_ms, int *diffusion_launches);

/* Quadrature tables the device uses (host outputs, may be NULL):
 * tau[M+1], Q[M][M+1] (eq. weights), QI[M][M] = U^T of the unit-lower LU of
 * (Q without its first column)^T, QE[M][M] = dt^j/dt for j <= m. */
misdc_status misdc_lobatto(int n_nodes, double *tau, double *Q, double *QI, double *QE);

/* ---- row-level entry points (device arrays, stream-ordered) ------------- */

/* h = sum_i Y_i h_i(T) for n cells. Y [N][n], T [n], h [n]. */
misdc_status misdc_enthalpy(misdc_solver *s, const double *Y, const double *T, double *h,
                            int n, void *stream);
/* T from sum_i Y_i h_i(T) = h, Newton safeguarded on [50, 6000] K. T in: guess
 * (<= 0 means none), out: temperature. */
misdc_status misdc_temperature(misdc_solver *s, const double *Y, const double *h, double *T,
                               int n, void *stream);
/* Production rates F_R = wdot/rho, [N][n] (Sec. 2, eq. species_equation). */
misdc_status misdc_production_rates(misdc_solver *s, const double *Y, const double *T,
                                    double *FR, int n, void *stream);
/* Reaction step S5 for n independent cells (Sec. 3.3, eq.
 * reaction_step_numerical_methodology):
 * Y - wdt wdot(Y,T)/rho = b,  sum_i Y_i h_i(T) = hstar, Newton from the guess
 * with the analytic Jacobian and partial-pivot LU, one warp per cell.
 * b [N][n], hstar [n]; x [N+1][n] in: guess (Y, T), out: solution;
 * FR [N][n] out: the reaction term of the solution, (Y - b)/wdt, which equals
 * wdot/rho up to the Newton tolerance (may be NULL); iters [n] out (may be
 * NULL): iterations, or -1 (limit), -2 (singular), -3 (non-finite or T <= 0). */
misdc_status misdc_reaction_solve(misdc_solver *s, double wdt, const double *b,
                                  const double *hstar, double *x, double *FR, int *iters,
                                  int n, void *stream);
/* Right-hand sides at a full state [N+1][cells] on the solver's grid:
 * FE = advection (+ explicit differential diffusion of h), FD = diffusion,
 * FR = reaction (each may be NULL). */
misdc_status misdc_operators(misdc_solver *s, const double *state, double *FE, double *FD,
                             double *FR, void *stream);
/* Implicit diffusion step: x - wdt F_D[coef](x) = rhs for every field but the
 * dominant species (closed by 1 - sum), coefficients frozen at coef_state,
 * followed by the flux-form reconstruction x := rhs + wdt F_D[coef](x). */
misdc_status misdc_diffusion_solve(misdc_solver *s, double wdt, const double *coef_state,
                                   const double *rhs, double *x, void *stream);
/* Linear combination out[o][e] = sum_k w[o][k] in[k][e] over n elements for
 * n_out <= 8 outputs and n_in <= 16 inputs (host arrays of device pointers and
 * weights): the spectral-integration kernel that applies Q to the node stack. */
misdc_status misdc_lincomb(int n_out, int n_in, double *const *out, const double *const *in,
                           const double *w, size_t n, void *stream);

/* The FP64 exponential of the rate kernels (production rates and the reaction
 * Newton: k_f = exp(ln A + beta ln T - Ea/(R T)) and k_r, Sec. 2), for testing:
 * y[i] = e^{x[i]} over n device elements, stream-ordered. Tang's table-driven
 * method (ACM TOMS 15(2), 1989) with a 32-entry table of 2^(j/32); about 1 ulp;
 * arguments outside (-700, 700) fall back to the CUDA exp. */
misdc_status misdc_exp(const double *x, double *y, size_t n, void *stream);

/* Arithmetic-throughput probe, the measured denominator of the roofline
 * fractions of the FP64-bound kernels. The paper has no counterpart (it reports
 * no hardware figures). kind 0: FP64 FMA, 8 independent chains per thread;
 * kind 1: FP64 tensor-core MMA (m8n8k4, 512 flops each), 4 independent
 * accumulators per warp; kind 2: FP32 FMA, 8 chains per thread. Launches
 * `blocks` blocks of 256 threads running `iters` iterations each, stream-ordered;
 * out: device [blocks * 256] doubles (results, so nothing is optimised away);
 * *flops (host) receives the flops the launch performs (an FMA counts 2). The
 * caller times the launch. MISDC_E_INVALID for a bad kind or size. */
misdc_status misdc_probe_flops(int kind, int blocks, int iters, double *out, double *flops,
                               void *stream);

/* ---- nonlinear scalar test PDE (Sec. 5.2, eq. nonlinear_test_pde) ---------
 * phi_t = a phi_x + d phi_xx + r phi (phi - 1)(phi - 1/2) on [0, length] with
 * phi(0) = left, phi(length) = right, in nx uniform cells: fourth-order advective
 * face values (7 (phi_i + phi_{i+1}) - (phi_{i-1} + phi_{i+2}))/12, the
 * fourth-order five-point Laplacian, and Dirichlet ghost cells from the cubic
 * through the wall value and the first three cell averages (the paper does not
 * state its closure). Advances n independent instances n_steps time steps of dt
 * with the scheme (misdc_scheme), n_nodes Gauss-Lobatto nodes, n_sweeps sweeps
 * and nu nested iterations (CISDCQ), each step starting from phi^n at all
 * nodes (Sec. 3.3, I1-I2). Diffusion steps solve (I - w L) x = rhs + w g
 * directly (banded LU with partial pivoting); reaction steps run scalar Newton
 * to |dy| <= 1e-15 (1 + |y|), at most 100 iterations.
 * Device arrays, stream-ordered: params [n][5] = (a, d, r, left, right);
 * phi_in, phi_out [n][nx] (may alias); incr [n][n_steps][n_sweeps] (may be NULL)
 * receives the sweep increments (1/nx) sum_i |phi^{M,(k+1)}_i - phi^{M,(k)}_i|;
 * status [n] (may be NULL): 0, or bits 1 (Newton limit), 2 (non-finite),
 * 4 (singular diffusion matrix). Below 4096 instances one block per instance
 * holds all node arrays in shared memory: misdc_pde_smem_bytes gives the need,
 * and a launch whose need exceeds the device's per-block limit returns
 * MISDC_E_INVALID (at 5 nodes about 340 cells, at 3 nodes about 610). From 4096
 * instances on, one thread per instance works on a workspace laid out
 * [array][cell][instance] (coalesced across a warp), which the call allocates
 * and frees stream-ordered (cudaMallocAsync / cudaFreeAsync; MISDC_E_OOM when it
 * does not fit). nx >= 8. */
misdc_status misdc_pde_step(int scheme, int n_nodes, int n_sweeps, int nu, double dt, int n_steps,
                            int nx, double length, int n, const double *params,
                            const double *phi_in, double *phi_out, double *incr, int *status,
                            void *stream);
misdc_status misdc_pde_smem_bytes(int n_nodes, int nx, size_t *bytes);

/* ---- variable-density low-Mach coupling, independent 1D flames -------------
 * The paper's own setting (Sec. 2: eqs. continuity_equation, species_equation,
 * enthalpy_equation, p_eos_definition, divergence_constraint and S_def; Sec. 3.3:
 * steps I1-I4 and S1-S7 with S2 the density update, S3-S4 the species and
 * enthalpy diffusion solved against the new density, S5 the reaction Newton at
 * the new density with h fixed, S6 the volume-discrepancy correction delta_chi
 * and the velocity from div U = S + delta_chi): one time step of CISDCQ-nu (or
 * the serial MISDCQ) for n independent flames on the solver's 1D grid, one thread
 * block per flame. State per flame q = [rho, rho Y_1..rho Y_N, rho h], [N+2][nx].
 * Open boundaries: at x = 0 an inflow Dirichlet state (Y_in, T_in, density from
 * the EOS at p0) and face velocity U_in; at x = nx dx zero-gradient outflow with
 * no diffusive flux. Advection: fourth-order centred face values of q (inflow
 * value on the inflow face and as the first face's outer ghost, the last cell
 * beyond the outflow); diffusion: second-order fluxes with harmonic-mean
 * rho theta(T) coefficients (the inflow face takes the first cell's, with the
 * gradient to the inflow value half a cell away), dominant species closed by
 * minus the others' flux, differential diffusion of h explicit; S with
 * Gamma_i = rho D_i grad Y_i; delta_chi per cell and node, incremented each sweep
 * by (2/p0)(p_EOS - p0)/dt_m (d->dchi = 0: no correction). The implicit diffusion
 * systems are tridiagonal and solved directly; S5 is Newton with the analytic
 * Jacobian (newton_rtol, newton_maxit of the solver's options).
 * The solver (created on a 1D grid) supplies the mechanism, nx, dx, n_nodes,
 * n_sweeps, nu, scheme and dominant_species. Device arrays, stream-ordered:
 * q_in, q_out [n][N+2][nx] (may alias); peos [n][nx] (may be NULL): p_EOS of the
 * result; status [n] (may be NULL): 0, or bits 1 (Newton limit), 2 (temperature
 * outside [50, 6000] K), 4 (non-finite or singular). The workspace (about
 * 8 ((M+1)(12 (N+2) + 6) + 30 N + (N+1)^2) nx bytes per flame) is allocated and freed
 * stream-ordered (MISDC_E_OOM when it does not fit). */
typedef struct misdc_lowmach_desc {
  double U_in;          /* velocity on the inflow face, m/s   */
  double T_in;          /* inflow temperature, K              */
  double p0;            /* thermodynamic pressure, Pa         */
  const double *Y_in;   /* [N] host: inflow mass fractions    */
  int dchi;             /* 1: the delta_chi correction of S6  */
} misdc_lowmach_desc;
misdc_status misdc_lowmach_step(misdc_solver *s, const misdc_lowmach_desc *d, double dt, int n,
                                const double *q_in, double *q_out, double *peos, int *status,
                                void *stream);

/* Reaction solve that allocates nothing. The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory during the call (host
 * callbacks, memory-pool-restricted or real-time processes, plugins whose host
 * owns every allocation). Same arguments, results and stream semantics as
 * misdc_reaction_solve; its scratch lives in one static 4 MiB device array that
 * every device loading the library keeps until the process exits. Needs
 * 32 + n (N+1) doubles of it: a larger n returns MISDC_E_INVALID. Calls share
 * the array, so calls that overlap on the GPU race; the first call on a device
 * looks the array up and should come before any stream capture. Accumulates
 * no solver statistics (the per-cell iteration codes are in iters). */
misdc_status misdc_reaction_solve_noalloc(misdc_solver *s, double wdt, const double *b,
                                          const double *hstar, double *x, double *FR, int *iters,
                                          int n, void *stream);

/* ---- learned initial guess of the reaction Newton ------------------------
 * The paper has no counterpart: this is the learned form of the reaction step
 * S5 (Sec. 3.3), whose Newton otherwise starts from the previous iterate
 * x_p = (Y_p, T_p) of the same node. A per-solver MLP
 * n_in -> 256 -> 256 -> 256 -> n_out (GELU, BF16 weights and activations,
 * FP32 accumulation, tensor-core kernels) maps the features of a cell
 *   r_i = b_i - Y_p,i + wdt F_p,i,  r_T = (h* - h_p)/(cp(x_p) T_p),
 *   s = max(max_i |r_i|, |r_T|),
 *   f = [Y_p (N), (T_p - 1150)/850, log10(wdt) + 6, r/s (N), r_T/s]   (n_in = 2N+3)
 * to p (n_out = N+1); Newton starts from Y_p + s p_Y, T_p (1 + s p_T) (the T
 * factor clamped to [0.5, 1.5]) when s > s_min, and keeps that start only if
 * the scaled residual max-norm there is below s; otherwise it starts from x_p.
 * Training targets are [(Y* - Y_p)/s, (T* - T_p)/(T_p s)] clipped to [-8, 8],
 * recorded from the solver's own reaction steps. BF16 feature rows have
 * ldx = n_in rounded up to 8 columns; target and output rows have ldo = n_out
 * rounded up to 16 columns (padding zero). The FP32 parameter vector is
 * W1 [256][ldx], W2 [256][256], W3 [256][256], W4 [ldo][256], b1, b2, b3 [256],
 * b4 [ldo] (row-major, y = W x + b); padded entries must be zero.
 * The network state lives in the solver and is created on first use. Calls that
 * change what misdc_step does (enable, collect) drop its captured graph. */
misdc_status misdc_surrogate_dims(misdc_solver *s, int *n_in, int *ldx, int *n_hidden, int *n_out,
                                  int *ldo, size_t *n_params);
/* Random initial parameters (seeded; output layer scaled by 0.1), Adam state reset. */
misdc_status misdc_surrogate_init(misdc_solver *s, unsigned long long seed);
/* Load / save the FP32 parameter vector (host arrays of n_params floats; synchronous). */
misdc_status misdc_surrogate_load(misdc_solver *s, const float *params, size_t n_params);
misdc_status misdc_surrogate_save(misdc_solver *s, float *params, size_t n_params);
/* on = 1: later misdc_step calls start each reaction Newton from the learned guess
 * (needs parameters). s_min: cells with s <= s_min keep x_p. */
misdc_status misdc_surrogate_enable(misdc_solver *s, int on, double s_min);
/* The learned guess serves only the first n_sweeps sweeps of every time step
 * (0, the default: all). Later sweeps start from iterates that the previous
 * sweep has already converged, where plain Newton (or a kept factor's
 * certification) needs no help and the network's inference is overhead. */
misdc_status misdc_surrogate_sweeps(misdc_solver *s, int n_sweeps);
/* capacity > 0: later misdc_step calls record (features, target) rows of every
 * reaction solve with s > s_min (plain Newton from x_p) until capacity rows are
 * held; a larger capacity starts a new, empty dataset. 0 stops recording. */
misdc_status misdc_surrogate_collect(misdc_solver *s, long long capacity);
/* Rows recorded so far and the library-owned device arrays holding them
 * (X: BF16 [rows][ldx], targets: FP32 [rows][ldo]); synchronises the solver. */
misdc_status misdc_surrogate_dataset(misdc_solver *s, long long *rows, const void **X,
                                     const float **targets);
/* Train on the recorded rows: steps AdamW steps (beta 0.9/0.999, eps 1e-8,
 * decoupled weight decay on the weights only, learning rate lr with cosine decay
 * to 0.05 lr) on minibatches of `batch` rows drawn with a counter-based
 * generator from `seed`; mean-squared loss over the n_out outputs. loss_curve:
 * host [steps] (may be NULL). Synchronous. */
misdc_status misdc_surrogate_train(misdc_solver *s, int steps, int batch, double lr,
                                   double weight_decay, unsigned long long seed,
                                   float *loss_curve);
/* Row-level entry points (device arrays, stream-ordered):
 * features of n cells: b, Yp, FRp [N][n]; hstar, Tp, hp [n]; X out BF16 [n][ldx];
 * scale out [n] (= s). */
misdc_status misdc_surrogate_features(misdc_solver *s, double wdt, const double *b,
                                      const double *hstar, const double *Yp, const double *Tp,
                                      const double *FRp, const double *hp, int n, void *X,
                                      double *scale, void *stream);
/* out FP32 [n][ldo] = MLP(X BF16 [n][ldx]): the fused inference kernel (all
 * four layers per 128-row tile on chip). */
misdc_status misdc_surrogate_forward(misdc_solver *s, const void *X, int n, float *out,
                                     void *stream);
/* Same result from one tensor-core GEMM launch per layer (the training kernels). */
misdc_status misdc_surrogate_forward_layers(misdc_solver *s, const void *X, int n, float *out,
                                            void *stream);
/* What a reaction step uses: features of n cells computed from the state (as in
 * misdc_surrogate_features) and the network's output, in one fused launch.
 * out FP32 [n][ldo], scale [n] (= s). */
misdc_status misdc_surrogate_guess(misdc_solver *s, double wdt, const double *b, const double *hstar,
                                   const double *Yp, const double *Tp, const double *FRp,
                                   const double *hp, int n, float *out, double *scale, void *stream);
/* Gradient of the mean-squared loss (mean over n rows and n_out outputs) against
 * targets FP32 [n][ldo]: grad [n_params] and loss [1] (device, may be NULL). */
misdc_status misdc_surrogate_gradient(misdc_solver *s, const void *X, const float *targets, int n,
                                      float *grad, float *loss, void *stream);
/* misdc_surrogate_gradient followed by one AdamW step with learning rate lr. */
misdc_status misdc_surrogate_train_batch(misdc_solver *s, const void *X, const float *targets, int n,
                                         double lr, double weight_decay, float *loss, void *stream);

/* ---- launch-shape autotuner -------------------------------------------------
 * Launch shapes of the two hot kernels. The paper has no counterpart (it runs
 * on CPU cores); these are GPU scheduling choices that leave results unchanged. */
typedef struct misdc_tuning {
  int newton_warps_per_block;   /* cells (one warp each) per block, 1..4; 0 = largest that fits */
  int newton_blocks_per_sm;     /* cap on resident blocks per SM; 0 = default */
  int newton_dynamic;           /* 1: warps take the next cell from a global counter */
  int cheb_block;               /* threads per block of the smoother sweep; 0 = 256 */
  int newton_keep_factors;      /* mixed precision: 1 (default) keeps each cell's FP32
                                   Jacobian factor between the solves of an SDC node,
                                   0 rebuilds it in every solve */
  int newton_chord_iters;       /* mixed precision with kept factors: chord iterations a
                                   cell may take in the thread-per-cell pass after
                                   certification before it goes to the warp-per-cell
                                   Newton (0: certification only); default 4. Unlike the
                                   other fields this changes which kernel solves a cell,
                                   so results move within the solver tolerance */
  double newton_ms;             /* autotune: best time of the probe reaction solve */
  double cheb_ms;               /* autotune: best time of the probe diffusion solve */
} misdc_tuning;
/* Time candidate shapes on this solver's grid and mechanism (a reaction step of
 * weight max_m dt q~I_mm from `state` with temperature T, and a diffusion solve
 * of the same weight; device arrays) and keep the fastest. Synchronous; resets
 * the statistics. */
misdc_status misdc_autotune(misdc_solver *s, const double *state, const double *T, double dt,
                            misdc_tuning *out);
misdc_status misdc_get_tuning(misdc_solver *s, misdc_tuning *out);
misdc_status misdc_set_tuning(misdc_solver *s, const misdc_tuning *t);

/* ---- batched stepping of independent flames ----------------------------------
 * A batch holds n solvers (each with its own mechanism, grid and options) and
 * advances all of them with one CUDA graph launch per time step: the flames'
 * step programs run concurrently, each on its own pair of streams, so that many
 * small grids fill the GPU together. The graph is captured on the first call and
 * again whenever a state or T pointer or a dt changes. states[i] / T[i]
 * (T may be NULL, or hold NULL entries) are device arrays of solver i; dts[i]
 * its time step. The solvers must not record solves while batched.
 *
 * Reaction steps (Sec. 3.3, S5) of the flames are grouped by default: the k-th
 * reaction step of every flame whose mechanism has the same species and reaction
 * counts and whose launch has the same shape becomes one persistent launch over
 * the cells of all of them, fed from one work counter (a warp takes the next free
 * cell of any of the flames), so uneven per-cell Newton work is balanced across
 * flames; each flame's stage waits for that launch. Grouping needs every flame to
 * have the same number of reaction steps per time step, each flame's steps in one
 * sequence (one stream pair, a fixed nu); otherwise, or with grouping off, every
 * flame keeps its own launches. Results are bitwise the same either way. */
typedef struct misdc_batch misdc_batch;
misdc_status misdc_batch_create(misdc_solver *const *solvers, int n, misdc_batch **out);
void misdc_batch_destroy(misdc_batch *b);
misdc_status misdc_batch_step(misdc_batch *b, double *const *states, double *const *T,
                              const double *dts, int n_steps, void *stream);
/* Statistics summed over the batch's solvers (synchronises). */
misdc_status misdc_batch_stats(misdc_batch *b, misdc_stats *out, int reset);
/* Grouping of the flames' reaction steps (on = 1, the default, or 0); takes
 * effect at the next capture (a change drops the current graph). */
misdc_status misdc_batch_set_grouping(misdc_batch *b, int on);
/* Of the current graph (zeros before the first step, or without grouping): the
 * grouped reaction launches per time step and the per-flame reaction steps they
 * replace. */
misdc_status misdc_batch_grouping(misdc_batch *b, int *grouped_launches, int *grouped_solves);

const char *misdc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
