/*
 * Plain serial FP64 CPU oracle for the multi-implicit SDC schemes of
 * Hamon, Day & Minion (arXiv:1801.01201).
 *
 * TEST INFRASTRUCTURE ONLY. This library is the independent checker of the
 * CUDA library: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it. It shares no code, header, table or constant with
 * the CUDA path.
 *
 * Contents
 *  - Gauss-Lobatto quadrature tables Q, S, Q~I (LU trick), Q~E  (Sec. 3.1)
 *  - generic sweeps MISDC, MISDCQ, CISDCQ-nu, IMEXQ over callbacks
 *    (Sec. 3.1 and 3.2, eqs. update_equation_misdc_discrete_form_D/R,
 *     update_equation_misdcq_discrete_form_D/R,
 *     update_equation_amisdcq_discrete_form_D/R/R_alt,
 *     initial_lagged_values_A/D/R)
 *  - problems: linear model ODE (Sec. 4), nonlinear test PDE (Sec. 5.2),
 *    low-Mach species/enthalpy ADR with prescribed velocity (Sec. 2, 3.3),
 *    and the 1D variable-density low-Mach system with open boundaries, the
 *    velocity from the divergence constraint and the volume-discrepancy
 *    correction (Sec. 2, eqs. divergence_constraint and S_def; Sec. 3.3 I3,
 *    I4, S2-S6)
 */
#ifndef MISDC_ORACLE_H
#define MISDC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_MISDC = 0, OR_MISDCQ = 1, OR_CISDCQ = 2, OR_IMEXQ = 3 };

/* Tables for M+1 Gauss-Lobatto nodes on [0,1].
 * tau[M+1]; Q[M][M+1] (row m-1 integrates 0 -> tau_m); S[M][M+1]
 * (row m-1 integrates tau_{m-1} -> tau_m); QI[M][M]; QE[M][M].
 * Returns 0 on success. */
int or_lobatto(int M, double *tau, double *Q, double *S, double *QI, double *QE);

/* ---- generic sweep over callbacks ------------------------------------- */
typedef struct or_problem {
  int n;         /* length of the state vector */
  void *ctx;
  /* explicit part F_E (advection, plus explicit differential diffusion) */
  void (*f_expl)(void *ctx, const double *phi, double *out);
  /* implicit diffusion F_D evaluated with the state's own coefficients */
  void (*f_diff)(void *ctx, const double *phi, double *out);
  /* reaction F_R */
  void (*f_reac)(void *ctx, const double *phi, double *out);
  /* x - wdt * F_D[coef](x) = rhs, coefficients frozen at coef_state */
  int (*solve_diff)(void *ctx, double wdt, const double *coef_state,
                    const double *rhs, double *x);
  /* x - wdt * F_R(x) = b, Newton started from guess */
  int (*solve_reac)(void *ctx, double wdt, const double *b,
                    const double *guess, double *x);
  /* x - wdt * (F_D + F_R)(x) = rhs (IMEXQ only; may be NULL) */
  int (*solve_coupled)(void *ctx, double wdt, const double *rhs,
                       const double *guess, double *x);
  /* the state is n_fields contiguous fields of n / n_fields entries (0 = 1);
   * only the adaptive nested-iteration rule looks at it */
  int n_fields;
} or_problem;

/* Adaptive number of nested iterations of a CISDCQ sweep (the paper leaves the
 * mechanism to future work, Sec. 4 and 5; this rule is a reading). delta_l is
 * the field-relative max-norm of phi^{(k+1,l+1)} - phi^{(k+1,l)} over nodes
 * 1..M (delta_0: the first nested iteration against sweep k). Iterations 0 and
 * 1 always run; after iteration l >= 1, iteration l+1 runs only while l+1 < nu,
 * delta_l > eta delta_0 (the nested iterations have not yet settled relative
 * to the sweep's own change) and delta_l < rho_stall delta_{l-1} (they still
 * contract fast enough to pay for another pass). eta <= 0: all nu run. */
typedef struct or_nu_rule {
  double eta, rho_stall;
} or_nu_rule;

/* One sweep (k) -> (k+1). Phi_k[(M+1)*n] holds node values of sweep k
 * (node 0 = phi^n), Phi_out[(M+1)*n] receives sweep k+1. */
int or_sweep(const or_problem *p, int scheme, int M, int nu, double dt,
             const double *Phi_k, double *Phi_out);

/* As or_sweep, with the adaptive rule (NULL: all nu); *nu_used (optional)
 * receives the nested iterations the sweep ran (1 for the other schemes). */
int or_sweep_ex(const or_problem *p, int scheme, int M, int nu, const or_nu_rule *rule,
                double dt, const double *Phi_k, double *Phi_out, int *nu_used);

/* One time step: spread phi_n to all nodes (I1-I2), n_sweeps sweeps,
 * phi_out = node M. incr[n_sweeps] (optional) receives the L1 norm (mean
 * over entries) of phi^{M,(k+1)} - phi^{M,(k)} per sweep. */
int or_step(const or_problem *p, int scheme, int M, int n_sweeps, int nu,
            double dt, const double *phi_n, double *phi_out, double *incr);
/* ... with the adaptive rule; nu_used[n_sweeps] optional */
int or_step_ex(const or_problem *p, int scheme, int M, int n_sweeps, int nu,
               const or_nu_rule *rule, double dt, const double *phi_n, double *phi_out,
               double *incr, int *nu_used);

/* ---- linear model problem phi' = (a + d + r) phi (Sec. 4) ------------- */
int or_linear_step(int scheme, int M, int n_sweeps, int nu, double dt,
                   double a, double d, double r, double phi0,
                   double *phi_out, double *incr);
int or_linear_step_ex(int scheme, int M, int n_sweeps, int nu, const or_nu_rule *rule,
                      double dt, double a, double d, double r, double phi0,
                      double *phi_out, double *incr, int *nu_used);
/* Iteration matrix G (M x M) of one sweep on the linear model problem. */
int or_linear_G(int scheme, int M, int nu, double dt, double a, double d,
                double r, double *G);

/* ---- nonlinear test PDE (Sec. 5.2) ------------------------------------ */
/* phi_t = a phi_x + d phi_xx + r phi (phi - 1)(phi - 1/2) on [0, Lx],
 * phi(0) = left, phi(Lx) = right; fourth-order finite volumes. */
int or_pde_step(int scheme, int M, int n_sweeps, int nu, double dt,
                int nx, double Lx, double a, double d, double r,
                double left, double right, const double *phi_n,
                double *phi_out, double *incr);

/* ---- combustion advection-diffusion-reaction (Sec. 2 and 3.3) -------- */
typedef struct or_mech {
  int N, R;
  const double *W;       /* [N] kg/mol */
  const double *nasa7;   /* [N][7] */
  const double *A, *beta, *Ea;   /* [R] SI, -, J/mol */
  const int *nu_f, *nu_r;        /* [R][N] */
  const double *D0;      /* [N] m^2/s at T_ref */
  double alpha0, T_ref, theta_exp, p_ref;
} or_mech;

typedef struct or_adr_cfg {
  int dim, nx, ny, nz;
  double dx;
  const double *vel;     /* [3][cells] low-face velocities */
  double rho;
  int i0;                /* dominant species */
  double newton_rtol;
  int newton_maxit;
  double lin_rtol;
  int lin_maxit;
} or_adr_cfg;

typedef struct or_adr_stats {
  long newton_solves, newton_iters, newton_fail, newton_maxit_seen;
  long lin_solves, lin_iters, lin_fail;
  long tdiag_fail;
  long newton_floor;     /* reaction solves that ended on the round-off-floor test */
} or_adr_stats;

/* State layout phi[(N+1)][cells]: Y_1..Y_N then h (J/kg). */
int or_adr_step(const or_mech *mech, const or_adr_cfg *cfg, int scheme, int M,
                int n_sweeps, int nu, double dt, const double *phi_n,
                double *phi_out, double *incr, or_adr_stats *stats);
int or_adr_step_ex(const or_mech *mech, const or_adr_cfg *cfg, int scheme, int M,
                   int n_sweeps, int nu, const or_nu_rule *rule, double dt,
                   const double *phi_n, double *phi_out, double *incr, int *nu_used,
                   or_adr_stats *stats);

/* pieces, exposed for pins */
/* ---- variable-density low-Mach coupling, 1D with open boundaries --------- */
typedef struct or_lm_cfg {
  int nx;
  double dx;
  double U_in;          /* velocity on the inflow face x = 0, m/s */
  const double *Y_in;   /* [N] inflow mass fractions */
  double T_in;          /* inflow temperature, K */
  double p0;            /* ambient thermodynamic pressure, Pa */
  int i0;               /* dominant species */
  double newton_rtol;
  int newton_maxit;
  int dchi;             /* 1: the volume-discrepancy correction of S6 */
} or_lm_cfg;

int or_lm_terms(const or_mech *m, const or_lm_cfg *g, const double *q, const double *dchi,
                const double *Uadv, double *FA, double *FD, double *FR, double *S, double *U,
                double *peos, double *T);
int or_lm_step(const or_mech *m, const or_lm_cfg *g, int M, int n_sweeps, int nu, double dt,
               const double *q_n, double *q_out, double *incr, double *peos_out);
int or_lm_step_ex(const or_mech *m, const or_lm_cfg *g, int scheme, int M, int n_sweeps, int nu,
                  double dt, const double *q_n, double *q_out, double *incr, double *peos_out);

double or_species_h(const or_mech *m, int i, double T);     /* J/kg */
double or_species_cp(const or_mech *m, int i, double T);    /* J/(kg K) */
double or_species_s_R(const or_mech *m, int i, double T);   /* s/R (molar) */
int or_h_from_T(const or_mech *m, int cells, const double *Y, const double *T,
                double *h);
int or_T_from_h(const or_mech *m, int cells, const double *Y, const double *h,
                double *T);
/* production rates wdot[N] (kg/m^3/s) of one cell; q[R] optional */
void or_wdot(const or_mech *m, double rho, const double *Y, double T,
             double *wdot, double *q);
/* analytic Jacobian of wdot wrt (Y_1..Y_N, T): J[N][N+1] */
void or_wdot_jac(const or_mech *m, double rho, const double *Y, double T,
                 double *J);
/* per-cell reaction solve  Y - wdt*wdot(Y,T)/rho = b, sum Y h(T) = hstar;
 * x[N+1] in: guess (Y,T), out: solution. Returns iterations (<0 failure). */
int or_reaction_newton(const or_mech *m, double rho, double wdt, const double *b,
                       double hstar, double *x, double rtol, int maxit);
/* the same; *floor_stop = 1 when the solve ended on the round-off-floor test
 * (d <= 1e-8 and d >= d_prev / 2 with d > rtol), else 0 (may be NULL) */
int or_reaction_newton_ex(const or_mech *m, double rho, double wdt, const double *b,
                          double hstar, double *x, double rtol, int maxit, int *floor_stop);
/* operators on a full state (for pins) */
int or_adr_operators(const or_mech *mech, const or_adr_cfg *cfg, const double *phi,
                     double *FE, double *FD, double *FR);
int or_adr_solve_diff(const or_mech *mech, const or_adr_cfg *cfg, double wdt,
                      const double *coef_state, const double *rhs, double *x);

#ifdef __cplusplus
}
#endif
#endif
