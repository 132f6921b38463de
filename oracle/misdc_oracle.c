/*
 * Plain serial FP64 CPU oracle for the multi-implicit SDC schemes of
 * Hamon, Day & Minion (arXiv:1801.01201).
 *
 * TEST INFRASTRUCTURE ONLY: the independent checker of the CUDA library.
 * Only tests, the smoke check and the benchmark's CPU-baseline leg load it.
 * Nothing here is shared with the CUDA path.
 *
 * Everything is written for clarity, not speed: loops follow the paper's
 * equations term by term, in the paper's order and notation. Readings of
 * passages that are silent, ambiguous or garbled are stated where they are
 * used.
 *
 * Pins (tests/test_oracle_*.py) fix this code against the paper: the worked
 * three-node tables, the collocation (Lobatto IIIA / Pade) fixed point of the
 * sweeps, the sweep counts behind Tables 1-3, time order on the nonlinear test
 * PDE, finite-difference Jacobians, detailed balance, conservation, and dense
 * brute-force solves on tiny grids.
 */
#include "misdc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define R_UNIV 8.314462618

/* ======================================================================= */
/* Quadrature tables (Sec. 3.1, eq. "weights" and the LU trick)            */
/* ======================================================================= */

/* Legendre P_M(x) and P'_M(x) by the three-term recurrence. */
static void legendre(int M, long double x, long double *p, long double *dp) {
  long double p0 = 1.0L, p1 = x;
  if (M == 0) { *p = 1.0L; *dp = 0.0L; return; }
  for (int k = 2; k <= M; ++k) {
    long double pk = ((2.0L * k - 1.0L) * x * p1 - (k - 1.0L) * p0) / k;
    p0 = p1; p1 = pk;
  }
  *p = p1;
  /* (1 - x^2) P'_M = M (P_{M-1} - x P_M) */
  *dp = M * (p0 - x * p1) / (1.0L - x * x);
}

/* Gauss-Lobatto nodes on [0,1]: endpoints plus the roots of P'_M. */
static int lobatto_nodes(int M, long double *tau) {
  tau[0] = 0.0L; tau[M] = 1.0L;
  for (int j = 1; j < M; ++j) {
    long double x = -cosl(3.14159265358979323846264338327950288L * j / M);
    for (int it = 0; it < 100; ++it) {
      long double p, dp;
      legendre(M, x, &p, &dp);
      /* Legendre ODE: (1-x^2) P'' = 2x P' - M(M+1) P */
      long double d2p = (2.0L * x * dp - M * (M + 1.0L) * p) / (1.0L - x * x);
      long double step = dp / d2p;
      x -= step;
      if (fabsl(step) < 1e-19L) break;
    }
    tau[j] = 0.5L * (x + 1.0L);
  }
  return 0;
}

/* integral over [a,b] of the Lagrange basis polynomial L_j on nodes tau */
static long double lagrange_integral(int M, const long double *tau, int j,
                                     long double a, long double b) {
  long double c[64];
  memset(c, 0, sizeof(c));
  c[0] = 1.0L;
  int deg = 0;
  for (int k = 0; k <= M; ++k) {
    if (k == j) continue;
    long double den = tau[j] - tau[k];
    /* multiply by (t - tau_k)/den */
    for (int p = deg + 1; p >= 0; --p) {
      long double v = (p > 0 ? c[p - 1] : 0.0L) - tau[k] * c[p];
      c[p] = v / den;
    }
    ++deg;
  }
  long double s = 0.0L;
  for (int p = 0; p <= deg; ++p)
    s += c[p] * (powl(b, p + 1) - powl(a, p + 1)) / (p + 1);
  return s;
}

int or_lobatto(int M, double *tau_out, double *Q, double *S, double *QI, double *QE) {
  if (M < 1 || M > 16) return 1;
  long double tau[17];
  lobatto_nodes(M, tau);
  for (int m = 0; m <= M; ++m) if (tau_out) tau_out[m] = (double)tau[m];
  long double Qt[16][16], U[16][16], L[16][16];
  for (int m = 1; m <= M; ++m)
    for (int j = 0; j <= M; ++j) {
      long double q = lagrange_integral(M, tau, j, 0.0L, tau[m]);
      long double s = lagrange_integral(M, tau, j, tau[m - 1], tau[m]);
      if (Q) Q[(m - 1) * (M + 1) + j] = (double)q;
      if (S) S[(m - 1) * (M + 1) + j] = (double)s;
      if (j >= 1) Qt[j - 1][m - 1] = q;     /* Qt = (Q~)^T, Q~ = Q without its first column */
    }
  /* Doolittle LU of (Q~)^T = L U with unit-diagonal L (Weiser's LU trick):
   * "the upper triangular matrix in the LU decomposition" is read as the U of
   * the unit-lower / upper factorisation. */
  for (int i = 0; i < M; ++i) {
    for (int j = i; j < M; ++j) {
      long double s = Qt[i][j];
      for (int k = 0; k < i; ++k) s -= L[i][k] * U[k][j];
      U[i][j] = s;
    }
    L[i][i] = 1.0L;
    for (int j = i + 1; j < M; ++j) {
      long double s = Qt[j][i];
      for (int k = 0; k < i; ++k) s -= L[j][k] * U[k][i];
      L[j][i] = s / U[i][i];
    }
    for (int j = 0; j < i; ++j) U[i][j] = 0.0L;
  }
  /* Q~I := U^T.
   * Q~E: forward Euler integrated from t^0, q~E_{m+1,j} = dt^j/dt for every
   * j <= m and 0 for j >= m+1. The printed definition ("q~E_{m+1,m} := dt^m/dt,
   * q~E_{m+1,j != m+1} := 0") is read as this cumulative rule: the CISDCQ
   * update keeps explicit terms for j <= m-1, which would vanish otherwise,
   * and only this reading reproduces the sweep counts of Tables 1 and 2.
   * For three nodes both readings give the same matrix. */
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      if (QI) QI[i * M + j] = (double)U[j][i];
      if (QE) QE[i * M + j] = (j < i) ? (double)(tau[j + 2] - tau[j + 1]) : 0.0;
    }
  return 0;
}

/* ======================================================================= */
/* Generic sweeps                                                          */
/* ======================================================================= */

typedef struct sweep_tables {
  int M;
  double tau[17], Q[16 * 17], S[16 * 17], QI[256], QE[256];
} sweep_tables;

/* weights addressed with 1-based node indices as in the paper */
#define QW(T, t, j) ((T)->Q[((t) - 1) * ((T)->M + 1) + (j)])
#define SW(T, t, j) ((T)->S[((t) - 1) * ((T)->M + 1) + (j)])
#define QIW(T, t, j) ((T)->QI[((t) - 1) * (T)->M + ((j) - 1)])
#define QEW(T, t, j) ((T)->QE[((t) - 1) * (T)->M + ((j) - 1)])

static double *vec(int n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

static void axpy(int n, double a, const double *x, double *y) {
  for (int i = 0; i < n; ++i) y[i] += a * x[i];
}

/* F^(k) at all nodes */
static void eval_all(const or_problem *p, const double *phi, double *FE, double *FD, double *FR) {
  p->f_expl(p->ctx, phi, FE);
  p->f_diff(p->ctx, phi, FD);
  p->f_reac(p->ctx, phi, FR);
}

/* Right-hand sides at the state x just produced by a reaction step
 * x - wdt F_R(x) = b. F_A and F_D are evaluated at x (S6); the reaction term is
 * the one the implicit equation assigns to x, F_R(x) = (x - b)/wdt (reading:
 * the paper recomputes only the diffusion terms after S5; the reaction term
 * of the new state is the unknown of eq. reaction_step_numerical_methodology).
 * It equals the evaluated rate up to the Newton tolerance and does not
 * amplify the round-off of near-equilibrium fluxes. */
static void eval_after_reaction(const or_problem *p, const double *x, const double *b, double wdt,
                                double *FE, double *FD, double *FR) {
  p->f_expl(p->ctx, x, FE);
  p->f_diff(p->ctx, x, FD);
  for (int i = 0; i < p->n; ++i) FR[i] = (wdt > 0.0) ? (x[i] - b[i]) / wdt : 0.0;
}

/* Delta t * Q^{0:t}(F(phi^(k))) + phi^0  (shared start of every update) */
static void base_rhs(const or_problem *p, const sweep_tables *T, int t, double dt,
                     const double *phi0, double *const *FEk, double *const *FDk,
                     double *const *FRk, double *rhs) {
  int n = p->n, M = T->M;
  memcpy(rhs, phi0, sizeof(double) * n);
  for (int j = 0; j <= M; ++j) {
    double w = dt * QW(T, t, j);
    axpy(n, w, FEk[j], rhs);
    axpy(n, w, FDk[j], rhs);
    axpy(n, w, FRk[j], rhs);
  }
}

/* field-relative max-norm of now - before over nodes 1..M (adaptive rule) */
static double nested_incr(const or_problem *p, int M, double *const *now, double *const *before) {
  const int F = p->n_fields > 0 ? p->n_fields : 1, C = p->n / F;
  double worst = 0.0;
  for (int f = 0; f < F; ++f) {
    double dmax = 0.0, smax = 0.0;
    for (int m = 1; m <= M; ++m)
      for (int c = 0; c < C; ++c) {
        const double a = now[m][(size_t)f * C + c], b = before[m][(size_t)f * C + c];
        dmax = fmax(dmax, fabs(a - b));
        smax = fmax(smax, fabs(a));
      }
    if (smax > 0.0) worst = fmax(worst, dmax / smax);
  }
  return worst;
}

int or_sweep(const or_problem *p, int scheme, int M, int nu, double dt,
             const double *Phi_k, double *Phi_out) {
  return or_sweep_ex(p, scheme, M, nu, NULL, dt, Phi_k, Phi_out, NULL);
}

int or_sweep_ex(const or_problem *p, int scheme, int M, int nu, const or_nu_rule *rule,
                double dt, const double *Phi_k, double *Phi_out, int *nu_used) {
  if (nu_used) *nu_used = 1;
  sweep_tables T;
  T.M = M;
  if (or_lobatto(M, T.tau, T.Q, T.S, T.QI, T.QE)) return 1;
  int n = p->n, rc = 0;
  double *FEk[17] = {0}, *FDk[17] = {0}, *FRk[17] = {0};
  double *cur[17] = {0}, *FEc[17] = {0}, *FDc[17] = {0}, *FRc[17] = {0};
  double *prv[17] = {0}, *FEp[17] = {0}, *FDp[17] = {0}, *FRp[17] = {0};
  double *AD[17] = {0}, *FEad[17] = {0}, *FDad[17] = {0};
  const double *phik[17] = {0};
  for (int m = 0; m <= M; ++m) {
    phik[m] = Phi_k + (size_t)m * n;
    FEk[m] = vec(n); FDk[m] = vec(n); FRk[m] = vec(n);
    cur[m] = vec(n); FEc[m] = vec(n); FDc[m] = vec(n); FRc[m] = vec(n);
    prv[m] = vec(n); FEp[m] = vec(n); FDp[m] = vec(n); FRp[m] = vec(n);
    AD[m] = vec(n); FEad[m] = vec(n); FDad[m] = vec(n);
    eval_all(p, phik[m], FEk[m], FDk[m], FRk[m]);
  }
  const double *phi0 = phik[0];
  double *rhs = vec(n), *b = vec(n);
  memcpy(Phi_out, Phi_k, sizeof(double) * n);   /* node 0 is fixed */

  if (scheme == OR_MISDC) {
    /* eqs. update_equation_misdc_discrete_form_D/R: node-to-node, backward
     * Euler for D and R, forward Euler for A, quadrature S^{m:m+1}. The extra
     * closing bracket in the printed R update is read as a typo. */
    memcpy(cur[0], phi0, sizeof(double) * n);
    memcpy(FEc[0], FEk[0], sizeof(double) * n);
    for (int m = 0; m < M && !rc; ++m) {
      int t = m + 1;
      double dtm = dt * (T.tau[t] - T.tau[m]);
      memcpy(rhs, cur[m], sizeof(double) * n);
      for (int i = 0; i < n; ++i) rhs[i] += dtm * (FEc[m][i] - FEk[m][i]) - dtm * FDk[t][i];
      for (int j = 0; j <= M; ++j) {
        double w = dt * SW(&T, t, j);
        axpy(n, w, FEk[j], rhs); axpy(n, w, FDk[j], rhs); axpy(n, w, FRk[j], rhs);
      }
      rc |= p->solve_diff(p->ctx, dtm, phik[t], rhs, AD[t]);
      for (int i = 0; i < n; ++i) b[i] = AD[t][i] - dtm * FRk[t][i];
      rc |= p->solve_reac(p->ctx, dtm, b, phik[t], cur[t]);
      eval_after_reaction(p, cur[t], b, dtm, FEc[t], FDc[t], FRc[t]);
    }
    for (int m = 1; m <= M; ++m) memcpy(Phi_out + (size_t)m * n, cur[m], sizeof(double) * n);
  } else if (scheme == OR_MISDCQ) {
    /* eqs. update_equation_misdcq_discrete_form_D and _R */
    for (int m = 0; m < M && !rc; ++m) {
      int t = m + 1;
      base_rhs(p, &T, t, dt, phi0, FEk, FDk, FRk, rhs);
      for (int j = 1; j <= m; ++j)
        for (int i = 0; i < n; ++i)
          rhs[i] += dt * QEW(&T, t, j) * (FEc[j][i] - FEk[j][i])
                  + dt * QIW(&T, t, j) * (FDc[j][i] - FDk[j][i]);
      for (int i = 0; i < n; ++i) rhs[i] -= dt * QIW(&T, t, t) * FDk[t][i];
      /* diffusion coefficient frozen at sweep k (there is no nested index) */
      rc |= p->solve_diff(p->ctx, dt * QIW(&T, t, t), phik[t], rhs, AD[t]);
      memcpy(b, AD[t], sizeof(double) * n);
      for (int j = 1; j <= m; ++j)
        for (int i = 0; i < n; ++i) b[i] += dt * QIW(&T, t, j) * (FRc[j][i] - FRk[j][i]);
      for (int i = 0; i < n; ++i) b[i] -= dt * QIW(&T, t, t) * FRk[t][i];
      rc |= p->solve_reac(p->ctx, dt * QIW(&T, t, t), b, phik[t], cur[t]);
      eval_after_reaction(p, cur[t], b, dt * QIW(&T, t, t), FEc[t], FDc[t], FRc[t]);
    }
    for (int m = 1; m <= M; ++m) memcpy(Phi_out + (size_t)m * n, cur[m], sizeof(double) * n);
  } else if (scheme == OR_IMEXQ) {
    /* IMEXQ: explicit A, fully coupled implicit D+R with the LU weights. */
    if (!p->solve_coupled) rc = 1;
    for (int m = 0; m < M && !rc; ++m) {
      int t = m + 1;
      base_rhs(p, &T, t, dt, phi0, FEk, FDk, FRk, rhs);
      for (int j = 1; j <= m; ++j)
        for (int i = 0; i < n; ++i)
          rhs[i] += dt * QEW(&T, t, j) * (FEc[j][i] - FEk[j][i])
                  + dt * QIW(&T, t, j) * (FDc[j][i] + FRc[j][i] - FDk[j][i] - FRk[j][i]);
      for (int i = 0; i < n; ++i) rhs[i] -= dt * QIW(&T, t, t) * (FDk[t][i] + FRk[t][i]);
      rc |= p->solve_coupled(p->ctx, dt * QIW(&T, t, t), rhs, phik[t], cur[t]);
      eval_all(p, cur[t], FEc[t], FDc[t], FRc[t]);
    }
    for (int m = 1; m <= M; ++m) memcpy(Phi_out + (size_t)m * n, cur[m], sizeof(double) * n);
  } else if (scheme == OR_CISDCQ) {
    /* CISDCQ-nu: eqs. update_equation_amisdcq_discrete_form_D and _R_alt.
     * Iteration l = 0 takes its lagged values from initial_lagged_values_A/D/R:
     * F_A and F_D at node m from the newest advection-diffusion state at node m
     * of the current iteration (phi_AD^{m,(k+1,1)}, the reading fixed by the
     * appendix's matrix form), F_R at nodes m and m+1 from sweep k. The lagged
     * diffusion coefficient at node m+1 is that of sweep k when l = 0 and that
     * of iteration l otherwise (eq. lagged_diffusion_flux). The reaction Newton
     * starts from the iteration-l state (Sec. 3.3, S5). */
    for (int m = 0; m <= M; ++m) {   /* iteration l = 0 is sweep k */
      memcpy(prv[m], phik[m], sizeof(double) * n);
      memcpy(FEp[m], FEk[m], sizeof(double) * n);
      memcpy(FDp[m], FDk[m], sizeof(double) * n);
      memcpy(FRp[m], FRk[m], sizeof(double) * n);
    }
    double delta[17] = {0};
    int ran = 0;
    for (int l = 0; l < nu && !rc; ++l) {
      for (int m = 0; m < M && !rc; ++m) {
        int t = m + 1;
        /* ---- diffusion step at node m+1, iteration l+1 ---- */
        base_rhs(p, &T, t, dt, phi0, FEk, FDk, FRk, rhs);
        for (int j = 1; j <= m - 1; ++j)
          for (int i = 0; i < n; ++i)
            rhs[i] += dt * QEW(&T, t, j) * (FEc[j][i] - FEk[j][i])
                    + dt * QIW(&T, t, j) * (FDc[j][i] - FDk[j][i] + FRc[j][i] - FRk[j][i]);
        if (m >= 1) {
          const double *lagE = (l == 0) ? FEad[m] : FEp[m];
          const double *lagD = (l == 0) ? FDad[m] : FDp[m];
          const double *lagR = (l == 0) ? FRk[m] : FRp[m];
          for (int i = 0; i < n; ++i)
            rhs[i] += dt * QEW(&T, t, m) * (lagE[i] - FEk[m][i])
                    + dt * QIW(&T, t, m) * (lagD[i] - FDk[m][i] + lagR[i] - FRk[m][i]);
        }
        const double *lagR1 = (l == 0) ? FRk[t] : FRp[t];
        for (int i = 0; i < n; ++i)
          rhs[i] += dt * QIW(&T, t, t) * (-FDk[t][i] + lagR1[i] - FRk[t][i]);
        const double *coef = (l == 0) ? phik[t] : prv[t];
        rc |= p->solve_diff(p->ctx, dt * QIW(&T, t, t), coef, rhs, AD[t]);
        if (l == 0 && t < M) {   /* S4: lag source for the next node */
          p->f_expl(p->ctx, AD[t], FEad[t]);
          p->f_diff(p->ctx, AD[t], FDad[t]);
        }
        /* ---- reaction step at node m+1, iteration l+1 (R_alt form) ---- */
        memcpy(b, AD[t], sizeof(double) * n);
        if (m >= 1) {
          const double *lagRm = (l == 0) ? FRk[m] : FRp[m];
          for (int i = 0; i < n; ++i) b[i] += dt * QIW(&T, t, m) * (FRc[m][i] - lagRm[i]);
        }
        for (int i = 0; i < n; ++i) b[i] -= dt * QIW(&T, t, t) * lagR1[i];
        const double *guess = (l == 0) ? phik[t] : prv[t];
        rc |= p->solve_reac(p->ctx, dt * QIW(&T, t, t), b, guess, cur[t]);
        /* S6: recompute the right-hand-side terms at the new state */
        eval_after_reaction(p, cur[t], b, dt * QIW(&T, t, t), FEc[t], FDc[t], FRc[t]);
      }
      for (int m = 1; m <= M; ++m) {   /* iteration l+1 becomes the lag source */
        double *s;
        s = prv[m]; prv[m] = cur[m]; cur[m] = s;
        s = FEp[m]; FEp[m] = FEc[m]; FEc[m] = s;
        s = FDp[m]; FDp[m] = FDc[m]; FDc[m] = s;
        s = FRp[m]; FRp[m] = FRc[m]; FRc[m] = s;
      }
      ran = l + 1;
      if (rule && rule->eta > 0.0 && l < 16) {   /* adaptive rule (or_nu_rule) */
        delta[l] = nested_incr(p, M, prv, cur);
        if (l >= 1 && l + 1 < nu &&
            !(delta[l] > rule->eta * delta[0] && delta[l] < rule->rho_stall * delta[l - 1]))
          break;
      }
    }
    if (nu_used) *nu_used = ran;
    /* S7 */
    for (int m = 1; m <= M; ++m) memcpy(Phi_out + (size_t)m * n, prv[m], sizeof(double) * n);
  } else {
    rc = 1;
  }

  for (int m = 0; m <= M; ++m) {
    free(FEk[m]); free(FDk[m]); free(FRk[m]);
    free(cur[m]); free(FEc[m]); free(FDc[m]); free(FRc[m]);
    free(prv[m]); free(FEp[m]); free(FDp[m]); free(FRp[m]);
    free(AD[m]); free(FEad[m]); free(FDad[m]);
  }
  free(rhs); free(b);
  return rc;
}

int or_step(const or_problem *p, int scheme, int M, int n_sweeps, int nu,
            double dt, const double *phi_n, double *phi_out, double *incr) {
  return or_step_ex(p, scheme, M, n_sweeps, nu, NULL, dt, phi_n, phi_out, incr, NULL);
}

int or_step_ex(const or_problem *p, int scheme, int M, int n_sweeps, int nu,
               const or_nu_rule *rule, double dt, const double *phi_n, double *phi_out,
               double *incr, int *nu_used) {
  int n = p->n, rc = 0;
  size_t sz = (size_t)(M + 1) * n;
  double *A = vec((int)sz), *B = vec((int)sz);
  for (int m = 0; m <= M; ++m) memcpy(A + (size_t)m * n, phi_n, sizeof(double) * n);   /* I1, I2 */
  for (int k = 0; k < n_sweeps && !rc; ++k) {
    rc |= or_sweep_ex(p, scheme, M, nu, rule, dt, A, B, nu_used ? nu_used + k : NULL);
    if (incr) {
      double s = 0.0;
      for (int i = 0; i < n; ++i) s += fabs(B[(size_t)M * n + i] - A[(size_t)M * n + i]);
      incr[k] = s / n;
    }
    double *t = A; A = B; B = t;
  }
  memcpy(phi_out, A + (size_t)M * n, sizeof(double) * n);
  free(A); free(B);
  return rc;
}

/* ======================================================================= */
/* Linear model problem (Sec. 4, eq. linear_model_problem)                 */
/* ======================================================================= */

typedef struct lin_ctx { double a, d, r; } lin_ctx;
static void lin_fe(void *c, const double *x, double *o) { o[0] = ((lin_ctx *)c)->a * x[0]; }
static void lin_fd(void *c, const double *x, double *o) { o[0] = ((lin_ctx *)c)->d * x[0]; }
static void lin_fr(void *c, const double *x, double *o) { o[0] = ((lin_ctx *)c)->r * x[0]; }
static int lin_sd(void *c, double w, const double *coef, const double *rhs, double *x) {
  (void)coef; x[0] = rhs[0] / (1.0 - w * ((lin_ctx *)c)->d); return 0;
}
static int lin_sr(void *c, double w, const double *b, const double *g, double *x) {
  (void)g; x[0] = b[0] / (1.0 - w * ((lin_ctx *)c)->r); return 0;
}
static int lin_sc(void *c, double w, const double *rhs, const double *g, double *x) {
  (void)g; lin_ctx *l = (lin_ctx *)c; x[0] = rhs[0] / (1.0 - w * (l->d + l->r)); return 0;
}

static or_problem lin_problem(lin_ctx *c) {
  or_problem p = {1, c, lin_fe, lin_fd, lin_fr, lin_sd, lin_sr, lin_sc};
  return p;
}

int or_linear_step(int scheme, int M, int n_sweeps, int nu, double dt,
                   double a, double d, double r, double phi0,
                   double *phi_out, double *incr) {
  lin_ctx c = {a, d, r};
  or_problem p = lin_problem(&c);
  return or_step(&p, scheme, M, n_sweeps, nu, dt, &phi0, phi_out, incr);
}

int or_linear_step_ex(int scheme, int M, int n_sweeps, int nu, const or_nu_rule *rule,
                      double dt, double a, double d, double r, double phi0,
                      double *phi_out, double *incr, int *nu_used) {
  lin_ctx c = {a, d, r};
  or_problem p = lin_problem(&c);
  return or_step_ex(&p, scheme, M, n_sweeps, nu, rule, dt, &phi0, phi_out, incr, nu_used);
}

int or_linear_G(int scheme, int M, int nu, double dt, double a, double d,
                double r, double *G) {
  /* The sweep is affine in Phi^(k); with phi^0 = 0 it is linear, and its
   * matrix is the iteration matrix G of Sec. 4. */
  lin_ctx c = {a, d, r};
  or_problem p = lin_problem(&c);
  double Pk[17], Po[17];
  for (int j = 1; j <= M; ++j) {
    for (int m = 0; m <= M; ++m) Pk[m] = (m == j) ? 1.0 : 0.0;
    if (or_sweep(&p, scheme, M, nu, dt, Pk, Po)) return 1;
    for (int i = 1; i <= M; ++i) G[(i - 1) * M + (j - 1)] = Po[i];
  }
  return 0;
}

/* ======================================================================= */
/* Dense LU with partial pivoting (shared by the small dense solves)       */
/* ======================================================================= */

/* Solves A x = b in place (A n x n row-major is overwritten). Returns 0, or 1
 * if a pivot is exactly zero. */
static int dense_solve(int n, double *A, double *b) {
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); piv = i; }
    if (best == 0.0) return 1;
    if (piv != k) {
      for (int j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t; }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / A[k * n + k];
      A[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
    b[i] = s / A[i * n + i];
  }
  return 0;
}

/* ======================================================================= */
/* Nonlinear test PDE (Sec. 5.2, eq. nonlinear_test_pde)                   */
/* ======================================================================= */

typedef struct pde_ctx {
  int nx; double dx, a, d, r, left, right;
  double wg[2][2][4];   /* [side][ghost 1/2][phi_b, phi_0, phi_1, phi_2] */
} pde_ctx;

/* Ghost cell averages from the cubic through the boundary value and the
 * first three cell averages (fourth-order Dirichlet closure; the paper does
 * not state its boundary treatment). */
static void pde_ghost_weights(pde_ctx *c) {
  /* p(xi) = sum c_k xi^k, xi in cell widths from the wall into the domain */
  long double A[4][4], inv[4][4];
  for (int k = 0; k < 4; ++k) A[0][k] = (k == 0) ? 1.0L : 0.0L;
  for (int row = 1; row < 4; ++row) {
    long double a0 = row - 1, a1 = row;
    for (int k = 0; k < 4; ++k) A[row][k] = (powl(a1, k + 1) - powl(a0, k + 1)) / (k + 1);
  }
  /* invert 4x4 by Gauss-Jordan */
  long double M[4][8];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 8; ++j) M[i][j] = (j < 4) ? A[i][j] : (j - 4 == i ? 1.0L : 0.0L);
  for (int k = 0; k < 4; ++k) {
    int piv = k;
    for (int i = k + 1; i < 4; ++i) if (fabsl(M[i][k]) > fabsl(M[piv][k])) piv = i;
    for (int j = 0; j < 8; ++j) { long double t = M[k][j]; M[k][j] = M[piv][j]; M[piv][j] = t; }
    long double d = M[k][k];
    for (int j = 0; j < 8; ++j) M[k][j] /= d;
    for (int i = 0; i < 4; ++i) if (i != k) {
      long double f = M[i][k];
      for (int j = 0; j < 8; ++j) M[i][j] -= f * M[k][j];
    }
  }
  for (int i = 0; i < 4; ++i) for (int j = 0; j < 4; ++j) inv[i][j] = M[i][j + 4];
  for (int g = 0; g < 2; ++g) {          /* ghost g covers xi in [-(g+1), -g] */
    long double a0 = -(g + 1), a1 = -g;
    for (int s = 0; s < 4; ++s) {
      long double w = 0.0L;
      for (int k = 0; k < 4; ++k) w += (powl(a1, k + 1) - powl(a0, k + 1)) / (k + 1) * inv[k][s];
      c->wg[0][g][s] = (double)w;
      c->wg[1][g][s] = (double)w;
    }
  }
}

/* extended array e[nx+4], interior at e[2..nx+1] */
static void pde_extend(const pde_ctx *c, const double *x, double *e) {
  int n = c->nx;
  for (int i = 0; i < n; ++i) e[i + 2] = x[i];
  for (int g = 0; g < 2; ++g) {
    const double *w = c->wg[0][g];
    e[1 - g] = w[0] * c->left + w[1] * x[0] + w[2] * x[1] + w[3] * x[2];
    w = c->wg[1][g];
    e[n + 2 + g] = w[0] * c->right + w[1] * x[n - 1] + w[2] * x[n - 2] + w[3] * x[n - 3];
  }
}

static void pde_fe(void *cv, const double *x, double *o) {
  pde_ctx *c = (pde_ctx *)cv;
  int n = c->nx;
  double *e = vec(n + 4);
  pde_extend(c, x, e);
  for (int i = 0; i < n; ++i) {
    int k = i + 2;
    double fr = (7.0 * (e[k] + e[k + 1]) - (e[k - 1] + e[k + 2])) / 12.0;
    double fl = (7.0 * (e[k - 1] + e[k]) - (e[k - 2] + e[k + 1])) / 12.0;
    o[i] = c->a * (fr - fl) / c->dx;
  }
  free(e);
}

static void pde_fd(void *cv, const double *x, double *o) {
  pde_ctx *c = (pde_ctx *)cv;
  int n = c->nx;
  double *e = vec(n + 4);
  pde_extend(c, x, e);
  for (int i = 0; i < n; ++i) {
    int k = i + 2;
    double gr = (15.0 * (e[k + 1] - e[k]) - (e[k + 2] - e[k - 1])) / (12.0 * c->dx);
    double gl = (15.0 * (e[k] - e[k - 1]) - (e[k + 1] - e[k - 2])) / (12.0 * c->dx);
    o[i] = c->d * (gr - gl) / c->dx;
  }
  free(e);
}

static void pde_fr(void *cv, const double *x, double *o) {
  pde_ctx *c = (pde_ctx *)cv;
  for (int i = 0; i < c->nx; ++i) o[i] = c->r * x[i] * (x[i] - 1.0) * (x[i] - 0.5);
}

/* x - w F_D(x) = rhs: F_D is affine, so assemble its matrix column by column
 * and solve directly (the paper solves a banded system directly). */
static int pde_sd(void *cv, double w, const double *coef, const double *rhs, double *x) {
  (void)coef;
  pde_ctx *c = (pde_ctx *)cv;
  int n = c->nx;
  double *A = vec(n * n), *z = vec(n), *f0 = vec(n), *fj = vec(n);
  pde_fd(c, z, f0);
  for (int j = 0; j < n; ++j) {
    z[j] = 1.0;
    pde_fd(c, z, fj);
    z[j] = 0.0;
    for (int i = 0; i < n; ++i) A[i * n + j] = (i == j ? 1.0 : 0.0) - w * (fj[i] - f0[i]);
  }
  for (int i = 0; i < n; ++i) x[i] = rhs[i] + w * f0[i];
  int rc = dense_solve(n, A, x);
  free(A); free(z); free(f0); free(fj);
  return rc;
}

static int pde_sr(void *cv, double w, const double *b, const double *g, double *x) {
  pde_ctx *c = (pde_ctx *)cv;
  for (int i = 0; i < c->nx; ++i) {
    double y = g[i];
    int it;
    for (it = 0; it < 100; ++it) {
      double f = y - w * c->r * y * (y - 1.0) * (y - 0.5) - b[i];
      double df = 1.0 - w * c->r * (3.0 * y * y - 3.0 * y + 0.5);
      double dy = -f / df;
      y += dy;
      if (fabs(dy) <= 1e-15 * (1.0 + fabs(y))) break;
    }
    if (it == 100) return 1;
    x[i] = y;
  }
  return 0;
}

int or_pde_step(int scheme, int M, int n_sweeps, int nu, double dt,
                int nx, double Lx, double a, double d, double r,
                double left, double right, const double *phi_n,
                double *phi_out, double *incr) {
  pde_ctx c;
  memset(&c, 0, sizeof(c));
  c.nx = nx; c.dx = Lx / nx; c.a = a; c.d = d; c.r = r; c.left = left; c.right = right;
  pde_ghost_weights(&c);
  or_problem p = {nx, &c, pde_fe, pde_fd, pde_fr, pde_sd, pde_sr, NULL};
  return or_step(&p, scheme, M, n_sweeps, nu, dt, phi_n, phi_out, incr);
}

/* ======================================================================= */
/* Combustion ADR (Sec. 2 and Sec. 3.3)                                    */
/* ======================================================================= */
/*
 * Model readings (the paper's 1D low-Mach solver is reduced to what the
 * hot path needs):
 *  - constant density rho and a prescribed, discretely divergence-free face
 *    velocity, so the continuity update S2 is trivial and the divergence
 *    constraint / volume-discrepancy correction are not solved;
 *  - state per cell: Y_1..Y_N and mass-specific enthalpy h (formation
 *    enthalpy included); T is diagnosed from sum_i Y_i h_i(T) = h;
 *  - since rho is constant, every F below is d(phi)/dt = (1/rho) times the
 *    right-hand side of eqs. species_equation / enthalpy_equation;
 *  - species diffusivity D_i(T) = D0_i (T/T_ref)^e and thermal diffusivity
 *    lambda/(rho cp) = alpha0 (T/T_ref)^e; face coefficients are harmonic
 *    means; second-order compact diffusion fluxes; fourth-order centred
 *    advective face values;
 *  - dominant species i0: its flux is minus the sum of the others, so after
 *    each diffusion step Y_i0 = 1 - sum_{i != i0} Y_i;
 *  - the differential-diffusion sum of eq. enthalpy_equation is explicit
 *    (weights Q~E), as in step S4, with the i0 flux from the closure;
 *  - mass-action kinetics, k_f = A T^beta exp(-Ea/(R T)), k_r = k_f/K_c,
 *    K_c = exp(-sum_i nu_i g_i/(R T)) (p_ref/(R T))^{sum_i nu_i};
 *  - each implicit diffusion solve ends with the flux-form reconstruction
 *    x := rhs + w F_D[coef](x), which makes every update conservative.
 */

typedef struct adr_ctx {
  const or_mech *m;
  const or_adr_cfg *g;
  int cells, N;
  or_adr_stats *st;
} adr_ctx;

/* thermo (NASA-7, one range) */
static double cp_R(const double *a, double T) {
  return a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
}
static double h_RT(const double *a, double T) {
  return a[0] + a[1] * T / 2.0 + a[2] * T * T / 3.0 + a[3] * T * T * T / 4.0
       + a[4] * T * T * T * T / 5.0 + a[5] / T;
}
static double s_R(const double *a, double T) {
  return a[0] * log(T) + a[1] * T + a[2] * T * T / 2.0 + a[3] * T * T * T / 3.0
       + a[4] * T * T * T * T / 4.0 + a[6];
}

double or_species_h(const or_mech *m, int i, double T) {
  return R_UNIV / m->W[i] * T * h_RT(m->nasa7 + 7 * i, T);
}
double or_species_cp(const or_mech *m, int i, double T) {
  return R_UNIV / m->W[i] * cp_R(m->nasa7 + 7 * i, T);
}
double or_species_s_R(const or_mech *m, int i, double T) {
  return s_R(m->nasa7 + 7 * i, T);
}

static double mix_h(const or_mech *m, const double *Y, int stride, double T) {
  double s = 0.0;
  for (int i = 0; i < m->N; ++i) s += Y[(size_t)i * stride] * or_species_h(m, i, T);
  return s;
}
static double mix_cp(const or_mech *m, const double *Y, int stride, double T) {
  double s = 0.0;
  for (int i = 0; i < m->N; ++i) s += Y[(size_t)i * stride] * or_species_cp(m, i, T);
  return s;
}

/* T from sum_i Y_i h_i(T) = h: Newton safeguarded by bisection on [50, 6000] K,
 * the range on which the one-range polynomials are used (cp > 0 there). */
static int T_of_cell(const or_mech *m, const double *Y, int stride, double h, double *Tout) {
  double lo = 50.0, hi = 6000.0;
  if (mix_h(m, Y, stride, lo) - h > 0.0 || mix_h(m, Y, stride, hi) - h < 0.0) { *Tout = NAN; return 1; }
  double T = 1000.0;
  for (int it = 0; it < 200; ++it) {
    double f = mix_h(m, Y, stride, T) - h;
    if (f > 0.0) hi = T; else lo = T;
    double df = mix_cp(m, Y, stride, T);
    double Tn = T - f / df;
    if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
    double dT = Tn - T;
    T = Tn;
    if (fabs(dT) <= 1e-14 * T) { *Tout = T; return 0; }
  }
  *Tout = T;
  return 0;
}

int or_h_from_T(const or_mech *m, int cells, const double *Y, const double *T, double *h) {
  for (int c = 0; c < cells; ++c) h[c] = mix_h(m, Y + c, cells, T[c]);
  return 0;
}

int or_T_from_h(const or_mech *m, int cells, const double *Y, const double *h, double *T) {
  int bad = 0;
  for (int c = 0; c < cells; ++c) bad |= T_of_cell(m, Y + c, cells, h[c], &T[c]);
  return bad;
}

/* mass-action production rates of one cell */
void or_wdot(const or_mech *m, double rho, const double *Y, double T, double *wdot, double *q) {
  int N = m->N;
  double conc[512];
  for (int i = 0; i < N; ++i) { conc[i] = rho * Y[i] / m->W[i]; wdot[i] = 0.0; }
  for (int r = 0; r < m->R; ++r) {
    const int *nf = m->nu_f + (size_t)r * N, *nr = m->nu_r + (size_t)r * N;
    double kf = m->A[r] * pow(T, m->beta[r]) * exp(-m->Ea[r] / (R_UNIV * T));
    double dg = 0.0, dn = 0.0;
    for (int i = 0; i < N; ++i) {
      int nu = nr[i] - nf[i];
      if (nu) {
        const double *a = m->nasa7 + 7 * i;
        dg += nu * (h_RT(a, T) - s_R(a, T));
        dn += nu;
      }
    }
    double Kc = exp(-dg) * pow(m->p_ref / (R_UNIV * T), dn);
    double kr = kf / Kc;
    double Ff = 1.0, Fr = 1.0;
    for (int i = 0; i < N; ++i) {
      for (int e = 0; e < nf[i]; ++e) Ff *= conc[i];
      for (int e = 0; e < nr[i]; ++e) Fr *= conc[i];
    }
    double qr = kf * Ff - kr * Fr;
    if (q) q[r] = qr;
    for (int i = 0; i < N; ++i) {
      int nu = nr[i] - nf[i];
      if (nu) wdot[i] += m->W[i] * nu * qr;
    }
  }
}

/* d(wdot_i)/d(Y_j, T), analytic; J[N][N+1] */
void or_wdot_jac(const or_mech *m, double rho, const double *Y, double T, double *J) {
  int N = m->N;
  double conc[512];
  for (int i = 0; i < N; ++i) conc[i] = rho * Y[i] / m->W[i];
  memset(J, 0, sizeof(double) * (size_t)N * (N + 1));
  for (int r = 0; r < m->R; ++r) {
    const int *nf = m->nu_f + (size_t)r * N, *nr = m->nu_r + (size_t)r * N;
    double kf = m->A[r] * pow(T, m->beta[r]) * exp(-m->Ea[r] / (R_UNIV * T));
    double dg = 0.0, dn = 0.0, dh = 0.0;
    for (int i = 0; i < N; ++i) {
      int nu = nr[i] - nf[i];
      if (nu) {
        const double *a = m->nasa7 + 7 * i;
        dg += nu * (h_RT(a, T) - s_R(a, T));
        dh += nu * h_RT(a, T);
        dn += nu;
      }
    }
    double Kc = exp(-dg) * pow(m->p_ref / (R_UNIV * T), dn);
    double kr = kf / Kc;
    /* d ln kf/dT = beta/T + Ea/(R T^2);  d ln Kc/dT = sum nu h/(R T^2) - dn/T */
    double dlnkf = m->beta[r] / T + m->Ea[r] / (R_UNIV * T * T);
    double dlnKc = dh / T - dn / T;
    double Ff = 1.0, Fr = 1.0;
    for (int i = 0; i < N; ++i) {
      for (int e = 0; e < nf[i]; ++e) Ff *= conc[i];
      for (int e = 0; e < nr[i]; ++e) Fr *= conc[i];
    }
    double dqdT = kf * dlnkf * Ff - kr * (dlnkf - dlnKc) * Fr;
    double dq[512];
    for (int j = 0; j < N; ++j) {
      /* d(prod_i c_i^{nu_i})/d c_j = nu_j c_j^{nu_j - 1} prod_{i != j} c_i^{nu_i} */
      double dFf = 0.0, dFr = 0.0;
      if (nf[j]) {
        dFf = nf[j];
        for (int e = 0; e < nf[j] - 1; ++e) dFf *= conc[j];
        for (int i = 0; i < N; ++i) if (i != j) for (int e = 0; e < nf[i]; ++e) dFf *= conc[i];
      }
      if (nr[j]) {
        dFr = nr[j];
        for (int e = 0; e < nr[j] - 1; ++e) dFr *= conc[j];
        for (int i = 0; i < N; ++i) if (i != j) for (int e = 0; e < nr[i]; ++e) dFr *= conc[i];
      }
      dq[j] = (kf * dFf - kr * dFr) * rho / m->W[j];
    }
    for (int i = 0; i < N; ++i) {
      int nu = nr[i] - nf[i];
      if (!nu) continue;
      double f = m->W[i] * nu;
      for (int j = 0; j < N; ++j) J[(size_t)i * (N + 1) + j] += f * dq[j];
      J[(size_t)i * (N + 1) + N] += f * dqdT;
    }
  }
}

/* Reaction step S5: rho Y - wdt wdot(Y) = rho b with h fixed; unknowns
 * x = (Y_1..Y_N, T); residual r_Y = Y - wdt wdot/rho - b,
 * r_T = sum Y_i h_i(T) - hstar; plain Newton from the guess with the analytic
 * Jacobian and dense partial-pivot LU. With d = max(max_i |dY_i|, |dT|/T) the
 * size of the applied step, it stops once d <= rtol, or once d <= 1e-8 stops
 * shrinking (d >= d_prev/2): the round-off floor of very stiff cells, where
 * the step can no longer fall below rtol. */
int or_reaction_newton(const or_mech *m, double rho, double wdt, const double *b,
                       double hstar, double *x, double rtol, int maxit) {
  return or_reaction_newton_ex(m, rho, wdt, b, hstar, x, rtol, maxit, NULL);
}

/* The same solve; *floor_stop (if given) is set to 1 when it ended on the
 * round-off-floor test (the last step above rtol), else 0. */
int or_reaction_newton_ex(const or_mech *m, double rho, double wdt, const double *b,
                          double hstar, double *x, double rtol, int maxit, int *floor_stop) {
  int N = m->N, n = N + 1;
  if (floor_stop) *floor_stop = 0;
  double J[64 * 64], Jw[64 * 65], r[64], wd[64];   /* n <= 64 */
  if (n > 64) return -1;
  double dprev = INFINITY;
  for (int it = 1; it <= maxit; ++it) {
    double T = x[N];
    or_wdot(m, rho, x, T, wd, NULL);
    for (int i = 0; i < N; ++i) r[i] = x[i] - wdt * wd[i] / rho - b[i];
    r[N] = mix_h(m, x, 1, T) - hstar;
    or_wdot_jac(m, rho, x, T, Jw);
    for (int i = 0; i < N; ++i)
      for (int j = 0; j <= N; ++j)
        J[i * n + j] = (i == j ? 1.0 : 0.0) - wdt * Jw[i * (N + 1) + j] / rho;
    for (int j = 0; j < N; ++j) J[N * n + j] = or_species_h(m, j, T);
    J[N * n + N] = mix_cp(m, x, 1, T);
    for (int i = 0; i < n; ++i) r[i] = -r[i];
    if (dense_solve(n, J, r)) return -2;
    double dmax = 0.0;
    for (int i = 0; i < N; ++i) { x[i] += r[i]; if (fabs(r[i]) > dmax) dmax = fabs(r[i]); }
    x[N] += r[N];
    if (!(x[N] > 0.0) || !isfinite(x[N])) return -3;
    double d = fabs(r[N]) / x[N];
    if (dmax > d) d = dmax;
    if (!isfinite(d)) return -3;
    if (d <= rtol) return it;
    if (d <= 1e-8 && d >= 0.5 * dprev) {
      if (floor_stop) *floor_stop = 1;
      return it;
    }
    dprev = d;
  }
  return -4;
}

/* periodic neighbour of cell c, offset s along direction d */
static int nbr(const or_adr_cfg *g, int c, int d, int s) {
  int x = c % g->nx, y = (c / g->nx) % g->ny, z = c / (g->nx * g->ny);
  if (d == 0) x = ((x + s) % g->nx + g->nx) % g->nx;
  else if (d == 1) y = ((y + s) % g->ny + g->ny) % g->ny;
  else z = ((z + s) % g->nz + g->nz) % g->nz;
  return x + g->nx * (y + g->ny * z);
}

/* theta(T) = (T/T_ref)^e at cells, harmonic mean at the low face of each cell */
static void face_theta(const or_mech *m, const or_adr_cfg *g, int cells, const double *T, double *thf) {
  double *th = vec(cells);
  for (int c = 0; c < cells; ++c) th[c] = pow(T[c] / m->T_ref, m->theta_exp);
  for (int d = 0; d < g->dim; ++d)
    for (int c = 0; c < cells; ++c) {
      double a = th[nbr(g, c, d, -1)], b = th[c];
      thf[(size_t)d * cells + c] = 2.0 * a * b / (a + b);
    }
  free(th);
}

/* sum_d [thf(c+e)(x(c+e) - x(c)) - thf(c)(x(c) - x(c-e))] */
static double lap_theta(const or_adr_cfg *g, int cells, const double *thf, const double *x, int c) {
  double s = 0.0;
  for (int d = 0; d < g->dim; ++d) {
    int cp = nbr(g, c, d, 1), cm = nbr(g, c, d, -1);
    s += thf[(size_t)d * cells + cp] * (x[cp] - x[c]) - thf[(size_t)d * cells + c] * (x[c] - x[cm]);
  }
  return s;
}

static void adr_T(adr_ctx *a, const double *phi, double *T) {
  if (or_T_from_h(a->m, a->cells, phi, phi + (size_t)a->N * a->cells, T) && a->st) a->st->tdiag_fail++;
}

/* F_E: advection of every field plus explicit differential diffusion of h */
static void adr_fe(void *cv, const double *phi, double *out) {
  adr_ctx *a = (adr_ctx *)cv;
  const or_adr_cfg *g = a->g;
  const or_mech *m = a->m;
  int C = a->cells, N = a->N;
  for (int f = 0; f <= N; ++f) {
    const double *x = phi + (size_t)f * C;
    for (int c = 0; c < C; ++c) {
      double s = 0.0;
      for (int d = 0; d < g->dim; ++d) {
        int cm2 = nbr(g, c, d, -2), cm = nbr(g, c, d, -1), cp = nbr(g, c, d, 1), cp2 = nbr(g, c, d, 2);
        double lo = (7.0 * (x[cm] + x[c]) - (x[cm2] + x[cp])) / 12.0;     /* low face of c  */
        double hi = (7.0 * (x[c] + x[cp]) - (x[cm] + x[cp2])) / 12.0;     /* low face of c+e */
        s += g->vel[(size_t)d * C + cp] * hi - g->vel[(size_t)d * C + c] * lo;
      }
      out[(size_t)f * C + c] = -s / g->dx;
    }
  }
  /* differential diffusion of h: flux/rho at each face
   * q = sum_i hbar_i (Gamma_i/rho + alpha theta dY_i/dx), Gamma_i/rho =
   * -D0_i theta dY_i/dx for i != i0 and minus their sum for i0 */
  double *T = vec(C), *thf = vec(3 * C), *q = vec(3 * C);
  adr_T(a, phi, T);
  face_theta(m, g, C, T, thf);
  for (int d = 0; d < g->dim; ++d)
    for (int c = 0; c < C; ++c) {
      int cm = nbr(g, c, d, -1);
      double th = thf[(size_t)d * C + c];
      double gam_i0 = 0.0, s = 0.0;
      for (int i = 0; i < N; ++i) {
        double dY = (phi[(size_t)i * C + c] - phi[(size_t)i * C + cm]) / g->dx;
        double hbar = 0.5 * (or_species_h(m, i, T[cm]) + or_species_h(m, i, T[c]));
        if (i != g->i0) {
          double gam = -m->D0[i] * th * dY;
          gam_i0 -= gam;
          s += hbar * (gam + m->alpha0 * th * dY);
        } else {
          s += hbar * m->alpha0 * th * dY;
        }
      }
      {
        int i = g->i0;
        double hbar = 0.5 * (or_species_h(m, i, T[cm]) + or_species_h(m, i, T[c]));
        s += hbar * gam_i0;
      }
      q[(size_t)d * C + c] = s;
    }
  for (int c = 0; c < C; ++c) {
    double s = 0.0;
    for (int d = 0; d < g->dim; ++d) s += q[(size_t)d * C + nbr(g, c, d, 1)] - q[(size_t)d * C + c];
    out[(size_t)N * C + c] += -s / g->dx;
  }
  free(T); free(thf); free(q);
}

/* F_D with the state's own coefficients */
static void adr_fd(void *cv, const double *phi, double *out) {
  adr_ctx *a = (adr_ctx *)cv;
  const or_adr_cfg *g = a->g;
  const or_mech *m = a->m;
  int C = a->cells, N = a->N;
  double *T = vec(C), *thf = vec(3 * C);
  adr_T(a, phi, T);
  face_theta(m, g, C, T, thf);
  double inv = 1.0 / (g->dx * g->dx);
  for (int c = 0; c < C; ++c) out[(size_t)g->i0 * C + c] = 0.0;
  for (int f = 0; f <= N; ++f) {
    if (f == g->i0) continue;
    double k = (f < N) ? m->D0[f] : m->alpha0;
    for (int c = 0; c < C; ++c) {
      double v = k * inv * lap_theta(g, C, thf, phi + (size_t)f * C, c);
      out[(size_t)f * C + c] = v;
      if (f < N) out[(size_t)g->i0 * C + c] -= v;
    }
  }
  free(T); free(thf);
}

static void adr_fr(void *cv, const double *phi, double *out) {
  adr_ctx *a = (adr_ctx *)cv;
  int C = a->cells, N = a->N;
  double *T = vec(C);
  double Y[512], wd[512];
  adr_T(a, phi, T);
  for (int c = 0; c < C; ++c) {
    for (int i = 0; i < N; ++i) Y[i] = phi[(size_t)i * C + c];
    or_wdot(a->m, a->g->rho, Y, T[c], wd, NULL);
    for (int i = 0; i < N; ++i) out[(size_t)i * C + c] = wd[i] / a->g->rho;
    out[(size_t)N * C + c] = 0.0;
  }
  free(T);
}

/* conjugate gradients on (I - cw L_theta) x = rhs (symmetric positive definite) */
static int cg_solve(adr_ctx *a, const double *thf, double cw, const double *rhs, double *x) {
  const or_adr_cfg *g = a->g;
  int C = a->cells;
  double *r = vec(C), *p = vec(C), *Ap = vec(C);
  double bn = 0.0, rr = 0.0;
  memcpy(x, rhs, sizeof(double) * C);
  for (int c = 0; c < C; ++c) {
    r[c] = rhs[c] - (x[c] - cw * lap_theta(g, C, thf, x, c));
    p[c] = r[c];
    rr += r[c] * r[c];
    bn += rhs[c] * rhs[c];
  }
  int it, rc = 1;
  double tol2 = g->lin_rtol * g->lin_rtol * bn;
  for (it = 0; it < g->lin_maxit; ++it) {
    if (rr <= tol2) { rc = 0; break; }
    double pAp = 0.0;
    for (int c = 0; c < C; ++c) { Ap[c] = p[c] - cw * lap_theta(g, C, thf, p, c); pAp += p[c] * Ap[c]; }
    double al = rr / pAp, rn = 0.0;
    for (int c = 0; c < C; ++c) { x[c] += al * p[c]; r[c] -= al * Ap[c]; rn += r[c] * r[c]; }
    double be = rn / rr;
    rr = rn;
    for (int c = 0; c < C; ++c) p[c] = r[c] + be * p[c];
  }
  if (a->st) { a->st->lin_solves++; a->st->lin_iters += it; if (rc) a->st->lin_fail++; }
  free(r); free(p); free(Ap);
  return rc;
}

/* D-step solve for every field but i0, flux-form reconstruction, closure */
static int adr_sd(void *cv, double wdt, const double *coef, const double *rhs, double *x) {
  adr_ctx *a = (adr_ctx *)cv;
  const or_adr_cfg *g = a->g;
  const or_mech *m = a->m;
  int C = a->cells, N = a->N, rc = 0;
  double *T = vec(C), *thf = vec(3 * C), *y = vec(C);
  adr_T(a, coef, T);
  face_theta(m, g, C, T, thf);
  double inv = 1.0 / (g->dx * g->dx);
  for (int f = 0; f <= N; ++f) {
    if (f == g->i0) continue;
    double cw = wdt * ((f < N) ? m->D0[f] : m->alpha0) * inv;
    const double *b = rhs + (size_t)f * C;
    rc |= cg_solve(a, thf, cw, b, y);
    for (int c = 0; c < C; ++c) x[(size_t)f * C + c] = b[c] + cw * lap_theta(g, C, thf, y, c);
  }
  for (int c = 0; c < C; ++c) {
    double s = 0.0;
    for (int i = 0; i < N; ++i) if (i != g->i0) s += x[(size_t)i * C + c];
    x[(size_t)g->i0 * C + c] = 1.0 - s;
  }
  free(T); free(thf); free(y);
  return rc;
}

static int adr_sr(void *cv, double wdt, const double *b, const double *guess, double *x) {
  adr_ctx *a = (adr_ctx *)cv;
  const or_adr_cfg *g = a->g;
  int C = a->cells, N = a->N, rc = 0;
  double *Tg = vec(C);
  adr_T(a, guess, Tg);
  double xx[512], bb[512];
  for (int c = 0; c < C; ++c) {
    for (int i = 0; i < N; ++i) { xx[i] = guess[(size_t)i * C + c]; bb[i] = b[(size_t)i * C + c]; }
    xx[N] = Tg[c];
    double hstar = b[(size_t)N * C + c];
    int floor_stop = 0;
    int it = or_reaction_newton_ex(a->m, g->rho, wdt, bb, hstar, xx, g->newton_rtol, g->newton_maxit,
                                   &floor_stop);
    if (a->st) {
      a->st->newton_solves++;
      a->st->newton_floor += floor_stop;
      if (it > 0) { a->st->newton_iters += it; if (it > a->st->newton_maxit_seen) a->st->newton_maxit_seen = it; }
      else a->st->newton_fail++;
    }
    if (it <= 0) rc = 1;
    for (int i = 0; i < N; ++i) x[(size_t)i * C + c] = xx[i];
    x[(size_t)N * C + c] = hstar;
  }
  free(Tg);
  return rc;
}

int or_adr_step(const or_mech *mech, const or_adr_cfg *cfg, int scheme, int M,
                int n_sweeps, int nu, double dt, const double *phi_n,
                double *phi_out, double *incr, or_adr_stats *stats) {
  return or_adr_step_ex(mech, cfg, scheme, M, n_sweeps, nu, NULL, dt, phi_n, phi_out, incr,
                        NULL, stats);
}

int or_adr_step_ex(const or_mech *mech, const or_adr_cfg *cfg, int scheme, int M,
                   int n_sweeps, int nu, const or_nu_rule *rule, double dt,
                   const double *phi_n, double *phi_out, double *incr, int *nu_used,
                   or_adr_stats *stats) {
  adr_ctx a = {mech, cfg, cfg->nx * cfg->ny * cfg->nz, mech->N, stats};
  or_problem p = {(mech->N + 1) * a.cells, &a, adr_fe, adr_fd, adr_fr, adr_sd, adr_sr, NULL,
                  mech->N + 1};
  return or_step_ex(&p, scheme, M, n_sweeps, nu, rule, dt, phi_n, phi_out, incr, nu_used);
}

int or_adr_operators(const or_mech *mech, const or_adr_cfg *cfg, const double *phi,
                     double *FE, double *FD, double *FR) {
  adr_ctx a = {mech, cfg, cfg->nx * cfg->ny * cfg->nz, mech->N, NULL};
  if (FE) adr_fe(&a, phi, FE);
  if (FD) adr_fd(&a, phi, FD);
  if (FR) adr_fr(&a, phi, FR);
  return 0;
}

int or_adr_solve_diff(const or_mech *mech, const or_adr_cfg *cfg, double wdt,
                      const double *coef_state, const double *rhs, double *x) {
  adr_ctx a = {mech, cfg, cfg->nx * cfg->ny * cfg->nz, mech->N, NULL};
  return adr_sd(&a, wdt, coef_state, rhs, x);
}

/* ======================================================================= */
/* Variable-density low-Mach coupling in 1D (Sec. 2; Sec. 3.3 I3, I4, S2, S6) */
/* ======================================================================= */
/*
 * The paper's own setting (1D, open boundaries): the state is conservative,
 * [rho, rho Y_1..rho Y_N, rho h] per cell; the velocity lives on the faces and
 * follows from the divergence constraint div U = S + delta_chi (eqs.
 * divergence_constraint, S_def) integrated from the inflow face, as the paper
 * does in 1D (I4). Readings (the paper states none of these closures):
 *  - inflow at x = 0: Dirichlet state (Y_in, T_in, rho_in from the EOS at p0)
 *    and velocity U_in; outflow at x = L: zero gradient, no diffusive flux;
 *  - advection: fourth-order centred face values of the conserved quantity,
 *    the inflow value on the inflow face and as the ghost of the first face,
 *    the last cell's value on and beyond the outflow face;
 *  - diffusion: second-order compact fluxes with harmonic-mean coefficients;
 *    on the inflow face the gradient to the inflow value half a cell away;
 *  - the dominant species' flux is minus the sum of the others (Sec. 2);
 *  - in eq. S_def the flux Gamma_i enters as rho D_i grad Y_i: deriving S from
 *    the EOS held at p0 along particle paths (D/Dt ln p_EOS = 0 with the
 *    species and enthalpy equations) gives
 *      S = (div(lambda grad T) + sum_i rho D_i grad Y_i . grad h_i) / (rho cp T)
 *          + sum_i (W/W_i) div(rho D_i grad Y_i) / rho
 *          + sum_i (W/W_i - h_i/(cp T)) wdot_i / rho,
 *    whereas the text's Gamma_i := -rho D_i grad Y_i would reverse the sign of
 *    the diffusive expansion;
 *  - lambda/cp = rho alpha(T) (the same transport model as the periodic ADR
 *    system), so lambda = rho cp alpha(T); the differential-diffusion flux
 *    sum_i h_i (rho D_i - lambda/cp) grad Y_i uses face means of h_i.
 */

typedef struct lm_ctx {
  const or_mech *m;
  const or_lm_cfg *g;
  int nx, N;
  double rho_in, h_in, T_in;
  double hsp_in[64];   /* species enthalpies at the inflow state, J/kg */
} lm_ctx;

static void lm_setup(lm_ctx *c, const or_mech *m, const or_lm_cfg *g) {
  c->m = m; c->g = g; c->nx = g->nx; c->N = m->N;
  double sw = 0.0;
  for (int i = 0; i < m->N; ++i) sw += g->Y_in[i] / m->W[i];
  c->T_in = g->T_in;
  c->rho_in = g->p0 / (R_UNIV * g->T_in * sw);
  c->h_in = mix_h(m, g->Y_in, 1, g->T_in);
  for (int i = 0; i < m->N; ++i) c->hsp_in[i] = or_species_h(m, i, g->T_in);
}

static double lm_theta(const or_mech *m, double T) { return pow(T / m->T_ref, m->theta_exp); }

/* primitive variables of every cell: Y [N][nx], h, T [nx]; returns non-zero if a
 * temperature cannot be diagnosed */
static int lm_prims(const lm_ctx *c, const double *q, double *Y, double *h, double *T,
                    const double *Tguess) {
  const int nx = c->nx, N = c->N;
  int rc = 0;
  for (int k = 0; k < nx; ++k) {
    const double rho = q[k];
    for (int i = 0; i < N; ++i) Y[(size_t)i * nx + k] = q[(size_t)(1 + i) * nx + k] / rho;
    h[k] = q[(size_t)(N + 1) * nx + k] / rho;
    (void)Tguess;
    rc |= T_of_cell(c->m, Y + k, nx, h[k], &T[k]);
  }
  return rc;
}

/* 12 x the fourth-order face value of field f on face j (j = 1..nx-1), with the
 * inflow ghost and zero-gradient outflow ghosts */
static double lm_face4(const lm_ctx *c, const double *f, double fin, int j) {
  const int nx = c->nx;
  const double a = (j - 2 >= 0) ? f[j - 2] : fin;
  const double b = f[j - 1], d = f[j];
  const double e = (j + 1 < nx) ? f[j + 1] : f[nx - 1];
  return 7.0 * (b + d) - (a + e);
}

/* A = -div(U f) for a conserved field f with inflow value fin */
static void lm_advect(const lm_ctx *c, const double *U, const double *f, double fin, double *out) {
  const int nx = c->nx;
  const double inv = 1.0 / c->g->dx;
  double Fl = U[0] * fin;
  for (int k = 0; k < nx; ++k) {
    const double Fr = (k + 1 < nx) ? U[k + 1] * lm_face4(c, f, fin, k + 1) / 12.0 : U[nx] * f[nx - 1];
    out[k] = -(Fr - Fl) * inv;
    Fl = Fr;
  }
}

/* diffusive fluxes on the nx+1 faces: G[i][j] = rho D_i grad Y_i (dominant
 * species closed), Q[j] = (lambda/cp) grad h, K[j] = lambda grad T,
 * gY[i][j] = grad Y_i and the face species enthalpies hf[i][j] */
typedef struct lm_faces {
  double *G, *Q, *K, *gY, *hf, *Lc, *gh;   /* Lc: lambda/cp; gh[i][j]: grad h_i */
} lm_faces;

static void lm_fluxes(const lm_ctx *c, const double *rho, const double *Y, const double *h,
                      const double *T, const double *hsp, lm_faces *F) {
  const or_mech *m = c->m;
  const int nx = c->nx, N = c->N, i0 = c->g->i0;
  const double dx = c->g->dx;
  for (int j = 0; j <= nx; ++j) {
    const int l = j - 1, r = j;
    double dist, th_l, th_r, rho_l, rho_r, cp_l, cp_r, T_l, T_r, h_l, h_r;
    if (j == nx) {   /* outflow: no diffusive flux */
      for (int i = 0; i < N; ++i) {
        F->G[(size_t)i * (nx + 1) + j] = 0.0;
        F->gY[(size_t)i * (nx + 1) + j] = 0.0;
        F->hf[(size_t)i * (nx + 1) + j] = hsp[(size_t)i * nx + nx - 1];
      }
      F->Q[j] = 0.0;
      F->K[j] = 0.0;
      F->Lc[j] = 0.0;
      for (int i = 0; i < N; ++i) F->gh[(size_t)i * (nx + 1) + j] = 0.0;
      continue;
    }
    if (j == 0) {    /* inflow: the boundary state half a cell away */
      dist = 0.5 * dx;
      rho_l = c->rho_in; T_l = c->T_in; h_l = c->h_in;
      cp_l = mix_cp(m, c->g->Y_in, 1, c->T_in);
    } else {
      dist = dx;
      rho_l = rho[l]; T_l = T[l]; h_l = h[l];
      cp_l = mix_cp(m, Y + l, nx, T[l]);
    }
    rho_r = rho[r]; T_r = T[r]; h_r = h[r];
    cp_r = mix_cp(m, Y + r, nx, T[r]);
    th_l = lm_theta(m, T_l);
    th_r = lm_theta(m, T_r);
    /* on the inflow face the coefficients are those of the first cell */
    const double a_l = (j == 0) ? rho_r * th_r : rho_l * th_l, a_r = rho_r * th_r;
    const double hm = 2.0 * a_l * a_r / (a_l + a_r);   /* (rho theta) at the face */
    const double lam_l = (j == 0) ? rho_r * cp_r * m->alpha0 * th_r : rho_l * cp_l * m->alpha0 * th_l;
    const double lam_r = rho_r * cp_r * m->alpha0 * th_r;
    F->Lc[j] = m->alpha0 * hm;
    F->Q[j] = F->Lc[j] * (h_r - h_l) / dist;
    F->K[j] = (2.0 * lam_l * lam_r / (lam_l + lam_r)) * (T_r - T_l) / dist;
    double sum = 0.0;
    for (int i = 0; i < N; ++i) {
      const double yl = (j == 0) ? c->g->Y_in[i] : Y[(size_t)i * nx + l];
      const double yr = Y[(size_t)i * nx + r];
      const double g = (yr - yl) / dist;
      F->gY[(size_t)i * (nx + 1) + j] = g;
      const double hl = (j == 0) ? c->hsp_in[i] : hsp[(size_t)i * nx + l];
      F->hf[(size_t)i * (nx + 1) + j] = 0.5 * (hl + hsp[(size_t)i * nx + r]);
      F->gh[(size_t)i * (nx + 1) + j] = (hsp[(size_t)i * nx + r] - hl) / dist;
      if (i == i0) continue;
      const double v = m->D0[i] * hm * g;
      F->G[(size_t)i * (nx + 1) + j] = v;
      sum += v;
    }
    F->G[(size_t)i0 * (nx + 1) + j] = -sum;
  }
}

/* Right-hand sides, S, velocity and thermodynamic pressure of a state
 * q = [rho, rho Y_1..rho Y_N, rho h] ([N+2][nx]):
 *  FA = explicit part: -div(U q) for every row, plus the differential
 *       diffusion of h (eq. enthalpy_equation, explicit as in S4);
 *  FD = implicit diffusion: div(rho D_i grad Y_i) for the species rows,
 *       div(lambda/cp grad h) for h, 0 for rho;
 *  FR = reaction: wdot_i for the species rows, 0 for rho and h;
 *  S [nx] (eq. S_def), U [nx+1] from div U = S + dchi with U_0 = U_in (I4, S6;
 *  dchi may be NULL), peos [nx] (eq. p_eos_definition), T [nx] in/out (guess). */
int or_lm_terms(const or_mech *m, const or_lm_cfg *g, const double *q, const double *dchi,
                const double *Uadv, double *FA, double *FD, double *FR, double *S, double *U,
                double *peos, double *T) {
  lm_ctx c;
  lm_setup(&c, m, g);
  const int nx = g->nx, N = m->N, F = N + 2;
  const double dx = g->dx, inv = 1.0 / dx;
  double *Y = vec(N * nx), *h = vec(nx), *hsp = vec(N * nx), *wd = vec(N);
  double *Yc = vec(N);
  lm_faces Fc;
  Fc.G = vec(N * (nx + 1)); Fc.gY = vec(N * (nx + 1)); Fc.hf = vec(N * (nx + 1));
  Fc.gh = vec(N * (nx + 1)); Fc.Q = vec(nx + 1); Fc.K = vec(nx + 1); Fc.Lc = vec(nx + 1);
  int rc = lm_prims(&c, q, Y, h, T, T);
  for (int k = 0; k < nx; ++k)
    for (int i = 0; i < N; ++i) hsp[(size_t)i * nx + k] = or_species_h(m, i, T[k]);
  lm_fluxes(&c, q, Y, h, T, hsp, &Fc);
  /* diffusion, reaction and S per cell */
  for (int k = 0; k < nx; ++k) {
    const double rho = q[k];
    for (int i = 0; i < N; ++i) Yc[i] = Y[(size_t)i * nx + k];
    or_wdot(m, rho, Yc, T[k], wd, NULL);
    double sw = 0.0;
    for (int i = 0; i < N; ++i) sw += Yc[i] / m->W[i];
    const double Wmix = 1.0 / sw, cp = mix_cp(m, Yc, 1, T[k]);
    double s2 = 0.0, s3 = 0.0, ghl = 0.0, ghr = 0.0;
    for (int i = 0; i < N; ++i) {
      const double dY = (Fc.G[(size_t)i * (nx + 1) + k + 1] - Fc.G[(size_t)i * (nx + 1) + k]) * inv;
      if (FD) FD[(size_t)(1 + i) * nx + k] = dY;
      if (FR) FR[(size_t)(1 + i) * nx + k] = wd[i];
      s2 += Wmix / m->W[i] * dY;
      s3 += (Wmix / m->W[i] - hsp[(size_t)i * nx + k] / (cp * T[k])) * wd[i];
      ghl += Fc.G[(size_t)i * (nx + 1) + k] * Fc.gh[(size_t)i * (nx + 1) + k];
      ghr += Fc.G[(size_t)i * (nx + 1) + k + 1] * Fc.gh[(size_t)i * (nx + 1) + k + 1];
    }
    if (FD) {
      FD[k] = 0.0;
      FD[(size_t)(N + 1) * nx + k] = (Fc.Q[k + 1] - Fc.Q[k]) * inv;
    }
    if (FR) { FR[k] = 0.0; FR[(size_t)(N + 1) * nx + k] = 0.0; }
    const double divK = (Fc.K[k + 1] - Fc.K[k]) * inv;
    S[k] = (divK + 0.5 * (ghl + ghr)) / (rho * cp * T[k]) + s2 / rho + s3 / rho;
    if (peos) peos[k] = rho * R_UNIV * T[k] * sw;
  }
  U[0] = g->U_in;
  for (int k = 0; k < nx; ++k) U[k + 1] = U[k] + dx * (S[k] + (dchi ? dchi[k] : 0.0));
  /* advection with the given face velocity (or the one just computed) and the
   * explicit differential diffusion of h */
  if (FA) {
    const double *Ua = Uadv ? Uadv : U;
    lm_advect(&c, Ua, q, c.rho_in, FA);
    for (int i = 0; i < N; ++i)
      lm_advect(&c, Ua, q + (size_t)(1 + i) * nx, c.rho_in * g->Y_in[i], FA + (size_t)(1 + i) * nx);
    lm_advect(&c, Ua, q + (size_t)(N + 1) * nx, c.rho_in * c.h_in, FA + (size_t)(N + 1) * nx);
    for (int k = 0; k < nx; ++k) {
      double fl = 0.0, fr = 0.0;
      for (int i = 0; i < N; ++i) {
        const size_t a = (size_t)i * (nx + 1) + k, b = a + 1;
        fl += Fc.hf[a] * (Fc.G[a] - Fc.Lc[k] * Fc.gY[a]);
        fr += Fc.hf[b] * (Fc.G[b] - Fc.Lc[k + 1] * Fc.gY[b]);
      }
      FA[(size_t)(N + 1) * nx + k] += (fr - fl) * inv;
    }
  }
  (void)F;
  free(Y); free(h); free(hsp); free(wd); free(Yc);
  free(Fc.G); free(Fc.gY); free(Fc.hf); free(Fc.gh); free(Fc.Q); free(Fc.K); free(Fc.Lc);
  return rc;
}

/* (rho theta) on the faces of a state (the diffusion coefficient without its
 * per-field factor D0_i or alpha0): harmonic means inside, the first cell's value
 * on the inflow face, 0 on the outflow face (no diffusive flux) */
static void lm_face_coef(const lm_ctx *c, const double *rho, const double *T, double *hm) {
  const int nx = c->nx;
  for (int j = 0; j <= nx; ++j) {
    if (j == nx) { hm[j] = 0.0; continue; }
    const double ar = rho[j] * lm_theta(c->m, T[j]);
    if (j == 0) { hm[j] = ar; continue; }
    const double al = rho[j - 1] * lm_theta(c->m, T[j - 1]);
    hm[j] = 2.0 * al * ar / (al + ar);
  }
}

/* rho_new x - w div(k grad x) = rhs on the open domain (inflow value xin on the
 * inflow face, half a cell away; no flux through the outflow face), k = f0 hm;
 * dense direct solve, then the flux-form reconstruction
 * rho_new x := rhs + w div(k grad x) (returned in out, conserved exactly) */
static int lm_solve_diff(const lm_ctx *c, double w, double f0, const double *hm, const double *rho_new,
                         const double *rhs, double xin, double *x, double *out) {
  const int nx = c->nx;
  const double dx = c->g->dx;
  double *A = vec(nx * nx);
  for (int k = 0; k < nx; ++k) {
    const double kl = f0 * hm[k] / ((k == 0 ? 0.5 : 1.0) * dx * dx);
    const double kr = f0 * hm[k + 1] / (dx * dx);
    A[k * nx + k] = rho_new[k] + w * (kl + kr);
    if (k > 0) A[k * nx + k - 1] = -w * kl;
    if (k + 1 < nx) A[k * nx + k + 1] = -w * kr;
    x[k] = rhs[k] + (k == 0 ? w * kl * xin : 0.0);
  }
  int rc = dense_solve(nx, A, x);
  free(A);
  for (int k = 0; k < nx; ++k) {
    const double fl = f0 * hm[k] * (x[k] - (k == 0 ? xin : x[k - 1])) / ((k == 0 ? 0.5 : 1.0) * dx);
    const double fr = (k + 1 < nx) ? f0 * hm[k + 1] * (x[k + 1] - x[k]) / dx : 0.0;
    out[k] = rhs[k] + w * (fr - fl) / dx;
  }
  return rc;
}

/* One time step of CISDCQ-nu (eqs. update_equation_amisdcq_discrete_form_D and
 * _R_alt, I1-I4, S1-S7) on the low-Mach system: per node, S2 (the density row of
 * the D update, advection only), S3 and S4 (species and enthalpy diffusion solved
 * against the new density with coefficients lagged as in eq.
 * lagged_diffusion_flux; the differential diffusion explicit), S5 (reaction
 * Newton at the new density, enthalpy fixed), S6 (delta_chi increment and the
 * velocity from div U = S + delta_chi). Readings beyond the periodic scheme's:
 * the lag source of iteration 0 at node m is the node's advection-diffusion
 * state with the velocity of its own S and the current delta_chi; delta_chi of
 * a sweep starts from the previous sweep's (as S6 writes it).
 * q_n, q_out: [N+2][nx]; incr[k] (may be NULL): max over cells of
 * |rho h^{M,(k+1)} - rho h^{M,(k)}| / max |rho h^{M,(k+1)}|; peos_out [nx] (may
 * be NULL): p_EOS of the result. */
int or_lm_step(const or_mech *m, const or_lm_cfg *g, int M, int n_sweeps, int nu, double dt,
               const double *q_n, double *q_out, double *incr, double *peos_out) {
  return or_lm_step_ex(m, g, OR_CISDCQ, M, n_sweeps, nu, dt, q_n, q_out, incr, peos_out);
}

/* scheme OR_CISDCQ as above, or OR_MISDCQ: the serial sweep of eqs.
 * update_equation_misdcq_discrete_form_D/_R on the same system (one pass per
 * sweep, nu ignored), whose D update takes the new values of nodes 1..m and no
 * reaction correction, and whose R update corrects the reaction terms of nodes
 * 1..m+1 */
int or_lm_step_ex(const or_mech *m, const or_lm_cfg *g, int scheme, int M, int n_sweeps, int nu,
                  double dt, const double *q_n, double *q_out, double *incr, double *peos_out) {
  if (scheme != OR_CISDCQ && scheme != OR_MISDCQ) return 1;
  if (scheme == OR_MISDCQ) nu = 1;
  sweep_tables Tb;
  Tb.M = M;
  if (or_lobatto(M, Tb.tau, Tb.Q, Tb.S, Tb.QI, Tb.QE)) return 1;
  lm_ctx c;
  lm_setup(&c, m, g);
  const int nx = g->nx, N = m->N, F = N + 2, n = F * nx, i0 = g->i0;
  int rc = 0;
  enum { KS = 0, XS = 1, CS = 2 };   /* sweep k, iteration l, iteration l+1 */
  double *q[3][17], *FA[3][17], *FD[3][17], *FR[3][17], *Tn[3][17], *dch[3][17];
  for (int s = 0; s < 3; ++s)
    for (int j = 0; j <= M; ++j) {
      q[s][j] = vec(n); FA[s][j] = vec(n); FD[s][j] = vec(n); FR[s][j] = vec(n);
      Tn[s][j] = vec(nx); dch[s][j] = vec(nx);
    }
  double *qad = vec(n), *lagA = vec(n), *lagD = vec(n), *rhs = vec(n), *b = vec(n);
  double *S = vec(nx), *U = vec(nx + 1), *pe = vec(nx), *Tad = vec(nx), *hm = vec(nx + 1);
  double *xs = vec(nx), *ys = vec(nx), *Yc = vec(N + 1), *bc = vec(N);
  /* I1, I2, I4: every node holds q^n, its terms and the velocity of S^n */
  for (int k = 0; k < nx; ++k) Tn[KS][0][k] = 1000.0;
  rc |= or_lm_terms(m, g, q_n, NULL, NULL, FA[KS][0], FD[KS][0], FR[KS][0], S, U, pe, Tn[KS][0]);
  for (int s = 0; s < 3; ++s)   /* node 0 is fixed: the same in every set */
    for (int j = 0; j <= M; ++j) {
      if (s != KS && j != 0) continue;
      memcpy(q[s][j], q_n, sizeof(double) * n);
      if (s == KS && j == 0) continue;
      memcpy(FA[s][j], FA[KS][0], sizeof(double) * n);
      memcpy(FD[s][j], FD[KS][0], sizeof(double) * n);
      memcpy(FR[s][j], FR[KS][0], sizeof(double) * n);
      memcpy(Tn[s][j], Tn[KS][0], sizeof(double) * nx);
    }
  int sK = KS, sX = XS, sC = CS;
  for (int kk = 0; kk < n_sweeps && !rc; ++kk) {
    for (int l = 0; l < nu && !rc; ++l) {
      for (int mm = 0; mm < M && !rc; ++mm) {
        const int t = mm + 1;
        const double w = dt * QIW(&Tb, t, t), dtm = dt * (Tb.tau[t] - Tb.tau[mm]);
        /* right-hand side of the D update (generic CISDCQ form on q) */
        memcpy(rhs, q_n, sizeof(double) * n);
        for (int j = 0; j <= M; ++j) {
          const double qw = dt * QW(&Tb, t, j);
          axpy(n, qw, FA[sK][j], rhs); axpy(n, qw, FD[sK][j], rhs); axpy(n, qw, FR[sK][j], rhs);
        }
        if (scheme == OR_MISDCQ) {
          for (int j = 1; j <= mm; ++j)
            for (int i = 0; i < n; ++i)
              rhs[i] += dt * QEW(&Tb, t, j) * (FA[sC][j][i] - FA[sK][j][i]) +
                        dt * QIW(&Tb, t, j) * (FD[sC][j][i] - FD[sK][j][i]);
          for (int i = 0; i < n; ++i) rhs[i] -= w * FD[sK][t][i];
        }
        for (int j = 1; j <= mm - 1 && scheme == OR_CISDCQ; ++j)
          for (int i = 0; i < n; ++i)
            rhs[i] += dt * QEW(&Tb, t, j) * (FA[sC][j][i] - FA[sK][j][i]) +
                      dt * QIW(&Tb, t, j) * (FD[sC][j][i] - FD[sK][j][i] + FR[sC][j][i] - FR[sK][j][i]);
        const double *lA = NULL, *lD = NULL, *lRm = NULL;
        if (mm >= 1 && scheme == OR_CISDCQ) {
          lA = (l == 0) ? lagA : FA[sX][mm];
          lD = (l == 0) ? lagD : FD[sX][mm];
          lRm = (l == 0) ? FR[sK][mm] : FR[sX][mm];
          for (int i = 0; i < n; ++i)
            rhs[i] += dt * QEW(&Tb, t, mm) * (lA[i] - FA[sK][mm][i]) +
                      dt * QIW(&Tb, t, mm) * (lD[i] - FD[sK][mm][i] + lRm[i] - FR[sK][mm][i]);
        }
        const double *lRt = (l == 0) ? FR[sK][t] : FR[sX][t];
        if (scheme == OR_CISDCQ)
          for (int i = 0; i < n; ++i) rhs[i] += w * (-FD[sK][t][i] + lRt[i] - FR[sK][t][i]);
        /* S2: the density row has no diffusion or reaction */
        memcpy(qad, rhs, sizeof(double) * nx);
        /* S3, S4: diffusion against rho_new, coefficients lagged (eq.
         * lagged_diffusion_flux: sweep k at l = 0, iteration l otherwise) */
        const double *qc = (l == 0) ? q[sK][t] : q[sX][t];
        const double *Tc = (l == 0) ? Tn[sK][t] : Tn[sX][t];
        lm_face_coef(&c, qc, Tc, hm);
        double *rhoY0 = qad + (size_t)(1 + i0) * nx;
        for (int k = 0; k < nx; ++k) rhoY0[k] = qad[k];
        for (int i = 0; i < N; ++i) {
          if (i == i0) continue;
          rc |= lm_solve_diff(&c, w, m->D0[i], hm, qad, rhs + (size_t)(1 + i) * nx, g->Y_in[i], xs,
                              qad + (size_t)(1 + i) * nx);
          for (int k = 0; k < nx; ++k) rhoY0[k] -= qad[(size_t)(1 + i) * nx + k];
        }
        rc |= lm_solve_diff(&c, w, m->alpha0, hm, qad, rhs + (size_t)(N + 1) * nx, c.h_in, xs,
                            qad + (size_t)(N + 1) * nx);
        /* S5: rho_new Y - w wdot(Y) = b (R_alt form), enthalpy fixed */
        memcpy(b, qad, sizeof(double) * n);
        if (scheme == OR_MISDCQ) {
          for (int j = 1; j <= mm; ++j)
            for (int i = 0; i < n; ++i) b[i] += dt * QIW(&Tb, t, j) * (FR[sC][j][i] - FR[sK][j][i]);
        } else if (mm >= 1) {
          for (int i = 0; i < n; ++i) b[i] += dt * QIW(&Tb, t, mm) * (FR[sC][mm][i] - lRm[i]);
        }
        for (int i = 0; i < n; ++i) b[i] -= w * lRt[i];
        const double *qg = (l == 0) ? q[sK][t] : q[sX][t];
        const double *Tg = (l == 0) ? Tn[sK][t] : Tn[sX][t];
        double *qn = q[sC][t];
        for (int k = 0; k < nx && !rc; ++k) {
          const double rho = qad[k];
          for (int i = 0; i < N; ++i) {
            Yc[i] = qg[(size_t)(1 + i) * nx + k] / qg[k];
            bc[i] = b[(size_t)(1 + i) * nx + k] / rho;
          }
          Yc[N] = Tg[k];
          const double hst = qad[(size_t)(N + 1) * nx + k] / rho;
          int it = or_reaction_newton(m, rho, w, bc, hst, Yc, g->newton_rtol, g->newton_maxit);
          if (it < 0) rc |= 2;
          qn[k] = rho;
          for (int i = 0; i < N; ++i) {
            qn[(size_t)(1 + i) * nx + k] = rho * Yc[i];
            FR[sC][t][(size_t)(1 + i) * nx + k] = (rho * Yc[i] - b[(size_t)(1 + i) * nx + k]) / w;
          }
          FR[sC][t][k] = 0.0;
          FR[sC][t][(size_t)(N + 1) * nx + k] = 0.0;
          qn[(size_t)(N + 1) * nx + k] = qad[(size_t)(N + 1) * nx + k];
          Tn[sC][t][k] = Yc[N];
        }
        /* S6: delta_chi from the thermodynamic-pressure discrepancy, velocity and
         * the advection / diffusion terms at the new state */
        for (int k = 0; k < nx; ++k) Tad[k] = Tn[sC][t][k];
        rc |= or_lm_terms(m, g, qn, NULL, NULL, NULL, NULL, NULL, S, U, pe, Tad);
        for (int k = 0; k < nx; ++k)
          dch[sC][t][k] = g->dchi ? dch[sK][t][k] + 2.0 / g->p0 * (pe[k] - g->p0) / dtm : 0.0;
        rc |= or_lm_terms(m, g, qn, dch[sC][t], NULL, FA[sC][t], FD[sC][t], NULL, S, U, pe, Tn[sC][t]);
        if (l == 0 && t < M && scheme == OR_CISDCQ) {   /* S4: lag source of the next node */
          for (int k = 0; k < nx; ++k) Tad[k] = Tn[sC][t][k];
          rc |= or_lm_terms(m, g, qad, dch[sC][t], NULL, lagA, lagD, NULL, S, U, pe, Tad);
        }
      }
      const int tmp = sX; sX = sC; sC = tmp;   /* iteration l+1 becomes the lag source */
    }
    /* S7 and the sweep increment of rho h at node M */
    if (incr) {
      double dm = 0.0, sm = 0.0;
      for (int k = 0; k < nx; ++k) {
        const double a = q[sX][M][(size_t)(N + 1) * nx + k], bb = q[sK][M][(size_t)(N + 1) * nx + k];
        dm = fmax(dm, fabs(a - bb));
        sm = fmax(sm, fabs(a));
      }
      incr[kk] = sm > 0.0 ? dm / sm : 0.0;
    }
    const int old = sK; sK = sX; sX = old;
  }
  memcpy(q_out, q[sK][M], sizeof(double) * n);
  if (peos_out) {
    for (int k = 0; k < nx; ++k) Tad[k] = Tn[sK][M][k];
    rc |= or_lm_terms(m, g, q_out, NULL, NULL, NULL, NULL, NULL, S, U, peos_out, Tad);
  }
  for (int s = 0; s < 3; ++s)
    for (int j = 0; j <= M; ++j) {
      free(q[s][j]); free(FA[s][j]); free(FD[s][j]); free(FR[s][j]); free(Tn[s][j]); free(dch[s][j]);
    }
  free(qad); free(lagA); free(lagD); free(rhs); free(b); free(S); free(U); free(pe); free(Tad); free(hm);
  free(xs); free(ys); free(Yc); free(bc);
  return rc;
}
