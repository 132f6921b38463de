// Host engine and C ABI of libmisdc.
//
// One time step (Sec. 3.3): I1-I2 copy phi^n into every node; I4 evaluates the
// right-hand sides at phi^n; each sweep k applies the quadrature Q to the node
// stack once (S1 and the sweep-k parts of every update), then runs the
// diffusion (S2-S4) and reaction (S5-S6) steps node by node and iteration by
// iteration; S7 keeps iteration nu as sweep k+1.
//
// CISDCQ runs diffusion steps on stream sD and reaction steps on stream sR.
// Dependencies follow the update equations: the diffusion step at node m+1 of
// iteration l+1 needs the iteration-l reaction results at nodes m and m+1 (for
// l >= 1) and the current-iteration reaction results at nodes < m; the reaction
// step at node m+1 needs its own diffusion step and the reaction step at node
// m (stream order). With three nodes the stages pair up as
//   D1 | D2 || R1 | R2 || D1' | D2' || R1' | R2'
// which is the two-processor pipelining of Sec. 3.2.2.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "misdc_internal.cuh"

using namespace misdc;

namespace {

thread_local std::string g_err;

misdc_status fail(misdc_status st, const std::string &msg) {
  g_err = msg;
  return st;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? MISDC_E_OOM : MISDC_E_CUDA,         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

// ---------------------------------------------------------------------------
// Gauss-Lobatto tables. Interior nodes are the roots of the Jacobi polynomial
// P^{(1,1)}_{M-1} (proportional to P'_M), found by Newton from Chebyshev
// guesses; integration weights come from the moment (Vandermonde) equations
// sum_j q_{m,j} tau_j^p = tau_m^{p+1}/(p+1), p = 0..M; Q~I is the transposed
// upper factor of Gaussian elimination without pivoting on (Q~)^T.
// ---------------------------------------------------------------------------
struct Tables {
  int M = 0;
  double tau[kMaxNodes + 1], Q[kMaxNodes][kMaxNodes + 1], S[kMaxNodes][kMaxNodes + 1];
  double QI[kMaxNodes][kMaxNodes], QE[kMaxNodes][kMaxNodes];
};

long double jacobi11(int n, long double x, long double *dp) {
  long double p0 = 1.0L, p1 = 2.0L * x, d0 = 0.0L, d1 = 2.0L;
  if (n == 0) { *dp = 0.0L; return 1.0L; }
  for (int k = 2; k <= n; ++k) {
    // k(k+2) P_k = (2k+1)(k+1) x P_{k-1} - k(k+1) P_{k-2}
    long double a = (2.0L * k + 1.0L) * (k + 1.0L), b = k * (k + 1.0L), c = k * (k + 2.0L);
    long double p2 = (a * x * p1 - b * p0) / c;
    long double d2 = (a * (p1 + x * d1) - b * d0) / c;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *dp = d1;
  return p1;
}

bool make_tables(int n_nodes, Tables &T) {
  const int M = n_nodes - 1;
  if (M < 1 || M >= kMaxNodes) return false;
  T.M = M;
  long double tau[kMaxNodes + 1];
  tau[0] = 0.0L;
  tau[M] = 1.0L;
  for (int j = 1; j < M; ++j) {
    long double x = cosl(3.141592653589793238462643383279502884L * (M - j) / M);
    for (int it = 0; it < 200; ++it) {
      long double dp, p = jacobi11(M - 1, x, &dp);
      long double dx = p / dp;
      x -= dx;
      if (fabsl(dx) <= 1e-20L) break;
    }
    tau[j] = 0.5L * (1.0L + x);
  }
  // moment equations V^T q = mu with V_{jp} = tau_j^p
  auto solve_weights = [&](long double a, long double b, long double *q) {
    long double A[kMaxNodes + 1][kMaxNodes + 2];
    for (int p = 0; p <= M; ++p) {
      for (int j = 0; j <= M; ++j) A[p][j] = powl(tau[j], p);
      A[p][M + 1] = (powl(b, p + 1) - powl(a, p + 1)) / (p + 1);
    }
    for (int k = 0; k <= M; ++k) {   // Gaussian elimination with partial pivoting
      int piv = k;
      for (int i = k + 1; i <= M; ++i) if (fabsl(A[i][k]) > fabsl(A[piv][k])) piv = i;
      for (int j = 0; j <= M + 1; ++j) std::swap(A[k][j], A[piv][j]);
      for (int i = k + 1; i <= M; ++i) {
        long double f = A[i][k] / A[k][k];
        for (int j = k; j <= M + 1; ++j) A[i][j] -= f * A[k][j];
      }
    }
    for (int i = M; i >= 0; --i) {
      long double s = A[i][M + 1];
      for (int j = i + 1; j <= M; ++j) s -= A[i][j] * q[j];
      q[i] = s / A[i][i];
    }
  };
  long double Ql[kMaxNodes][kMaxNodes + 1];
  for (int m = 1; m <= M; ++m) {
    long double q[kMaxNodes + 1], s[kMaxNodes + 1];
    solve_weights(0.0L, tau[m], q);
    solve_weights(tau[m - 1], tau[m], s);
    for (int j = 0; j <= M; ++j) {
      Ql[m - 1][j] = q[j];
      T.Q[m - 1][j] = (double)q[j];
      T.S[m - 1][j] = (double)s[j];
    }
  }
  for (int m = 0; m <= M; ++m) T.tau[m] = (double)tau[m];
  // (Q~)^T = L U, L unit lower: eliminate below the diagonal, U is what remains
  long double U[kMaxNodes][kMaxNodes];
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) U[i][j] = Ql[j][i + 1];
  for (int k = 0; k < M; ++k)
    for (int i = k + 1; i < M; ++i) {
      long double f = U[i][k] / U[k][k];
      for (int j = k; j < M; ++j) U[i][j] -= f * U[k][j];
    }
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j) {
      T.QI[i][j] = (j <= i) ? (double)U[j][i] : 0.0;
      // forward Euler from t^0: q~E_{i+1, j+1} = (tau_{j+2} - tau_{j+1}) for j < i
      T.QE[i][j] = (j < i) ? (double)(tau[j + 2] - tau[j + 1]) : 0.0;
    }
  return true;
}

struct NodeBuf {
  double *phi = nullptr, *T = nullptr, *theta = nullptr, *hsp = nullptr;
  double *FE = nullptr, *FD = nullptr, *FR = nullptr;
};

}  // namespace

struct misdc_solver {
  int N = 0, R = 0, cs = 0, i0 = 0;
  DevGrid g{};
  DevMech m{};
  misdc_opts o{};
  Tables tab;
  std::vector<void *> allocs;
  std::vector<double> D0h;
  double *vel = nullptr;
  NodeBuf node0, K[kMaxNodes + 1], X[kMaxNodes + 1], Y[kMaxNodes + 1], AD[kMaxNodes + 1];
  double *B[kMaxNodes + 1] = {};
  double *rhsD = nullptr, *bR = nullptr, *thfD = nullptr, *thfR = nullptr;
  double *stage_state = nullptr, *stage_T = nullptr;   // host-step staging
  int *iters = nullptr;
  // learned Newton guess (created on first use)
  Surrogate *sg = nullptr;
  bool sg_on = false, sg_collect = false;
  int sg_sweeps = 0;        // the learned guess serves sweeps k < sg_sweeps (0: all)
  bool sg_this_sweep = true;  // set per sweep while a step is enqueued
  double sg_smin = 1e-8;
  // reaction-Newton launch shape (autotuned)
  NewtonLaunch nl{};
  // mixed precision: FP32 Jacobian factors kept per node between its solves
  ChordStore cst[kMaxNodes + 1];
  bool keep_factors = true;
  double store_dt = -1.0;   // the time step the kept factors belong to
  DiffWork dw{};
  DevStats *st = nullptr;
  cudaStream_t sD = nullptr, sR = nullptr;
  std::vector<cudaEvent_t> evD, evR;   // [M+1][nu]
  cudaEvent_t evIn = nullptr, evOut = nullptr, evFork = nullptr, evJoin = nullptr;
  // CUDA graph of one step
  cudaGraphExec_t gexec = nullptr;
  // adaptive nested iterations (opts.nu_eta > 0, CISDCQ, nu > 2): per-field
  // reduction bits [2F], delta_l [nu], flags {continue, iterations run}, a
  // stream pair and a fork event per nesting level of the IF bodies
  unsigned long long *nu_bits = nullptr;
  double *nu_delta = nullptr;
  int *nu_flags = nullptr;
  std::vector<cudaStream_t> body_streams;
  std::vector<cudaEvent_t> evBody;
  bool in_body = false;
  long long nested_host = 0;   // nested iterations of fixed-nu steps
  int nu_body_kernels = 0;     // kernels of one captured nested-iteration body
  // captured standalone diffusion solve (keyed by its weight) and its output
  cudaGraphExec_t dgexec = nullptr;
  double dg_wdt = -1.0;
  double *dout = nullptr;
  double *g_state = nullptr, *g_T = nullptr;
  double g_dt = 0.0;
  // further stream pairs for the nested iterations of CISDCQ (opts.lanes > 1):
  // iteration l runs on pair l mod lanes, pair 0 being (sD, sR) with the solver's
  // own stage scratch; pairs 1.. have their own
  struct Lane {
    double *rhsD = nullptr, *bR = nullptr, *thfD = nullptr, *thfR = nullptr;
    int *iters = nullptr;
    NewtonLaunch nl{};
    DiffWork dw{};
    cudaStream_t sD = nullptr, sR = nullptr;
  };
  int lanes = 1;
  Lane lane[kMaxLanes];
  int cheb_sweeps = 0;
  double rho_bound = 0.0, rho_dt = -1.0;
  long long kernels_per_step = 0, kernels_launched = 0;
  // optional stage timing (opts.profile)
  std::vector<cudaEvent_t> prof_n, prof_d;   // pairs: start, end
  int n_used = 0, d_used = 0;

  template <typename T>
  cudaError_t alloc(T **p, size_t n) {
    cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) allocs.push_back(*p);
    return e;
  }
  cudaEvent_t &eD(int t, int l) { return evD[(size_t)t * o.nu + l]; }
  cudaEvent_t &eR(int t, int l) { return evR[(size_t)t * o.nu + l]; }
  NodeBuf &nodeK(int j) { return j == 0 ? node0 : K[j]; }
};

namespace {

misdc_status alloc_node(misdc_solver *s, NodeBuf &b) {
  const size_t cs = s->cs, F = s->N + 1;
  CK(s->alloc(&b.phi, F * cs));
  CK(s->alloc(&b.T, cs));
  CK(s->alloc(&b.theta, cs));
  CK(s->alloc(&b.hsp, (size_t)s->N * cs));
  CK(s->alloc(&b.FE, F * cs));
  CK(s->alloc(&b.FD, F * cs));
  CK(s->alloc(&b.FR, F * cs));
  CK(cudaMemset(b.FR, 0, F * cs * sizeof(double)));   // the enthalpy row of F_R stays zero
  CK(cudaMemset(b.T, 0, cs * sizeof(double)));         // "no guess" until a step writes it
  return MISDC_OK;
}

void copy_node(misdc_solver *s, NodeBuf &d, const NodeBuf &a, cudaStream_t st) {
  const size_t cs = s->cs, F = s->N + 1, b = sizeof(double);
  cudaMemcpyAsync(d.phi, a.phi, F * cs * b, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(d.T, a.T, cs * b, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(d.theta, a.theta, cs * b, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(d.hsp, a.hsp, (size_t)s->N * cs * b, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(d.FE, a.FE, F * cs * b, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(d.FD, a.FD, F * cs * b, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(d.FR, a.FR, F * cs * b, cudaMemcpyDeviceToDevice, st);
}

// F_E and F_D of a node state whose theta and hsp are current
void node_operators(misdc_solver *s, NodeBuf &b, double *thf, cudaStream_t st) {
  launch_theta_faces(s->g, b.theta, thf, st);
  launch_operators(s->m, s->g, s->i0, b.phi, b.hsp, thf, s->vel, b.FE, b.FD, thf + 3 * s->cs, st);
}

double rho_bound_for(misdc_solver *s, double wdt_max) {
  // Gershgorin bound of the Jacobi iteration matrix of I - c L_theta, with
  // theta at most (T_max/T_ref)^e on every face
  const double th = pow(kThi / s->m.T_ref, s->m.theta_exp);
  double dmax = s->m.alpha0;
  for (int i = 0; i < s->N; ++i) if (i != s->i0) dmax = std::max(dmax, s->D0h[i]);
  const double cS = wdt_max * dmax / (s->g.dx * s->g.dx) * 2.0 * s->g.dim * th;
  return cS / (1.0 + cS);
}

struct LC {
  LinComb lc;
  LC(double *out) { memset(&lc, 0, sizeof(lc)); lc.n_out = 1; lc.out[0] = out; }
  void add(const double *in, double w) {
    if (w == 0.0 || !in) return;
    for (int k = 0; k < lc.n_in; ++k)
      if (lc.in[k] == in) { lc.w[0][k] += w; return; }
    lc.in[lc.n_in] = in;
    lc.w[0][lc.n_in] = w;
    ++lc.n_in;
  }
};

// Quadrature of sweep k: the parts of every node update that depend on
// sweep k only (one pass over the node stack).
void sweep_quadrature(misdc_solver *s, double dt, cudaStream_t st) {
  const Tables &T = s->tab;
  const int M = T.M, sch = s->o.scheme;
  const size_t n = (size_t)(s->N + 1) * s->cs;
  LinComb lc;
  memset(&lc, 0, sizeof(lc));
  lc.n_out = M;
  lc.in[0] = s->node0.phi;
  int k = 1;
  int idxE[kMaxNodes + 1], idxD[kMaxNodes + 1], idxR[kMaxNodes + 1];
  for (int j = 0; j <= M; ++j) {
    NodeBuf &b = s->nodeK(j);
    idxE[j] = k; lc.in[k++] = b.FE;
    idxD[j] = k; lc.in[k++] = b.FD;
    idxR[j] = k; lc.in[k++] = b.FR;
  }
  lc.n_in = k;
  for (int t = 1; t <= M; ++t) {
    double *w = lc.w[t - 1];
    lc.out[t - 1] = s->B[t];
    const int m = t - 1;
    w[0] = 1.0;
    if (sch == MISDC_SCHEME_MISDC) {
      const double dtm = dt * (T.tau[t] - T.tau[m]);
      for (int j = 0; j <= M; ++j) {
        const double q = dt * T.S[t - 1][j];
        w[idxE[j]] += q; w[idxD[j]] += q; w[idxR[j]] += q;
      }
      w[0] = 0.0;   // MISDC starts from the new state at node m, added per stage
      w[idxE[m]] -= dtm;
      w[idxD[t]] -= dtm;
      continue;
    }
    for (int j = 0; j <= M; ++j) {
      const double q = dt * T.Q[t - 1][j];
      w[idxE[j]] += q; w[idxD[j]] += q; w[idxR[j]] += q;
    }
    for (int j = 1; j <= m; ++j) {
      w[idxE[j]] -= dt * T.QE[t - 1][j - 1];
      w[idxD[j]] -= dt * T.QI[t - 1][j - 1];
      if (sch == MISDC_SCHEME_CISDCQ) w[idxR[j]] -= dt * T.QI[t - 1][j - 1];
    }
    w[idxD[t]] -= dt * T.QI[t - 1][t - 1];
    if (sch == MISDC_SCHEME_CISDCQ) w[idxR[t]] -= dt * T.QI[t - 1][t - 1];
  }
  launch_lincomb(lc, n, st);
}

// temperature, theta and species enthalpies of node 0 (I4) and its F's
void prepare_node0(misdc_solver *s, const double *state, const double *Tin, cudaStream_t st) {
  const size_t cs = s->cs, F = s->N + 1;
  NodeBuf &b = s->node0;
  cudaMemcpyAsync(b.phi, state, F * cs * sizeof(double), cudaMemcpyDeviceToDevice, st);
  // first guess of the temperature: the caller's T, else the last step's final T
  const double *guess = Tin ? Tin : s->K[s->tab.M].T;
  launch_temperature(s->m, s->cs, s->cs, b.phi, b.phi + (size_t)s->N * cs, guess, b.T, b.theta,
                     b.hsp, s->st, st);
  node_operators(s, b, s->thfD, st);
  launch_rates(s->m, s->cs, s->cs, b.phi, b.T, b.FR, st, s->o.rates_mma != 0);
}

// diffusion step at node t: rhs already in s->rhsD; writes AD[t]
// stage scratch of stream pair p (0: the solver's own)
double *lane_rhsD(misdc_solver *s, int p) { return p ? s->lane[p].rhsD : s->rhsD; }
double *lane_bR(misdc_solver *s, int p) { return p ? s->lane[p].bR : s->bR; }
double *lane_thfD(misdc_solver *s, int p) { return p ? s->lane[p].thfD : s->thfD; }
double *lane_thfR(misdc_solver *s, int p) { return p ? s->lane[p].thfR : s->thfR; }
int *lane_iters(misdc_solver *s, int p) { return p ? s->lane[p].iters : s->iters; }
NewtonLaunch *lane_nl(misdc_solver *s, int p) { return p ? &s->lane[p].nl : &s->nl; }
DiffWork &lane_dw(misdc_solver *s, int p) { return p ? s->lane[p].dw : s->dw; }

void d_stage(misdc_solver *s, int t, const double *theta_coef, double wdt, bool lag_source,
             const NodeBuf *Tguess, cudaStream_t st, int p = 0) {
  NodeBuf &ad = s->AD[t];
  const bool prof = s->o.profile && !s->in_body && 2 * (s->d_used + 1) <= (int)s->prof_d.size();
  if (prof) cudaEventRecordWithFlags(s->prof_d[2 * s->d_used], st, cudaEventRecordExternal);
  diffusion_solve(s->m, s->g, s->i0, wdt, theta_coef, lane_rhsD(s, p), ad.phi, lane_dw(s, p),
                  s->cheb_sweeps, s->rho_bound, s->o.lin_rtol, s->st, st);
  if (prof) cudaEventRecordWithFlags(s->prof_d[2 * s->d_used++ + 1], st, cudaEventRecordExternal);
  if (lag_source) {
    launch_temperature(s->m, s->cs, s->cs, ad.phi, ad.phi + (size_t)s->N * s->cs, Tguess->T, ad.T,
                       ad.theta, ad.hsp, s->st, st);
    node_operators(s, ad, lane_thfD(s, p), st);
  }
}

// reaction step at node t: b already in s->bR; writes out (phi, T, theta, hsp, F's)
void r_stage(misdc_solver *s, int t, double wdt, const NodeBuf &guess, NodeBuf &out,
             cudaStream_t st, int p = 0) {
  const size_t cs = s->cs, N = s->N;
  const NodeBuf &ad = s->AD[t];
  const bool prof = s->o.profile && !s->in_body && 2 * (s->n_used + 1) <= (int)s->prof_n.size();
  if (prof) cudaEventRecordWithFlags(s->prof_n[2 * s->n_used], st, cudaEventRecordExternal);
  Surrogate *sg = s->sg;
  const float *pred = nullptr;
  NewtonLaunch nlc = *lane_nl(s, p);
  if (sg && s->sg_collect) {
    // record the features of every solve worth learning (plain Newton follows)
    mlp_features(s->m, s->cs, s->cs, wdt, lane_bR(s, p), ad.phi + N * cs, guess.phi, guess.T, guess.FR,
                 guess.phi + N * cs, sg->ldx, sg->DX, sg->scale, s->sg_smin, sg->ds_count,
                 sg->ds_cap, sg->rowmap, st);
  } else if (sg && s->sg_on && s->sg_this_sweep) {
    // mixed precision with kept factors: certification first, so that the learned
    // guess is computed only for the cells it leaves (a certified guess is
    // converged and needs none)
    const bool pre = s->o.precision == MISDC_PREC_MIXED && s->keep_factors &&
                     launch_certify(s->m, s->cs, s->cs, wdt, s->o.newton_rtol, s->o.newton_maxit, lane_bR(s, p),
                                    ad.phi + N * cs, guess.phi, guess.T, out.phi, out.T, out.FR,
                                    out.hsp, out.theta, lane_iters(s, p), s->st, guess.FR,
                                    guess.phi + N * cs, &s->cst[t], guess.hsp, guess.theta, &nlc, st);
    nlc.precertified = pre;
    // learned guess: features of the cells worth it (s > s_min) gathered into
    // compact rows, then the four layers in one fused kernel over those rows
    cudaMemsetAsync(sg->inf_count, 0, sizeof(unsigned long long), st);
    mlp_features(s->m, s->cs, s->cs, wdt, lane_bR(s, p), ad.phi + N * cs, guess.phi, guess.T, guess.FR,
                 guess.phi + N * cs, sg->ldx, sg->Xi, sg->scale, s->sg_smin, sg->inf_count, s->cs,
                 sg->rowmap, st, pre ? nlc.list : nullptr, pre ? nlc.list_n : nullptr);
    mlp_fused_forward(*sg, nullptr, 0, 0.0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                      nullptr, sg->Xi, s->cs, sg->Oi, st, sg->inf_count);
    pred = sg->Oi;
  }
  launch_newton(s->m, s->cs, s->cs, wdt, s->o.newton_rtol, s->o.newton_maxit, lane_bR(s, p),
                ad.phi + N * cs, guess.phi, guess.T, out.phi, out.T, out.FR, out.hsp, out.theta,
                lane_iters(s, p), s->st, st, s->o.precision == MISDC_PREC_MIXED, pred, sg ? sg->ldo : 0,
                sg ? sg->scale : nullptr, s->sg_smin, guess.FR, guess.phi + N * cs, &nlc,
                s->keep_factors ? &s->cst[t] : nullptr, pred ? sg->rowmap : nullptr, guess.hsp,
                guess.theta);
  if (sg && s->sg_collect)
    mlp_targets(s->N, s->cs, s->cs, guess.phi, guess.T, out.phi, out.T, sg->scale, sg->rowmap,
                sg->ldo, sg->DT, st);
  if (prof) cudaEventRecordWithFlags(s->prof_n[2 * s->n_used++ + 1], st, cudaEventRecordExternal);
  cudaMemcpyAsync(out.phi + N * cs, ad.phi + N * cs, cs * sizeof(double), cudaMemcpyDeviceToDevice, st);
  node_operators(s, out, lane_thfR(s, p), st);
}

// stream pairs a step uses for its nested iterations (the learned guess and the
// adaptive rule keep one pair: their scratch and decisions are per solver)
int step_lanes(const misdc_solver *s) {
  const bool two = s->o.two_streams && s->o.scheme == MISDC_SCHEME_CISDCQ;
  return (two && s->nu_bits == nullptr && !(s->sg && (s->sg_on || s->sg_collect))) ? s->lanes : 1;
}

// Enqueue one full time step on s->sD (and s->sR).
void enqueue_step(misdc_solver *s, double *state, double *Tio, double dt) {
  const Tables &T = s->tab;
  const int M = T.M, nu = s->o.nu, sch = s->o.scheme;
  const size_t cs = s->cs, F = s->N + 1, n = F * cs;
  const bool two = s->o.two_streams && sch == MISDC_SCHEME_CISDCQ;
  cudaStream_t sD = s->sD, sR = two ? s->sR : s->sD;
  s->n_used = s->d_used = 0;
  const int lanes = step_lanes(s);

  prepare_node0(s, state, Tio, sD);
  for (int m = 1; m <= M; ++m) copy_node(s, s->K[m], s->node0, sD);   // I1-I2
  if (two) {
    cudaEventRecord(s->evFork, sD);
    cudaStreamWaitEvent(sR, s->evFork, 0);
    for (int p = 1; p < lanes; ++p) {
      cudaStreamWaitEvent(s->lane[p].sD, s->evFork, 0);
      cudaStreamWaitEvent(s->lane[p].sR, s->evFork, 0);
    }
  }
  for (int k = 0; k < s->o.n_sweeps; ++k) {
    s->sg_this_sweep = s->sg_sweeps <= 0 || k < s->sg_sweeps;
    sweep_quadrature(s, dt, sD);
    if (sch == MISDC_SCHEME_CISDCQ) {
      // one nested iteration l on streams qD (diffusion) and qR (reaction); `fresh`:
      // everything of iteration l-1 is complete before the first node starts (an
      // adaptive iteration that starts after the decision), so no waits on it
      auto iteration = [&](int l, cudaStream_t qD, cudaStream_t qR, bool fresh, bool join, int lp = 0) {
        const bool dual = qD != qR;
        NodeBuf *C = (l % 2 == 0) ? s->X : s->Y;
        NodeBuf *P = (l == 0) ? s->K : ((l % 2 == 1) ? s->X : s->Y);
        for (int m = 0; m < M; ++m) {
          const int t = m + 1;
          // ---- diffusion step at node t ----
          if (dual && l >= 1 && !fresh) {
            if (m >= 1) cudaStreamWaitEvent(qD, s->eR(m, l - 1), 0);
            cudaStreamWaitEvent(qD, s->eR(t, l - 1), 0);
            // on its own stream pair iteration l overtakes l-1: before this node's
            // buffers (those of iteration l-2) are rewritten, iteration l-1 must have
            // read them, its last reader being the reaction step at node t+1
            if (lanes > 1 && t < M) cudaStreamWaitEvent(qD, s->eR(t + 1, l - 1), 0);
          }
          if (dual) for (int j = 1; j <= m - 1; ++j) cudaStreamWaitEvent(qD, s->eR(j, l), 0);
          LC r(lane_rhsD(s, lp));
          r.add(s->B[t], 1.0);
          for (int j = 1; j <= m - 1; ++j) {
            r.add(C[j].FE, dt * T.QE[t - 1][j - 1]);
            r.add(C[j].FD, dt * T.QI[t - 1][j - 1]);
            r.add(C[j].FR, dt * T.QI[t - 1][j - 1]);
          }
          if (m >= 1) {
            const double *lagE = (l == 0) ? s->AD[m].FE : P[m].FE;
            const double *lagD = (l == 0) ? s->AD[m].FD : P[m].FD;
            const double *lagR = (l == 0) ? s->K[m].FR : P[m].FR;
            r.add(lagE, dt * T.QE[t - 1][m - 1]);
            r.add(lagD, dt * T.QI[t - 1][m - 1]);
            r.add(lagR, dt * T.QI[t - 1][m - 1]);
          }
          const double *lagR1 = (l == 0) ? s->K[t].FR : P[t].FR;
          r.add(lagR1, dt * T.QI[t - 1][t - 1]);
          launch_lincomb(r.lc, n, qD);
          const double wdt = dt * T.QI[t - 1][t - 1];
          const double *coef = (l == 0) ? s->K[t].theta : P[t].theta;
          d_stage(s, t, coef, wdt, l == 0 && t < M, &s->K[t], qD, lp);
          if (dual) cudaEventRecord(s->eD(t, l), qD);
          // ---- reaction step at node t (R_alt form) ----
          if (dual) cudaStreamWaitEvent(qR, s->eD(t, l), 0);
          LC b(lane_bR(s, lp));
          b.add(s->AD[t].phi, 1.0);
          if (m >= 1) {
            const double *lagRm = (l == 0) ? s->K[m].FR : P[m].FR;
            b.add(C[m].FR, dt * T.QI[t - 1][m - 1]);
            b.add(lagRm, -dt * T.QI[t - 1][m - 1]);
          }
          b.add(lagR1, -dt * T.QI[t - 1][t - 1]);
          launch_lincomb(b.lc, n, qR);
          r_stage(s, t, wdt, P[t], C[t], qR, lp);
          if (dual) cudaEventRecord(s->eR(t, l), qR);
        }
        if (dual && join) cudaStreamWaitEvent(qD, s->eR(M, l), 0);   // the iteration ends on qD
      };
      // the adaptive rule after iteration l (on qD): delta_l from the node stacks
      // of iterations l and l-1 (sweep k for l = 0)
      auto decide = [&](int l, cudaStream_t qD, const cudaGraphConditionalHandle *h, bool body) {
        NodePtrs now{}, before{};
        NodeBuf *C = (l % 2 == 0) ? s->X : s->Y;
        NodeBuf *P = (l == 0) ? s->K : ((l % 2 == 1) ? s->X : s->Y);
        for (int m = 1; m <= M; ++m) { now.p[m - 1] = C[m].phi; before.p[m - 1] = P[m].phi; }
        launch_nu_decide((int)F, (int)cs, M, now, before, l, nu, s->o.nu_eta, s->o.nu_rho_stall,
                         s->nu_bits, s->nu_delta, s->nu_flags, s->nu_flags + 1, s->st, h,
                         body ? s->nu_flags + 2 : nullptr, qD);
      };
      const bool adapt = s->nu_bits != nullptr;
      if (!adapt) {
        for (int l = 0; l < nu; ++l) {
          const int lp = l % lanes;
          iteration(l, lp ? s->lane[lp].sD : sD, lp ? s->lane[lp].sR : sR, false, l == nu - 1, lp);
        }
        // the sweep's last reaction step follows every other stage of the sweep
        if (lanes > 1) cudaStreamWaitEvent(sD, s->eR(M, nu - 1), 0);
      } else {
        // iterations 0 and 1 always run; iteration l >= 2 runs inside an IF graph
        // node (nested in the body of l-1) that the decision after l-1 sets, or, in
        // an eager step, after the host has read that decision
        iteration(0, sD, sR, false, true);
        decide(0, sD, nullptr, false);
        iteration(1, sD, sR, false, true);
        cudaGraphConditionalHandle h;
        if (graph_conditional_handle(sD, 0, &h)) {
          decide(1, sD, &h, false);
          cudaStream_t outer = sD;
          s->in_body = true;
          int opened = 0;
          for (int l = 2; l < nu; ++l) {
            cudaGraph_t body = graph_conditional_node(outer, cudaGraphCondTypeIf, h);
            if (!body) break;   // the capture reports the failure at its end
            cudaStream_t bD = s->body_streams[2 * opened], bR = two ? s->body_streams[2 * opened + 1] : bD;
            cudaStreamBeginCaptureToGraph(bD, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (two) {
              cudaEventRecord(s->evBody[opened], bD);
              cudaStreamWaitEvent(bR, s->evBody[opened], 0);
            }
            ++opened;
            iteration(l, bD, bR, true, true);
            const bool more = l + 1 < nu && graph_conditional_handle(bD, 0, &h);
            decide(l, bD, more ? &h : nullptr, true);
            outer = bD;
            if (!more) break;
          }
          // close the nested captures from the innermost out (the bodies belong to
          // their conditional nodes)
          for (int d = opened - 1; d >= 0; --d) {
            cudaGraph_t done = nullptr;
            if (cudaStreamEndCapture(s->body_streams[2 * d], &done) == cudaSuccess && d == 0 && done) {
              // kernels of one nested iteration (a body without its nested IF), counted
              // by the device each time a body runs
              size_t nn = 0;
              cudaGraphGetNodes(done, nullptr, &nn);
              std::vector<cudaGraphNode_t> nodes(nn);
              cudaGraphGetNodes(done, nodes.data(), &nn);
              int kernels = 0;
              for (auto nd : nodes) {
                cudaGraphNodeType ty;
                cudaGraphNodeGetType(nd, &ty);
                if (ty == cudaGraphNodeTypeKernel) ++kernels;
              }
              s->nu_body_kernels = kernels;   // uploaded once the capture has ended
            }
          }
          s->in_body = false;
        } else {
          decide(1, sD, nullptr, false);
          for (int l = 2; l < nu; ++l) {
            int cont = 0;
            cudaMemcpyAsync(&cont, s->nu_flags, sizeof(int), cudaMemcpyDeviceToHost, sD);
            cudaStreamSynchronize(sD);
            if (!cont) break;
            iteration(l, sD, sR, false, true);
            decide(l, sD, nullptr, false);
          }
        }
        // the result must sit in the buffer S7 takes (that of iteration nu-1)
        CopyList cl{};
        NodeBuf *last = ((nu - 1) % 2 == 0) ? s->X : s->Y, *other = ((nu - 1) % 2 == 0) ? s->Y : s->X;
        const size_t sizes[7] = {F * cs, cs, cs, (size_t)s->N * cs, F * cs, F * cs, F * cs};
        for (int m = 1; m <= M; ++m) {
          double *dst[7] = {last[m].phi, last[m].T, last[m].theta, last[m].hsp, last[m].FE, last[m].FD, last[m].FR};
          const double *src[7] = {other[m].phi, other[m].T, other[m].theta, other[m].hsp, other[m].FE, other[m].FD, other[m].FR};
          for (int q = 0; q < 7; ++q) {
            cl.dst[cl.count] = dst[q];
            cl.src[cl.count] = src[q];
            cl.n[cl.count++] = sizes[q];
          }
        }
        launch_copy_if_parity(cl, s->nu_flags + 1, (nu - 1) & 1, sD);
      }
      NodeBuf *last = ((nu - 1) % 2 == 0) ? s->X : s->Y;   // S7
      for (int m = 1; m <= M; ++m) std::swap(s->K[m], last[m]);
    } else {
      NodeBuf *C = s->X;
      for (int m = 0; m < M; ++m) {
        const int t = m + 1;
        LC r(s->rhsD);
        r.add(s->B[t], 1.0);
        double wdt;
        if (sch == MISDC_SCHEME_MISDCQ) {
          for (int j = 1; j <= m; ++j) {
            r.add(C[j].FE, dt * T.QE[t - 1][j - 1]);
            r.add(C[j].FD, dt * T.QI[t - 1][j - 1]);
          }
          wdt = dt * T.QI[t - 1][t - 1];
        } else {   // MISDC: from the new state at node m
          const double dtm = dt * (T.tau[t] - T.tau[m]);
          const NodeBuf &prev = (m == 0) ? s->node0 : C[m];
          r.add(prev.phi, 1.0);
          r.add(prev.FE, dtm);
          wdt = dtm;
        }
        launch_lincomb(r.lc, n, sD);
        d_stage(s, t, s->K[t].theta, wdt, false, nullptr, sD);
        LC b(s->bR);
        b.add(s->AD[t].phi, 1.0);
        if (sch == MISDC_SCHEME_MISDCQ) {
          for (int j = 1; j <= m; ++j) {
            b.add(C[j].FR, dt * T.QI[t - 1][j - 1]);
            b.add(s->K[j].FR, -dt * T.QI[t - 1][j - 1]);
          }
        }
        b.add(s->K[t].FR, -wdt);
        launch_lincomb(b.lc, n, sD);
        r_stage(s, t, wdt, s->K[t], C[t], sD);
      }
      for (int m = 1; m <= M; ++m) std::swap(s->K[m], C[m]);
    }
  }
  NodeBuf &fin = s->K[M];
  cudaMemcpyAsync(state, fin.phi, n * sizeof(double), cudaMemcpyDeviceToDevice, sD);
  if (Tio) cudaMemcpyAsync(Tio, fin.T, cs * sizeof(double), cudaMemcpyDeviceToDevice, sD);
}

misdc_status configure_dt(misdc_solver *s, double dt) {
  if (s->rho_dt == dt) return MISDC_OK;
  double qmax = 0.0;
  for (int t = 0; t < s->tab.M; ++t) {
    qmax = std::max(qmax, s->tab.QI[t][t]);
    qmax = std::max(qmax, s->tab.tau[t + 1] - s->tab.tau[t]);
  }
  s->rho_bound = rho_bound_for(s, dt * qmax);
  s->cheb_sweeps = std::min(kMaxCheb, chebyshev_sweeps(s->rho_bound, std::max(1e-3 * s->o.lin_rtol, 1e-17)));
  s->rho_dt = dt;
  if (s->store_dt != dt) {
    // kept Jacobian factors belong to the weights w dt of another time step
    if (s->store_dt > 0.0) {
      cudaStreamSynchronize(s->sD);
      cudaStreamSynchronize(s->sR);
      for (int j = 1; j <= s->tab.M; ++j)
        if (s->cst[j].valid) cudaMemsetAsync(s->cst[j].valid, 0, (size_t)s->cs * sizeof(int), s->sD);
      cudaStreamSynchronize(s->sD);
    }
    s->store_dt = dt;
  }
  return MISDC_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *misdc_last_error(void) { return g_err.c_str(); }

void misdc_default_opts(misdc_opts *o) {
  memset(o, 0, sizeof(*o));
  o->n_nodes = 3;
  o->n_sweeps = 4;
  o->nu = 2;
  o->scheme = MISDC_SCHEME_CISDCQ;
  o->precision = MISDC_PREC_FP64;
  o->dominant_species = 0;
  o->rho = 1.0;
  o->newton_rtol = 1e-12;
  o->newton_maxit = 50;
  o->lin_rtol = 1e-14;
  o->mg_levels = 1;
  o->two_streams = 1;
  o->lanes = 1;
  o->lin_rounds = 0;
  o->use_graph = 1;
}

misdc_status misdc_lobatto(int n_nodes, double *tau, double *Q, double *QI, double *QE) {
  Tables T;
  if (!make_tables(n_nodes, T)) return fail(MISDC_E_INVALID, "n_nodes must be in 2..9");
  const int M = T.M;
  for (int m = 0; m <= M; ++m) if (tau) tau[m] = T.tau[m];
  for (int i = 0; i < M; ++i) {
    for (int j = 0; j <= M; ++j) if (Q) Q[i * (M + 1) + j] = T.Q[i][j];
    for (int j = 0; j < M; ++j) {
      if (QI) QI[i * M + j] = T.QI[i][j];
      if (QE) QE[i * M + j] = T.QE[i][j];
    }
  }
  return MISDC_OK;
}

misdc_status misdc_create(const misdc_mech_desc *md, const misdc_grid_desc *gd,
                          const misdc_opts *op, const double *face_vel, misdc_solver **out) {
  if (!md || !gd || !op || !out) return fail(MISDC_E_INVALID, "null argument");
  *out = nullptr;
  const int N = md->n_species, R = md->n_reactions;
  if (N < 1 || N > kMaxSpecies || R < 1 || R > 1024) return fail(MISDC_E_INVALID, "n_species must be 1..63 and n_reactions 1..1024");
  if (!md->W || !md->nasa7 || !md->A || !md->beta || !md->Ea || !md->nu_f || !md->nu_r || !md->D0)
    return fail(MISDC_E_INVALID, "null mechanism array");
  if (op->rates_mma) {   // 32 cells' reaction rates are staged in shared memory
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if ((size_t)(32 * (size_t)mma_qld(R) + 20 * (size_t)N) * sizeof(double) > (size_t)optin)
      return fail(MISDC_E_INVALID, "rates_mma: too many reactions for shared memory");
  }
  if (gd->dim < 1 || gd->dim > 3 || gd->nx < 2 || gd->ny < 1 || gd->nz < 1 || !(gd->dx > 0.0))
    return fail(MISDC_E_INVALID, "bad grid");
  if ((gd->dim < 2 && gd->ny != 1) || (gd->dim < 3 && gd->nz != 1) || (gd->dim >= 2 && gd->ny < 2) ||
      (gd->dim >= 3 && gd->nz < 2))
    return fail(MISDC_E_INVALID, "grid extents do not match dim");
  const long long cells = (long long)gd->nx * gd->ny * gd->nz;
  if (cells > (1LL << 30)) return fail(MISDC_E_INVALID, "grid too large");
  if (op->n_nodes < 2 || op->n_nodes > 5) return fail(MISDC_E_INVALID, "n_nodes must be 2..5");
  if (op->n_sweeps < 1 || op->nu < 1 || op->nu > 16) return fail(MISDC_E_INVALID, "bad n_sweeps/nu");
  if (op->nu_eta > 0.0 && !(op->nu_rho_stall > 0.0))
    return fail(MISDC_E_INVALID, "adaptive nu needs nu_rho_stall > 0");
  if (op->scheme < 0 || op->scheme > 2) return fail(MISDC_E_INVALID, "bad scheme");
  if (op->precision != MISDC_PREC_FP64 && op->precision != MISDC_PREC_MIXED)
    return fail(MISDC_E_INVALID, "precision must be MISDC_PREC_FP64 or MISDC_PREC_MIXED");
  if (op->dominant_species < 0 || op->dominant_species >= N) return fail(MISDC_E_INVALID, "bad dominant species");
  if (!(op->rho > 0.0) || !(op->newton_rtol > 0.0) || op->newton_maxit < 1 || !(op->lin_rtol > 0.0))
    return fail(MISDC_E_INVALID, "bad tolerances or density");
  if (op->mg_levels < 0 || op->mg_levels > 6) return fail(MISDC_E_INVALID, "mg_levels must be 0..6");
  if (!face_vel) return fail(MISDC_E_INVALID, "null face velocity");
  for (int i = 0; i < N; ++i)
    if (!(md->W[i] > 0.0) || !(md->D0[i] >= 0.0)) return fail(MISDC_E_INVALID, "bad W or D0");
  CK(init_exp_table());   // the rate kernels' exponential, once per device

  misdc_solver *s = new misdc_solver();
  auto bail = [&](misdc_status st) { misdc_destroy(s); return st; };
  s->N = N; s->R = R; s->cs = (int)cells; s->i0 = op->dominant_species; s->o = *op;
  if (s->o.mg_levels == 0) s->o.mg_levels = 1;
  if (!make_tables(op->n_nodes, s->tab)) return bail(fail(MISDC_E_INVALID, "bad n_nodes"));
  s->g.dim = gd->dim; s->g.nx = gd->nx; s->g.ny = gd->ny; s->g.nz = gd->nz;
  s->g.cells = (int)cells; s->g.dx = gd->dx;
  s->D0h.assign(md->D0, md->D0 + N);

  // ---- mechanism tables ----
  std::vector<double> invW(N), hc(6 * N), sc(6 * N), cpc(5 * N), lnA(R), beta(R), TA(R), dn(R);
  std::vector<signed char> fwd(kMaxSlots * R, -1), rev(kMaxSlots * R, -1);
  std::vector<int> sp_ptr(N + 1, 0), sp_rx;
  std::vector<double> sp_coef;
  for (int i = 0; i < N; ++i) {
    const double *a = md->nasa7 + 7 * i;
    invW[i] = 1.0 / md->W[i];
    const double h6[6] = {a[0], a[1] / 2, a[2] / 3, a[3] / 4, a[4] / 5, a[5]};
    const double s6[6] = {a[0], a[1], a[2] / 2, a[3] / 3, a[4] / 4, a[6]};
    for (int k = 0; k < 6; ++k) { hc[6 * i + k] = h6[k]; sc[6 * i + k] = s6[k]; }
    for (int k = 0; k < 5; ++k) cpc[5 * i + k] = a[k];
  }
  for (int r = 0; r < R; ++r) {
    if (!(md->A[r] > 0.0)) return bail(fail(MISDC_E_INVALID, "A must be positive"));
    lnA[r] = log(md->A[r]);
    beta[r] = md->beta[r];
    TA[r] = md->Ea[r] / kRu;
    int nf = 0, nr = 0, d = 0;
    for (int i = 0; i < N; ++i) {
      const int a = md->nu_f[(size_t)r * N + i], b = md->nu_r[(size_t)r * N + i];
      if (a < 0 || b < 0) return bail(fail(MISDC_E_INVALID, "negative stoichiometry"));
      for (int k = 0; k < a; ++k) { if (nf >= kMaxSlots) return bail(fail(MISDC_E_INVALID, "more than 3 reactant molecules")); fwd[kMaxSlots * r + nf++] = (signed char)i; }
      for (int k = 0; k < b; ++k) { if (nr >= kMaxSlots) return bail(fail(MISDC_E_INVALID, "more than 3 product molecules")); rev[kMaxSlots * r + nr++] = (signed char)i; }
      d += b - a;
    }
    dn[r] = d;
  }
  for (int i = 0; i < N; ++i) {
    for (int r = 0; r < R; ++r) {
      const int nu = md->nu_r[(size_t)r * N + i] - md->nu_f[(size_t)r * N + i];
      if (nu) { sp_rx.push_back(r); sp_coef.push_back(md->W[i] * nu); }
    }
    sp_ptr[i + 1] = (int)sp_rx.size();
  }
  // Newton assembly list (see DevMech::jc_pack): for every species row i and every
  // reaction r it takes part in, with c = W_i nu_ri: the residual term (-c/rho, q_r),
  // the temperature column (c/rho, dq_r/dT) and one entry per molecule slot s of r,
  // (c/W_s, slot derivative of q_r). Sorted by target, cut into 32 lane segments.
  const int ldn = newton_ld(N), nnn = N + 1;
  struct Contrib { int t, s; double w; };
  std::vector<Contrib> cl;
  for (int i = 0; i < N; ++i)
    for (int r = 0; r < R; ++r) {
      const int nu = md->nu_r[(size_t)r * N + i] - md->nu_f[(size_t)r * N + i];
      if (!nu) continue;
      const double c = md->W[i] * nu;
      cl.push_back({i * ldn + nnn, r, -c / op->rho});
      cl.push_back({i * ldn + N, R + r, c / op->rho});
      for (int p = 0; p < kMaxSlots; ++p) {
        const int sf = fwd[kMaxSlots * r + p], sr = rev[kMaxSlots * r + p];
        if (sf >= 0) cl.push_back({i * ldn + sf, 2 * R + 6 * r + p, c / md->W[sf]});
        if (sr >= 0) cl.push_back({i * ldn + sr, 2 * R + 6 * r + 3 + p, c / md->W[sr]});
      }
    }
  std::stable_sort(cl.begin(), cl.end(), [](const Contrib &a, const Contrib &b) {
    return a.t != b.t ? a.t < b.t : a.s < b.s;
  });
  std::vector<int> jc_pack(cl.size()), jc_seg(33, (int)cl.size());
  std::vector<double> jc_w(cl.size());
  for (size_t k = 0; k < cl.size(); ++k) {
    jc_pack[k] = (cl[k].t << 16) | cl[k].s;
    jc_w[k] = cl[k].w;
  }
  jc_seg[0] = 0;
  {
    int lanes = 1;
    const double per = (double)cl.size() / 32.0;
    for (size_t k = 1; k < cl.size() && lanes < 32; ++k)
      if (cl[k].t != cl[k - 1].t && (double)k >= per * lanes) jc_seg[lanes++] = (int)k;
  }
  // tensor-core tiles of [W_i nu_ri] (see DevMech::mma_b)
  const int mma_nt = (N + 7) / 8, mma_kbs = (R + 3) / 4;
  std::vector<int> mma_ptr(1, 0), mma_kb;
  std::vector<double> mma_b;
  for (int jt = 0; jt < mma_nt; ++jt) {
    for (int kb = 0; kb < mma_kbs; ++kb) {
      double frag[32];
      bool any = false;
      for (int l = 0; l < 32; ++l) {
        const int r = 4 * kb + (l & 3), i = 8 * jt + (l >> 2);
        frag[l] = 0.0;
        if (r < R && i < N) {
          const int nu = md->nu_r[(size_t)r * N + i] - md->nu_f[(size_t)r * N + i];
          if (nu) { frag[l] = md->W[i] * nu; any = true; }
        }
      }
      if (!any) continue;
      mma_kb.push_back(kb);
      mma_b.insert(mma_b.end(), frag, frag + 32);
    }
    mma_ptr.push_back((int)mma_kb.size());
  }
  auto up = [&](auto &vec, auto **dst) -> cudaError_t {
    using T = typename std::remove_reference<decltype(vec)>::type::value_type;
    cudaError_t e = s->alloc((T **)dst, vec.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy((void *)*dst, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice);
  };
  std::vector<double> D0v(md->D0, md->D0 + N), Wv(md->W, md->W + N);
  double *p_W, *p_invW, *p_hc, *p_sc, *p_cpc, *p_D0, *p_lnA, *p_beta, *p_TA, *p_dn, *p_spc, *p_jcw, *p_mb;
  signed char *p_fwd, *p_rev;
  int *p_spp, *p_spr, *p_jcp, *p_jcs, *p_mp, *p_mk;
  if (up(Wv, &p_W) || up(invW, &p_invW) || up(hc, &p_hc) || up(sc, &p_sc) || up(cpc, &p_cpc) || up(D0v, &p_D0) ||
      up(lnA, &p_lnA) || up(beta, &p_beta) || up(TA, &p_TA) || up(dn, &p_dn) || up(fwd, &p_fwd) ||
      up(rev, &p_rev) || up(sp_ptr, &p_spp) || up(sp_rx, &p_spr) || up(sp_coef, &p_spc) ||
      up(jc_pack, &p_jcp) || up(jc_w, &p_jcw) || up(jc_seg, &p_jcs) || up(mma_b, &p_mb) ||
      up(mma_ptr, &p_mp) || up(mma_kb, &p_mk))
    return bail(fail(MISDC_E_OOM, "mechanism upload failed"));
  DevMech &m = s->m;
  m.N = N; m.R = R; m.rho = op->rho; m.T_ref = md->T_ref; m.theta_exp = md->theta_exp;
  m.alpha0 = md->alpha0; m.ln_p_over_R = log(md->p_ref / kRu); m.ln_Tref = log(md->T_ref);
  m.W = p_W; m.invW = p_invW; m.hcoef = p_hc; m.scoef = p_sc; m.cpcoef = p_cpc; m.D0 = p_D0;
  m.lnA = p_lnA; m.beta = p_beta; m.TA = p_TA; m.dn = p_dn; m.fwd = p_fwd; m.rev = p_rev;
  m.sp_ptr = p_spp; m.sp_rx = p_spr; m.sp_coef = p_spc;
  m.D0_host = s->D0h.data();
  m.jc_pack = p_jcp; m.jc_w = p_jcw; m.jc_seg = p_jcs;
  m.mma_b = p_mb; m.mma_ptr = p_mp; m.mma_kb = p_mk; m.mma_nt = mma_nt;
  m.mma_ntiles = (int)mma_kb.size();
  prepare_chem_kernels(m);

  // ---- buffers ----
  const size_t cs = s->cs, F = N + 1;
  misdc_status st;
  if (s->alloc(&s->vel, 3 * cs)) return bail(fail(MISDC_E_OOM, "velocity"));
  if (cudaMemset(s->vel, 0, 3 * cs * sizeof(double)) ||
      cudaMemcpy(s->vel, face_vel, (size_t)gd->dim * cs * sizeof(double), cudaMemcpyDefault))
    return bail(fail(MISDC_E_CUDA, "velocity copy failed"));
  if ((st = alloc_node(s, s->node0))) return bail(st);
  const int M = s->tab.M;
  for (int j = 1; j <= M; ++j) {
    if ((st = alloc_node(s, s->K[j])) || (st = alloc_node(s, s->X[j])) || (st = alloc_node(s, s->AD[j])))
      return bail(st);
    if (op->scheme == MISDC_SCHEME_CISDCQ && op->nu > 1 && (st = alloc_node(s, s->Y[j]))) return bail(st);
    if (s->alloc(&s->B[j], F * cs)) return bail(fail(MISDC_E_OOM, "B"));
  }
  // per stream: theta on the faces [3][cs], then the operators' face fluxes
  const size_t thf_n = 3 * cs + operator_face_doubles(s->g, s->N);
  if (s->alloc(&s->rhsD, F * cs) || s->alloc(&s->bR, F * cs) || s->alloc(&s->thfD, thf_n) ||
      s->alloc(&s->thfR, thf_n) || s->alloc(&s->iters, cs) || s->alloc(&s->st, 1) ||
      s->alloc(&s->nl.work, 1) || s->alloc(&s->nl.list, cs) || s->alloc(&s->nl.list_n, 1) ||
      s->alloc(&s->nl.list2, cs) || s->alloc(&s->nl.list2_n, 1) ||
      s->alloc(&s->dw.thf, 3 * cs) || s->alloc(&s->dw.invdiag, F * cs) || s->alloc(&s->dw.xa, F * cs) ||
      s->alloc(&s->dw.cdiag, F * cs) || s->alloc(&s->dw.bdiag, F * cs) ||
      s->alloc(&s->dw.xb, F * cs) || s->alloc(&s->dw.xc, F * cs) ||
      s->alloc(&s->dw.rho_bits, 1) || s->alloc(&s->dw.kdev, 1) || s->alloc(&s->dw.omega, kMaxCheb))
    return bail(fail(MISDC_E_OOM, "work buffers"));
  cudaMemset(s->st, 0, sizeof(DevStats));
  if (s->o.precision == MISDC_PREC_MIXED) {
    DiffWork &w = s->dw;
    if (s->alloc(&w.thf32, 3 * cs) || s->alloc(&w.invdiag32, F * cs) || s->alloc(&w.r32, F * cs) ||
        s->alloc(&w.e32[0], F * cs) || s->alloc(&w.e32[1], F * cs) || s->alloc(&w.e32[2], F * cs) ||
        s->alloc(&w.kdev32, 1) || s->alloc(&w.omega32, kMaxCheb))
      return bail(fail(MISDC_E_OOM, "mixed diffusion buffers"));
    w.refine_rounds = (s->o.lin_rounds > 0) ? std::min(s->o.lin_rounds, 8) : 3;
    for (int j = 1; j <= M; ++j) {
      ChordStore &c = s->cst[j];
      c.fs = chord_floats(N);
      c.swld = (int)((F + 3) / 4 * 4);
      if (s->alloc(&c.f, (size_t)c.fs * cs) || s->alloc(&c.sw, (size_t)c.swld * cs) ||
          s->alloc(&c.valid, cs) || s->alloc(&c.z32, (size_t)F * F * cs) ||
          s->alloc(&c.xc, (size_t)F * cs) || s->alloc(&c.sT, cs))
        return bail(fail(MISDC_E_OOM, "factor store"));
      cudaMemset(c.valid, 0, cs * sizeof(int));
    }
  }
  // multigrid hierarchy (levels with even extents only); in mixed precision the
  // coarse levels are FP32
  s->dw.levels = 1;
  s->dw.cycles = 40;
  s->dw.lg[0] = s->g;
  if (s->o.mg_levels > 1) {
    DiffWork &w = s->dw;
    const size_t nfs = N;
    w.mg32 = s->o.precision == MISDC_PREC_MIXED;
    if (s->alloc(&w.lb[0], nfs * cs) || s->alloc(&w.lx[0], nfs * cs) || s->alloc(&w.lr[0], nfs * cs) ||
        s->alloc(&w.ly[0], nfs * cs) || s->alloc(&w.mg_done, 1) || s->alloc(&w.mg_res, 1) ||
        s->alloc(&w.mg_cycle, 1))
      return bail(fail(MISDC_E_OOM, "multigrid"));
    if (cudaStreamCreateWithFlags(&w.mg_stream, cudaStreamNonBlocking))
      return bail(fail(MISDC_E_CUDA, "stream creation failed"));
    for (int l = 1; l < s->o.mg_levels; ++l) {
      DevGrid c = w.lg[l - 1];
      if ((c.nx % 2) || (c.dim > 1 && c.ny % 2) || (c.dim > 2 && c.nz % 2) || c.nx < 4) break;
      c.nx /= 2;
      if (c.dim > 1) c.ny /= 2;
      if (c.dim > 2) c.nz /= 2;
      c.cells = c.nx * c.ny * c.nz;
      c.dx *= 2.0;
      w.lg[l] = c;
      const size_t cc = c.cells;
      const bool bad = w.mg32
          ? (s->alloc(&w.lthf32[l], 3 * cc) || s->alloc(&w.linvdiag32[l], nfs * cc) ||
             s->alloc(&w.lb32[l], nfs * cc) || s->alloc(&w.lx32[l], nfs * cc) ||
             s->alloc(&w.lr32[l], nfs * cc) || s->alloc(&w.ly32[l], nfs * cc))
          : (s->alloc(&w.lthf[l], 3 * cc) || s->alloc(&w.linvdiag[l], nfs * cc) ||
             s->alloc(&w.lb[l], nfs * cc) || s->alloc(&w.lx[l], nfs * cc) ||
             s->alloc(&w.lr[l], nfs * cc) || s->alloc(&w.ly[l], nfs * cc));
      if (bad) return bail(fail(MISDC_E_OOM, "multigrid"));
      w.levels = l + 1;
    }
  }
  if (cudaStreamCreateWithFlags(&s->sD, cudaStreamNonBlocking) ||
      cudaStreamCreateWithFlags(&s->sR, cudaStreamNonBlocking))
    return bail(fail(MISDC_E_CUDA, "stream creation failed"));
  // further stream pairs of the nested iterations: CISDCQ on two streams with the
  // Chebyshev diffusion solve (multigrid keeps one pair: its loop state is shared)
  s->lanes = 1;
  if (op->lanes > 1 && op->scheme == MISDC_SCHEME_CISDCQ && op->two_streams && op->nu > 1 &&
      s->dw.levels <= 1)
    s->lanes = std::min(std::min(op->lanes, op->nu), kMaxLanes);
  for (int p = 1; p < s->lanes; ++p) {
    misdc_solver::Lane &L = s->lane[p];
    DiffWork &w = L.dw;
    w = s->dw;   // options and sizes; the arrays below are the lane's own
    const size_t thf_n = 3 * cs + operator_face_doubles(s->g, s->N);
    if (s->alloc(&L.rhsD, F * cs) || s->alloc(&L.bR, F * cs) || s->alloc(&L.thfD, thf_n) ||
        s->alloc(&L.thfR, thf_n) || s->alloc(&L.iters, cs) || s->alloc(&L.nl.work, 1) ||
        s->alloc(&L.nl.list, cs) || s->alloc(&L.nl.list_n, 1) ||
        s->alloc(&L.nl.list2, cs) || s->alloc(&L.nl.list2_n, 1) || s->alloc(&w.thf, 3 * cs) ||
        s->alloc(&w.invdiag, F * cs) || s->alloc(&w.cdiag, F * cs) || s->alloc(&w.bdiag, F * cs) ||
        s->alloc(&w.xa, F * cs) || s->alloc(&w.xb, F * cs) || s->alloc(&w.xc, F * cs) ||
        s->alloc(&w.rho_bits, 1) || s->alloc(&w.kdev, 1) || s->alloc(&w.omega, kMaxCheb))
      return bail(fail(MISDC_E_OOM, "stream-pair buffers"));
    if (s->o.precision == MISDC_PREC_MIXED &&
        (s->alloc(&w.thf32, 3 * cs) || s->alloc(&w.invdiag32, F * cs) || s->alloc(&w.r32, F * cs) ||
         s->alloc(&w.e32[0], F * cs) || s->alloc(&w.e32[1], F * cs) || s->alloc(&w.e32[2], F * cs) ||
         s->alloc(&w.kdev32, 1) || s->alloc(&w.omega32, kMaxCheb)))
      return bail(fail(MISDC_E_OOM, "stream-pair buffers"));
    L.nl.wpb = s->nl.wpb;
    L.nl.blocks_per_sm = s->nl.blocks_per_sm;
    L.nl.dynamic = s->nl.dynamic;
    if (cudaStreamCreateWithFlags(&L.sD, cudaStreamNonBlocking) ||
        cudaStreamCreateWithFlags(&L.sR, cudaStreamNonBlocking))
      return bail(fail(MISDC_E_CUDA, "stream creation failed"));
  }
  s->evD.assign((size_t)(M + 1) * op->nu, nullptr);
  s->evR.assign((size_t)(M + 1) * op->nu, nullptr);
  for (auto *v : {&s->evD, &s->evR})
    for (auto &e : *v)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming)) return bail(fail(MISDC_E_CUDA, "event"));
  for (cudaEvent_t *e : {&s->evIn, &s->evOut, &s->evFork, &s->evJoin})
    if (cudaEventCreateWithFlags(e, cudaEventDisableTiming)) return bail(fail(MISDC_E_CUDA, "event"));
  if (op->scheme == MISDC_SCHEME_CISDCQ && op->nu > 2 && op->nu_eta > 0.0) {
    if (s->alloc(&s->nu_bits, 2 * F) || s->alloc(&s->nu_delta, (size_t)op->nu) || s->alloc(&s->nu_flags, 3))
      return bail(fail(MISDC_E_OOM, "adaptive nested iterations"));
    cudaMemset(s->nu_bits, 0, 2 * F * sizeof(unsigned long long));
    s->body_streams.assign(2 * (size_t)(op->nu - 2), nullptr);
    s->evBody.assign((size_t)(op->nu - 2), nullptr);
    for (auto &q : s->body_streams)
      if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking)) return bail(fail(MISDC_E_CUDA, "stream creation failed"));
    for (auto &e : s->evBody)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming)) return bail(fail(MISDC_E_CUDA, "event"));
  }
  if (op->profile) {
    const int stages = op->n_sweeps * M * (op->scheme == MISDC_SCHEME_CISDCQ ? op->nu : 1);
    s->prof_n.assign(2 * (size_t)stages, nullptr);
    s->prof_d.assign(2 * (size_t)stages, nullptr);
    for (auto *v : {&s->prof_n, &s->prof_d})
      for (auto &ev : *v)
        if (cudaEventCreate(&ev)) return bail(fail(MISDC_E_CUDA, "event"));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bail(fail(MISDC_E_CUDA, cudaGetErrorString(e)));
  *out = s;
  return MISDC_OK;
}

void misdc_destroy(misdc_solver *s) {
  if (!s) return;
  if (s->sD) cudaStreamSynchronize(s->sD);
  if (s->sR) cudaStreamSynchronize(s->sR);
  for (int p = 1; p < kMaxLanes; ++p) {
    if (s->lane[p].sD) cudaStreamSynchronize(s->lane[p].sD);
    if (s->lane[p].sR) cudaStreamSynchronize(s->lane[p].sR);
  }
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->dgexec) cudaGraphExecDestroy(s->dgexec);
  for (auto *v : {&s->evD, &s->evR})
    for (auto &ev : *v) if (ev) cudaEventDestroy(ev);
  for (cudaEvent_t ev : {s->evIn, s->evOut, s->evFork, s->evJoin}) if (ev) cudaEventDestroy(ev);
  for (auto *v : {&s->prof_n, &s->prof_d})
    for (auto &ev : *v) if (ev) cudaEventDestroy(ev);
  if (s->sD) cudaStreamDestroy(s->sD);
  if (s->sR) cudaStreamDestroy(s->sR);
  for (int p = 1; p < kMaxLanes; ++p) {
    if (s->lane[p].sD) cudaStreamDestroy(s->lane[p].sD);
    if (s->lane[p].sR) cudaStreamDestroy(s->lane[p].sR);
  }
  if (s->dw.mg_stream) cudaStreamDestroy(s->dw.mg_stream);
  for (cudaStream_t q : s->body_streams) if (q) cudaStreamDestroy(q);
  for (cudaEvent_t e : s->evBody) if (e) cudaEventDestroy(e);
  for (void *p : s->allocs) cudaFree(p);
  delete s->sg;
  delete s;
}

misdc_status misdc_step(misdc_solver *s, double *state, double *T, double dt, int n_steps,
                        void *stream) {
  if (!s || !state) return fail(MISDC_E_INVALID, "null argument");
  if (!(dt > 0.0) || n_steps < 0) return fail(MISDC_E_INVALID, "dt must be > 0 and n_steps >= 0");
  if (n_steps == 0) return MISDC_OK;
  cudaStream_t us = (cudaStream_t)stream;
  configure_dt(s, dt);
  if (s->o.scheme == MISDC_SCHEME_CISDCQ && !s->nu_bits)
    s->nested_host += (long long)n_steps * s->o.n_sweeps * s->o.nu;
  CK(cudaEventRecord(s->evIn, us));
  CK(cudaStreamWaitEvent(s->sD, s->evIn, 0));
  if (s->o.use_graph) {
    if (!s->gexec || s->g_state != state || s->g_T != T || s->g_dt != dt) {
      if (s->gexec) { cudaGraphExecDestroy(s->gexec); s->gexec = nullptr; }
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(s->sD, cudaStreamCaptureModeThreadLocal));
      enqueue_step(s, state, T, dt);
      cudaError_t ec = cudaStreamEndCapture(s->sD, &graph);
      if (ec != cudaSuccess) return fail(MISDC_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
      size_t nn = 0;
      cudaGraphGetNodes(graph, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      cudaGraphGetNodes(graph, nodes.data(), &nn);
      s->kernels_per_step = 0;
      for (auto nd : nodes) {
        cudaGraphNodeType ty;
        cudaGraphNodeGetType(nd, &ty);
        if (ty == cudaGraphNodeTypeKernel) ++s->kernels_per_step;
      }
      ec = cudaGraphInstantiate(&s->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ec != cudaSuccess) return fail(MISDC_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ec));
      s->g_state = state; s->g_T = T; s->g_dt = dt;
      if (s->nu_flags) CK(cudaMemcpy(s->nu_flags + 2, &s->nu_body_kernels, sizeof(int), cudaMemcpyHostToDevice));
    }
    for (int i = 0; i < n_steps; ++i) CK(cudaGraphLaunch(s->gexec, s->sD));
    s->kernels_launched += s->kernels_per_step * n_steps;
  } else {
    for (int i = 0; i < n_steps; ++i) enqueue_step(s, state, T, dt);
  }
  CK(cudaGetLastError());
  CK(cudaEventRecord(s->evOut, s->sD));
  CK(cudaStreamWaitEvent(us, s->evOut, 0));
  return MISDC_OK;
}

misdc_status misdc_step_host(misdc_solver *s, double *state_host, double *T_host, double dt,
                             int n_steps, void *stream) {
  if (!s || !state_host) return fail(MISDC_E_INVALID, "null argument");
  const size_t cs = s->cs, F = s->N + 1;
  if (!s->stage_state) {
    CK(s->alloc(&s->stage_state, F * cs));
    CK(s->alloc(&s->stage_T, cs));
  }
  cudaStream_t us = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(s->stage_state, state_host, F * cs * sizeof(double), cudaMemcpyHostToDevice, us));
  if (T_host) CK(cudaMemcpyAsync(s->stage_T, T_host, cs * sizeof(double), cudaMemcpyHostToDevice, us));
  misdc_status st = misdc_step(s, s->stage_state, T_host ? s->stage_T : nullptr, dt, n_steps, stream);
  if (st) return st;
  CK(cudaMemcpyAsync(state_host, s->stage_state, F * cs * sizeof(double), cudaMemcpyDeviceToHost, us));
  if (T_host) CK(cudaMemcpyAsync(T_host, s->stage_T, cs * sizeof(double), cudaMemcpyDeviceToHost, us));
  CK(cudaStreamSynchronize(us));
  return MISDC_OK;
}

misdc_status misdc_get_stats(misdc_solver *s, misdc_stats *out, int reset) {
  if (!s || !out) return fail(MISDC_E_INVALID, "null argument");
  CK(cudaStreamSynchronize(s->sD));
  CK(cudaStreamSynchronize(s->sR));
  DevStats d;
  CK(cudaMemcpy(&d, s->st, sizeof(d), cudaMemcpyDeviceToHost));
  out->newton_solves = (long long)d.newton_solves;
  out->newton_iters = (long long)d.newton_iters;
  out->newton_fail = (long long)d.newton_fail;
  out->newton_max = d.newton_max;
  out->lin_sweeps = (long long)d.lin_sweeps;
  double r;
  memcpy(&r, &d.lin_resid_bits, sizeof(r));
  out->lin_resid_max = r;
  out->kernel_launches = s->kernels_launched + (long long)d.body_launches;
  out->nested_iterations = (long long)d.nested_iters + s->nested_host;
  out->surrogate_used = (long long)d.sg_used;
  out->surrogate_rejected = (long long)d.sg_rejected;
  out->newton_fp64_fallbacks = (long long)d.fp64_fallbacks;
  out->newton_jacobians = (long long)d.jacobians;
  out->newton_lu_fp64 = (long long)d.lu64;
  out->newton_certified = (long long)d.certified;
  out->newton_stored_steps = (long long)d.stored_steps;
  out->newton_floor_stops = (long long)d.floor_stops;
  out->newton_chord_cells = (long long)d.chord_cells;
  int st = MISDC_OK;
  if (d.status_bits & kBitTdiag) st = MISDC_E_TDIAG;
  else if (d.status_bits & (kBitNan | kBitSingular)) st = MISDC_E_NAN;
  else if (d.status_bits & kBitNewton) st = MISDC_E_NEWTON;
  else if (d.status_bits & kBitMG) st = MISDC_E_MG;
  else if (d.status_bits & kBitTimeout) st = MISDC_E_TIMEOUT;
  out->status = st;
  if (reset) {
    CK(cudaMemset(s->st, 0, sizeof(DevStats)));
    s->kernels_launched = 0;
    s->nested_host = 0;
  }
  return MISDC_OK;
}

misdc_status misdc_stage_times(misdc_solver *s, double *newton_ms, int *newton_launches,
                               double *diffusion_ms, int *diffusion_launches) {
  if (!s) return fail(MISDC_E_INVALID, "null argument");
  if (!s->o.profile) return fail(MISDC_E_INVALID, "solver was created without opts.profile");
  CK(cudaStreamSynchronize(s->sD));
  CK(cudaStreamSynchronize(s->sR));
  double tn = 0.0, td = 0.0;
  for (int i = 0; i < s->n_used; ++i) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, s->prof_n[2 * i], s->prof_n[2 * i + 1]));
    tn += ms;
  }
  for (int i = 0; i < s->d_used; ++i) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, s->prof_d[2 * i], s->prof_d[2 * i + 1]));
    td += ms;
  }
  if (newton_ms) *newton_ms = tn;
  if (newton_launches) *newton_launches = s->n_used;
  if (diffusion_ms) *diffusion_ms = td;
  if (diffusion_launches) *diffusion_launches = s->d_used;
  return MISDC_OK;
}

misdc_status misdc_enthalpy(misdc_solver *s, const double *Y, const double *T, double *h, int n,
                            void *stream) {
  if (!s || !Y || !T || !h || n < 0) return fail(MISDC_E_INVALID, "bad argument");
  launch_enthalpy(s->m, n, n, Y, T, h, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return MISDC_OK;
}

misdc_status misdc_temperature(misdc_solver *s, const double *Y, const double *h, double *T, int n,
                               void *stream) {
  if (!s || !Y || !T || !h || n < 0) return fail(MISDC_E_INVALID, "bad argument");
  launch_temperature(s->m, n, n, Y, h, T, T, nullptr, nullptr, s->st, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return MISDC_OK;
}

misdc_status misdc_production_rates(misdc_solver *s, const double *Y, const double *T, double *FR,
                                    int n, void *stream) {
  if (!s || !Y || !T || !FR || n < 0) return fail(MISDC_E_INVALID, "bad argument");
  launch_rates(s->m, n, n, Y, T, FR, (cudaStream_t)stream, s->o.rates_mma != 0);
  CK(cudaGetLastError());
  return MISDC_OK;
}

misdc_status misdc_reaction_solve(misdc_solver *s, double wdt, const double *b, const double *hstar,
                                  double *x, double *FR, int *iters, int n, void *stream) {
  if (!s || !b || !hstar || !x || n < 0) return fail(MISDC_E_INVALID, "bad argument");
  if (!(wdt >= 0.0)) return fail(MISDC_E_INVALID, "wdt must be >= 0");
  if (n == 0) return MISDC_OK;
  const size_t N = s->N;
  double *hsp = nullptr, *th = nullptr;
  CK(cudaMallocAsync(&hsp, N * n * sizeof(double), (cudaStream_t)stream));
  CK(cudaMallocAsync(&th, n * sizeof(double), (cudaStream_t)stream));
  NewtonLaunch nl = s->nl;
  nl.dynamic = 0;   // the counter belongs to the step's stream
  nl.list = nl.list_n = nullptr;
  launch_newton(s->m, n, n, wdt, s->o.newton_rtol, s->o.newton_maxit, b, hstar, x, x + N * n, x,
                x + N * n, FR, hsp, th, iters, s->st, (cudaStream_t)stream,
                s->o.precision == MISDC_PREC_MIXED, nullptr, 0, nullptr, 0.0, nullptr, nullptr, &nl);
  cudaFreeAsync(hsp, (cudaStream_t)stream);
  cudaFreeAsync(th, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return MISDC_OK;
}

misdc_status misdc_operators(misdc_solver *s, const double *state, double *FE, double *FD, double *FR,
                             void *stream) {
  if (!s || !state) return fail(MISDC_E_INVALID, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaStreamSynchronize(s->sD));
  NodeBuf &b = s->node0;
  const size_t cs = s->cs, F = s->N + 1;
  CK(cudaMemcpyAsync(b.phi, state, F * cs * sizeof(double), cudaMemcpyDeviceToDevice, st));
  launch_temperature(s->m, s->cs, s->cs, b.phi, b.phi + (size_t)s->N * cs, nullptr, b.T, b.theta,
                     b.hsp, s->st, st);
  launch_theta_faces(s->g, b.theta, s->thfD, st);
  if (FE || FD)
    launch_operators(s->m, s->g, s->i0, b.phi, b.hsp, s->thfD, s->vel, FE, FD, s->thfD + 3 * cs, st);
  if (FR) {
    launch_rates(s->m, s->cs, s->cs, b.phi, b.T, FR, st, s->o.rates_mma != 0);
    CK(cudaMemsetAsync(FR + (size_t)s->N * cs, 0, cs * sizeof(double), st));
  }
  CK(cudaGetLastError());
  return MISDC_OK;
}

misdc_status misdc_diffusion_solve(misdc_solver *s, double wdt, const double *coef_state,
                                   const double *rhs, double *x, void *stream) {
  if (!s || !coef_state || !rhs || !x) return fail(MISDC_E_INVALID, "bad argument");
  if (!(wdt >= 0.0)) return fail(MISDC_E_INVALID, "wdt must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaStreamSynchronize(s->sD));
  NodeBuf &b = s->node0;
  const size_t cs = s->cs, F = s->N + 1;
  s->rho_dt = -1.0;
  s->rho_bound = rho_bound_for(s, wdt);
  s->cheb_sweeps = std::min(kMaxCheb, chebyshev_sweeps(s->rho_bound, std::max(1e-3 * s->o.lin_rtol, 1e-17)));
  auto enqueue = [&](double *out, cudaStream_t q) {
    launch_temperature(s->m, s->cs, s->cs, b.phi, b.phi + (size_t)s->N * cs, nullptr, b.T, b.theta,
                       nullptr, s->st, q);
    diffusion_solve(s->m, s->g, s->i0, wdt, b.theta, s->rhsD, out, s->dw, s->cheb_sweeps,
                    s->rho_bound, s->o.lin_rtol, s->st, q);
  };
  if (!s->o.use_graph) {
    CK(cudaMemcpyAsync(b.phi, coef_state, F * cs * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(s->rhsD, rhs, F * cs * sizeof(double), cudaMemcpyDeviceToDevice, st));
    enqueue(x, st);
    CK(cudaGetLastError());
    return MISDC_OK;
  }
  // captured once per weight (multigrid cycles then run as a WHILE graph node):
  // inputs copied into the solver's buffers, the result copied out
  if (!s->dout) CK(s->alloc(&s->dout, F * cs));
  CK(cudaEventRecord(s->evIn, st));
  CK(cudaStreamWaitEvent(s->sD, s->evIn, 0));
  CK(cudaMemcpyAsync(b.phi, coef_state, F * cs * sizeof(double), cudaMemcpyDeviceToDevice, s->sD));
  CK(cudaMemcpyAsync(s->rhsD, rhs, F * cs * sizeof(double), cudaMemcpyDeviceToDevice, s->sD));
  if (!s->dgexec || s->dg_wdt != wdt) {
    if (s->dgexec) { cudaGraphExecDestroy(s->dgexec); s->dgexec = nullptr; }
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(s->sD, cudaStreamCaptureModeThreadLocal));
    enqueue(s->dout, s->sD);
    cudaError_t ec = cudaStreamEndCapture(s->sD, &graph);
    if (ec != cudaSuccess) return fail(MISDC_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    ec = cudaGraphInstantiate(&s->dgexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) return fail(MISDC_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ec));
    s->dg_wdt = wdt;
  }
  CK(cudaGraphLaunch(s->dgexec, s->sD));
  CK(cudaMemcpyAsync(x, s->dout, F * cs * sizeof(double), cudaMemcpyDeviceToDevice, s->sD));
  CK(cudaEventRecord(s->evOut, s->sD));
  CK(cudaStreamWaitEvent(st, s->evOut, 0));
  return MISDC_OK;
}

misdc_status misdc_lincomb(int n_out, int n_in, double *const *out, const double *const *in,
                           const double *w, size_t n, void *stream) {
  if (n_out < 1 || n_out > 8 || n_in < 1 || n_in > 16 || !out || !in || !w)
    return fail(MISDC_E_INVALID, "lincomb supports 1..8 outputs and 1..16 inputs");
  LinComb lc;
  memset(&lc, 0, sizeof(lc));
  lc.n_out = n_out;
  lc.n_in = n_in;
  for (int o = 0; o < n_out; ++o) {
    if (!out[o]) return fail(MISDC_E_INVALID, "null output");
    lc.out[o] = out[o];
    for (int k = 0; k < n_in; ++k) lc.w[o][k] = w[o * n_in + k];
  }
  for (int k = 0; k < n_in; ++k) {
    if (!in[k]) return fail(MISDC_E_INVALID, "null input");
    lc.in[k] = in[k];
  }
  launch_lincomb(lc, n, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return MISDC_OK;
}

misdc_status misdc_exp(const double *x, double *y, size_t n, void *stream) {
  if (n == 0) return MISDC_OK;
  if (!x || !y) return fail(MISDC_E_INVALID, "exp: null array");
  CK(init_exp_table());
  CK(launch_exp(x, y, n, (cudaStream_t)stream));
  return MISDC_OK;
}

misdc_status misdc_pde_smem_bytes(int n_nodes, int nx, size_t *bytes) {
  if (!bytes || n_nodes < 2 || n_nodes > kMaxNodes || nx < 1)
    return fail(MISDC_E_INVALID, "pde_smem_bytes: bad argument");
  *bytes = pde_smem_bytes(n_nodes - 1, nx);
  return MISDC_OK;
}

misdc_status misdc_pde_step(int scheme, int n_nodes, int n_sweeps, int nu, double dt, int n_steps,
                            int nx, double length, int n, const double *params,
                            const double *phi_in, double *phi_out, double *incr, int *status,
                            void *stream) {
  if (scheme < MISDC_SCHEME_MISDC || scheme > MISDC_SCHEME_CISDCQ)
    return fail(MISDC_E_INVALID, "pde_step: unknown scheme");
  if (n_sweeps < 1 || nu < 1 || n_steps < 1 || !(dt > 0.0) || !(length > 0.0) || n < 0)
    return fail(MISDC_E_INVALID, "pde_step: n_sweeps, nu, n_steps, dt, length must be positive");
  if (nx < 8) return fail(MISDC_E_INVALID, "pde_step: nx must be at least 8");
  if (n == 0) return MISDC_OK;
  if (!params || !phi_in || !phi_out) return fail(MISDC_E_INVALID, "pde_step: null array");
  Tables T;
  if (!make_tables(n_nodes, T)) return fail(MISDC_E_INVALID, "pde_step: n_nodes must be in 2..9");
  const bool batch = n >= kPdeBatchMin;
  if (!batch) {
    int dev = 0, smem_max = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (pde_smem_bytes(T.M, nx) > (size_t)smem_max)
      return fail(MISDC_E_INVALID, "pde_step: nx too large for one block's shared memory (" +
                                       std::to_string(pde_smem_bytes(T.M, nx)) + " > " +
                                       std::to_string(smem_max) + " bytes)");
  }
  PdeLaunch p;
  memset(&p, 0, sizeof(p));
  p.scheme = scheme; p.M = T.M; p.n_sweeps = n_sweeps; p.nu = nu; p.n_steps = n_steps;
  p.nx = nx; p.n = n; p.dt = dt; p.dx = length / nx;
  memcpy(p.tau, T.tau, sizeof(p.tau));
  memcpy(p.Q, T.Q, sizeof(p.Q));
  memcpy(p.S, T.S, sizeof(p.S));
  memcpy(p.QI, T.QI, sizeof(p.QI));
  memcpy(p.QE, T.QE, sizeof(p.QE));
  p.params = params; p.phi_in = phi_in; p.phi_out = phi_out; p.incr = incr; p.status = status;
  cudaStream_t cs = (cudaStream_t)stream;
  if (!batch) {
    CK(launch_pde_step(p, cs));
    return MISDC_OK;
  }
  // stream-ordered workspace of the batched layout, freed behind the launch
  double *ws = nullptr;
  CK(cudaMallocAsync((void **)&ws, pde_batch_bytes(T.M, nx, n), cs));
  const cudaError_t e = launch_pde_batch(p, ws, cs);
  cudaFreeAsync(ws, cs);
  CK(e);
  return MISDC_OK;
}

misdc_status misdc_lowmach_step(misdc_solver *s, const misdc_lowmach_desc *d, double dt, int n,
                                const double *q_in, double *q_out, double *peos, int *status,
                                void *stream) {
  if (!s || !d || !d->Y_in) return fail(MISDC_E_INVALID, "lowmach_step: null argument");
  if (s->g.dim != 1 || s->g.nx < 4)
    return fail(MISDC_E_INVALID, "lowmach_step: the solver's grid must be 1D with at least 4 cells");
  if (s->o.scheme != MISDC_SCHEME_CISDCQ && s->o.scheme != MISDC_SCHEME_MISDCQ)
    return fail(MISDC_E_INVALID, "lowmach_step: the scheme must be CISDCQ or MISDCQ");
  if (!(dt > 0.0) || n < 0 || !(d->p0 > 0.0) || !(d->T_in > 0.0))
    return fail(MISDC_E_INVALID, "lowmach_step: dt, p0 and T_in must be positive, n >= 0");
  if (n == 0) return MISDC_OK;
  if (!q_in || !q_out) return fail(MISDC_E_INVALID, "lowmach_step: null state");
  cudaStream_t cs = (cudaStream_t)stream;
  const int nx = s->g.nx, M = s->tab.M;
  double *ws = nullptr;
  const cudaError_t ea = cudaMallocAsync((void **)&ws, lowmach_work_bytes(s->N, nx, M, n), cs);
  if (ea != cudaSuccess) return fail(MISDC_E_OOM, "lowmach_step: workspace");
  const cudaError_t e = launch_lowmach(s->m, nx, s->g.dx, M, s->tab.tau, s->tab.Q, s->tab.QI, s->tab.QE,
                                       s->o.scheme, s->o.n_sweeps, s->o.nu, s->i0, s->o.newton_rtol,
                                       s->o.newton_maxit, dt, d->U_in, d->T_in, d->p0, d->dchi ? 1 : 0,
                                       d->Y_in, n, q_in, q_out, peos, status, ws, cs);
  cudaFreeAsync(ws, cs);
  CK(e);
  return MISDC_OK;
}

}  // extern "C"

// ===========================================================================
// Reaction solve without any device allocation.
//
// Some callers cannot allocate device memory while they run: code executing
// inside a host callback or a memory-pool-restricted process, plugins whose host
// application owns every allocation, and real-time loops that forbid the
// implicit synchronisation cudaMalloc/cudaFree can cause. For them this entry
// point runs the same per-cell reaction Newton as misdc_reaction_solve, but
// takes its scratch (per-call counters, theta and the species enthalpies of the
// solution, which this call discards) from one statically sized device array
// instead of cudaMallocAsync. It allocates nothing.
//
// Limits and rules: the array holds kNoAllocScratchDoubles doubles (4 MiB) on
// every device that loads the library, for the life of the process; a call
// needs 32 + n (N + 1) of them and larger n is rejected with MISDC_E_INVALID.
// All calls share the array: calls that overlap on the GPU (different streams,
// or several solvers at once) race on it. The first call on a device looks the
// array's device address up (cudaGetSymbolAddress); make that first call before
// any stream capture. Each call clears its counters before the kernel runs.
// ===========================================================================
namespace {

constexpr size_t kNoAllocScratchDoubles = size_t(1) << 19;   // 4 MiB
constexpr size_t kNoAllocStatsDoubles = 32;                   // 256 bytes for DevStats

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_noalloc_mu;
double *g_noalloc_addr[64] = {};   // device address of the array, per device ordinal

// Device address of the scratch array on the current device (looked up once).
misdc_status noalloc_scratch(double **out) {
  static_assert(sizeof(DevStats) <= kNoAllocStatsDoubles * sizeof(double), "stats block");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(MISDC_E_INVALID, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(MISDC_E_CUDA, std::string("cudaGetSymbolAddress(no-allocation scratch): ") +
                                    cudaGetErrorString(e));
    g_noalloc_addr[dev] = static_cast<double *>(p);
  }
  *out = g_noalloc_addr[dev];
  return MISDC_OK;
}

}  // namespace

extern "C" misdc_status misdc_reaction_solve_noalloc(misdc_solver *s, double wdt, const double *b,
                                                     const double *hstar, double *x, double *FR,
                                                     int *iters, int n, void *stream) {
  if (!s || !b || !hstar || !x || n < 0) return fail(MISDC_E_INVALID, "bad argument");
  if (!(wdt >= 0.0)) return fail(MISDC_E_INVALID, "wdt must be >= 0");
  const size_t N = s->N;
  const size_t need = kNoAllocStatsDoubles + (size_t)n * (N + 1);
  if (need > kNoAllocScratchDoubles)
    return fail(MISDC_E_INVALID, "n = " + std::to_string(n) + " needs " + std::to_string(need) +
                                     " scratch doubles; the no-allocation scratch holds " +
                                     std::to_string(kNoAllocScratchDoubles) + " (at most " +
                                     std::to_string((kNoAllocScratchDoubles - kNoAllocStatsDoubles) / (N + 1)) +
                                     " cells for this mechanism)");
  if (n == 0) return MISDC_OK;
  double *base = nullptr;
  misdc_status st = noalloc_scratch(&base);
  if (st != MISDC_OK) return st;
  cudaStream_t cs = (cudaStream_t)stream;
  DevStats *stats = reinterpret_cast<DevStats *>(base);
  double *theta = base + kNoAllocStatsDoubles;
  double *hsp = theta + n;
  CK(cudaMemsetAsync(stats, 0, sizeof(DevStats), cs));
  NewtonLaunch nl = s->nl;   // the solver's (autotuned) launch shape, as misdc_reaction_solve
  nl.dynamic = 0;            // the work counter is solver memory: static cell scheduling here
  nl.list = nl.list_n = nullptr;
  launch_newton(s->m, n, n, wdt, s->o.newton_rtol, s->o.newton_maxit, b, hstar, x, x + N * n, x,
                x + N * n, FR, hsp, theta, iters, stats, cs, s->o.precision == MISDC_PREC_MIXED,
                nullptr, 0, nullptr, 0.0, nullptr, nullptr, &nl);
  CK(cudaGetLastError());
  return MISDC_OK;
}

// ===========================================================================
// Learned initial guess of the reaction Newton
// ===========================================================================
namespace {

misdc_status sg_ready(misdc_solver *s, bool need_params) {
  if (!s) return fail(MISDC_E_INVALID, "null solver");
  if (!s->sg) {
    Surrogate *g = new Surrogate();
    cudaError_t e = g->setup(s->N);
    if (e != cudaSuccess) {
      delete g;
      return fail(e == cudaErrorMemoryAllocation ? MISDC_E_OOM : MISDC_E_CUDA,
                  std::string("surrogate setup: ") + cudaGetErrorString(e));
    }
    mlp_prepare();
    s->sg = g;
  }
  if (need_params && !s->sg->ready)
    return fail(MISDC_E_INVALID, "surrogate parameters are not initialised or loaded");
  return MISDC_OK;
}

// a changed step program must be captured again
void drop_graph(misdc_solver *s) {
  if (s->gexec || s->dgexec) cudaStreamSynchronize(s->sD);
  if (s->gexec) {
    cudaGraphExecDestroy(s->gexec);
    s->gexec = nullptr;
  }
  if (s->dgexec) {
    cudaGraphExecDestroy(s->dgexec);
    s->dgexec = nullptr;
  }
}

misdc_status sg_check_err(misdc_solver *s, cudaStream_t st) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, s->sg->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (e) {
    CK(cudaMemset(s->sg->err, 0, sizeof(int)));
    return fail(MISDC_E_TIMEOUT, "a tensor-core MMA wait gave up");
  }
  return MISDC_OK;
}

}  // namespace

extern "C" {

misdc_status misdc_surrogate_dims(misdc_solver *s, int *n_in, int *ldx, int *n_hidden, int *n_out,
                                  int *ldo, size_t *n_params) {
  misdc_status st = sg_ready(s, false);
  if (st) return st;
  const Surrogate &g = *s->sg;
  if (n_in) *n_in = g.n_in;
  if (ldx) *ldx = g.ldx;
  if (n_hidden) *n_hidden = g.H;
  if (n_out) *n_out = g.n_out;
  if (ldo) *ldo = g.ldo;
  if (n_params) *n_params = g.n_params;
  return MISDC_OK;
}

misdc_status misdc_surrogate_init(misdc_solver *s, unsigned long long seed) {
  misdc_status st = sg_ready(s, false);
  if (st) return st;
  std::vector<float> h;
  s->sg->init_params(seed, h);
  CK(s->sg->upload(h.data(), s->sD));
  CK(cudaStreamSynchronize(s->sD));
  return MISDC_OK;
}

misdc_status misdc_surrogate_load(misdc_solver *s, const float *params, size_t n_params) {
  misdc_status st = sg_ready(s, false);
  if (st) return st;
  if (!params || n_params != s->sg->n_params) return fail(MISDC_E_INVALID, "parameter count mismatch");
  CK(s->sg->upload(params, s->sD));
  CK(cudaStreamSynchronize(s->sD));
  return MISDC_OK;
}

misdc_status misdc_surrogate_save(misdc_solver *s, float *params, size_t n_params) {
  misdc_status st = sg_ready(s, true);
  if (st) return st;
  if (!params || n_params != s->sg->n_params) return fail(MISDC_E_INVALID, "parameter count mismatch");
  CK(cudaStreamSynchronize(s->sD));
  CK(cudaStreamSynchronize(s->sR));
  CK(cudaMemcpy(params, s->sg->P, n_params * sizeof(float), cudaMemcpyDeviceToHost));
  return MISDC_OK;
}

misdc_status misdc_surrogate_sweeps(misdc_solver *s, int n_sweeps) {
  if (!s || n_sweeps < 0) return fail(MISDC_E_INVALID, "surrogate_sweeps: bad argument");
  drop_graph(s);
  s->sg_sweeps = n_sweeps;
  return MISDC_OK;
}

misdc_status misdc_surrogate_enable(misdc_solver *s, int on, double s_min) {
  misdc_status st = sg_ready(s, on != 0);
  if (st) return st;
  if (!(s_min >= 0.0)) return fail(MISDC_E_INVALID, "s_min must be >= 0");
  if (on) {
    cudaError_t e = s->sg->ensure_inference(s->cs);
    if (e != cudaSuccess) return fail(MISDC_E_OOM, cudaGetErrorString(e));
  }
  drop_graph(s);
  s->sg_on = on != 0;
  s->sg_smin = s_min;
  return MISDC_OK;
}

misdc_status misdc_surrogate_collect(misdc_solver *s, long long capacity) {
  misdc_status st = sg_ready(s, false);
  if (st) return st;
  if (capacity < 0) return fail(MISDC_E_INVALID, "capacity must be >= 0");
  drop_graph(s);
  if (capacity == 0) {
    s->sg_collect = false;
    return MISDC_OK;
  }
  cudaError_t e = s->sg->ensure_inference(s->cs);
  if (e == cudaSuccess) e = s->sg->ensure_dataset(capacity);
  if (e != cudaSuccess) return fail(MISDC_E_OOM, cudaGetErrorString(e));
  s->sg_collect = true;
  return MISDC_OK;
}

misdc_status misdc_surrogate_dataset(misdc_solver *s, long long *rows, const void **X,
                                     const float **targets) {
  misdc_status st = sg_ready(s, false);
  if (st) return st;
  long long r = 0;
  if (s->sg->ds_count) {
    CK(cudaStreamSynchronize(s->sD));
    CK(cudaStreamSynchronize(s->sR));
    unsigned long long c = 0;
    CK(cudaMemcpy(&c, s->sg->ds_count, sizeof(c), cudaMemcpyDeviceToHost));
    r = (long long)std::min<unsigned long long>(c, (unsigned long long)s->sg->ds_cap);
  }
  if (rows) *rows = r;
  if (X) *X = s->sg->DX;
  if (targets) *targets = s->sg->DT;
  return MISDC_OK;
}

misdc_status misdc_surrogate_features(misdc_solver *s, double wdt, const double *b,
                                      const double *hstar, const double *Yp, const double *Tp,
                                      const double *FRp, const double *hp, int n, void *X,
                                      double *scale, void *stream) {
  misdc_status st = sg_ready(s, false);
  if (st) return st;
  if (!b || !hstar || !Yp || !Tp || !FRp || !hp || !X || !scale || n < 0 || !(wdt > 0.0))
    return fail(MISDC_E_INVALID, "bad argument");
  mlp_features(s->m, n, n, wdt, b, hstar, Yp, Tp, FRp, hp, s->sg->ldx, (__nv_bfloat16 *)X, scale,
               0.0, nullptr, 0, nullptr, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return MISDC_OK;
}

misdc_status misdc_surrogate_forward(misdc_solver *s, const void *X, int n, float *out,
                                     void *stream) {
  misdc_status st = sg_ready(s, true);
  if (st) return st;
  if (!X || !out || n < 0) return fail(MISDC_E_INVALID, "bad argument");
  if (n == 0) return MISDC_OK;
  cudaError_t e = s->sg->ensure_inference(n);
  if (e != cudaSuccess) return fail(MISDC_E_OOM, cudaGetErrorString(e));
  cudaStream_t us = (cudaStream_t)stream;
  mlp_fused_forward(*s->sg, nullptr, 0, 0.0, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                    nullptr, (const __nv_bfloat16 *)X, n, out, us);
  CK(cudaGetLastError());
  return sg_check_err(s, us);
}

misdc_status misdc_surrogate_forward_layers(misdc_solver *s, const void *X, int n, float *out,
                                            void *stream) {
  misdc_status st = sg_ready(s, true);
  if (st) return st;
  if (!X || !out || n < 0) return fail(MISDC_E_INVALID, "bad argument");
  if (n == 0) return MISDC_OK;
  cudaError_t e = s->sg->ensure_inference(n);
  if (e != cudaSuccess) return fail(MISDC_E_OOM, cudaGetErrorString(e));
  cudaStream_t us = (cudaStream_t)stream;
  s->sg->forward((const __nv_bfloat16 *)X, n, out, false, us);
  CK(cudaGetLastError());
  return sg_check_err(s, us);
}

misdc_status misdc_surrogate_guess(misdc_solver *s, double wdt, const double *b, const double *hstar,
                                   const double *Yp, const double *Tp, const double *FRp,
                                   const double *hp, int n, float *out, double *scale, void *stream) {
  misdc_status st = sg_ready(s, true);
  if (st) return st;
  if (!b || !hstar || !Yp || !Tp || !FRp || !hp || !out || !scale || n < 0 || !(wdt > 0.0))
    return fail(MISDC_E_INVALID, "bad argument");
  if (n == 0) return MISDC_OK;
  cudaStream_t us = (cudaStream_t)stream;
  mlp_fused_forward(*s->sg, &s->m, n, wdt, b, hstar, Yp, Tp, FRp, hp, scale, nullptr, n, out, us);
  CK(cudaGetLastError());
  return sg_check_err(s, us);
}

misdc_status misdc_surrogate_gradient(misdc_solver *s, const void *X, const float *targets, int n,
                                      float *grad, float *loss, void *stream) {
  misdc_status st = sg_ready(s, true);
  if (st) return st;
  if (!X || !targets || n <= 0) return fail(MISDC_E_INVALID, "bad argument");
  Surrogate &g = *s->sg;
  cudaError_t e = g.ensure_training(n, 1);
  if (e != cudaSuccess) return fail(MISDC_E_OOM, cudaGetErrorString(e));
  cudaStream_t us = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(g.Yt, targets, (size_t)n * g.ldo * sizeof(float), cudaMemcpyDeviceToDevice, us));
  CK(cudaMemsetAsync(g.loss, 0, sizeof(float), us));
  g.forward((const __nv_bfloat16 *)X, n, g.Ot, true, us);
  g.backward((const __nv_bfloat16 *)X, n, g.loss, us);
  if (grad) CK(cudaMemcpyAsync(grad, g.G, g.n_params * sizeof(float), cudaMemcpyDeviceToDevice, us));
  if (loss) CK(cudaMemcpyAsync(loss, g.loss, sizeof(float), cudaMemcpyDeviceToDevice, us));
  CK(cudaGetLastError());
  return sg_check_err(s, us);
}

misdc_status misdc_surrogate_train_batch(misdc_solver *s, const void *X, const float *targets, int n,
                                         double lr, double weight_decay, float *loss, void *stream) {
  misdc_status st = misdc_surrogate_gradient(s, X, targets, n, nullptr, loss, stream);
  if (st) return st;
  s->sg->adamw((float)lr, (float)weight_decay, (cudaStream_t)stream);
  CK(cudaGetLastError());
  return MISDC_OK;
}

misdc_status misdc_surrogate_train(misdc_solver *s, int steps, int batch, double lr,
                                   double weight_decay, unsigned long long seed,
                                   float *loss_curve) {
  misdc_status st = sg_ready(s, true);
  if (st) return st;
  if (steps <= 0 || batch <= 0 || !(lr > 0.0) || !(weight_decay >= 0.0))
    return fail(MISDC_E_INVALID, "bad argument");
  long long rows = 0;
  if ((st = misdc_surrogate_dataset(s, &rows, nullptr, nullptr))) return st;
  if (rows <= 0) return fail(MISDC_E_INVALID, "no recorded solves to train on");
  Surrogate &g = *s->sg;
  cudaError_t e = g.ensure_training(batch, steps);
  if (e != cudaSuccess) return fail(MISDC_E_OOM, cudaGetErrorString(e));
  cudaStream_t us = s->sD;
  CK(cudaMemsetAsync(g.loss, 0, (size_t)steps * sizeof(float), us));
  for (int t = 0; t < steps; ++t) {
    // cosine decay of the learning rate to 5% of lr
    const double lrt = lr * std::max(0.05, 0.5 * (1.0 + cos(M_PI * t / steps)));
    mlp_gather(batch, rows, seed + (unsigned long long)t * (unsigned long long)batch, g.ldx, g.ldo,
               g.DX, g.DT, g.Xt, g.Yt, us);
    g.forward(g.Xt, batch, g.Ot, true, us);
    g.backward(g.Xt, batch, g.loss + t, us);
    g.adamw((float)lrt, (float)weight_decay, us);
  }
  CK(cudaGetLastError());
  if (loss_curve)
    CK(cudaMemcpyAsync(loss_curve, g.loss, (size_t)steps * sizeof(float), cudaMemcpyDeviceToHost, us));
  return sg_check_err(s, us);
}

}  // extern "C"

// ===========================================================================
// Autotuner of the launch shapes, and batched stepping of many flames
// ===========================================================================
namespace {

// time one enqueue (ms) with events on the stream
template <typename F>
float time_ms(cudaStream_t st, cudaEvent_t a, cudaEvent_t b, F &&f) {
  cudaEventRecord(a, st);
  f();
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, a, b);
  return ms;
}

}  // namespace

struct misdc_batch {
  std::vector<misdc_solver *> sv;
  cudaStream_t cs = nullptr;
  cudaEvent_t evIn = nullptr, evOut = nullptr, evFork = nullptr;
  std::vector<cudaEvent_t> evDone;
  cudaGraphExec_t gexec = nullptr;
  std::vector<double *> g_state, g_T;
  std::vector<double> g_dt;
  long long kernels_per_step = 0, kernels_launched = 0;
  // grouped reaction steps: the job tables and work counters of the current graph
  bool group = true;
  int grouped_launches = 0, grouped_solves = 0;
  NewtonArgs *d_jobs = nullptr;
  int *d_counters = nullptr;
};

namespace {

void free_groups(misdc_batch *b) {
  if (b->d_jobs) cudaFree(b->d_jobs);
  if (b->d_counters) cudaFree(b->d_counters);
  b->d_jobs = nullptr;
  b->d_counters = nullptr;
  b->grouped_launches = b->grouped_solves = 0;
}

// Nodes of g in a topological order (empty if g has a cycle or cannot be read).
std::vector<cudaGraphNode_t> topo_order(cudaGraph_t g) {
  size_t nn = 0, ne = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess) return {};
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn && cudaGraphGetNodes(g, nodes.data(), &nn) != cudaSuccess) return {};
  if (cudaGraphGetEdges(g, nullptr, nullptr, nullptr, &ne) != cudaSuccess) return {};
  std::vector<cudaGraphNode_t> from(ne), to(ne);
  if (ne && cudaGraphGetEdges(g, from.data(), to.data(), nullptr, &ne) != cudaSuccess) return {};
  std::unordered_map<cudaGraphNode_t, int> id;
  for (size_t i = 0; i < nn; ++i) id[nodes[i]] = (int)i;
  std::vector<int> indeg(nn, 0), head(nn, -1), nxt(ne), dst(ne);
  for (size_t e = 0; e < ne; ++e) {
    const int a = id[from[e]], c = id[to[e]];
    dst[e] = c;
    nxt[e] = head[a];
    head[a] = (int)e;
    ++indeg[c];
  }
  std::vector<int> queue;
  for (size_t i = 0; i < nn; ++i)
    if (!indeg[i]) queue.push_back((int)i);
  std::vector<cudaGraphNode_t> out;
  for (size_t q = 0; q < queue.size(); ++q) {
    const int a = queue[q];
    out.push_back(nodes[a]);
    for (int e = head[a]; e >= 0; e = nxt[e])
      if (--indeg[dst[e]] == 0) queue.push_back(dst[e]);
  }
  if (out.size() != nn) out.clear();
  return out;
}

// Replace the k-th reaction-Newton launch of every flame by one grouped launch
// per mechanism shape (k_newton2_group). Returns false, with g unchanged, when the
// flames do not qualify; an error after g was changed is reported as such.
misdc_status group_newton(misdc_batch *b, cudaGraph_t g, bool *changed) {
  *changed = false;
  const int n = (int)b->sv.size();
  if (n < 2) return MISDC_OK;
  for (misdc_solver *s : b->sv)
    if (s->nu_bits || step_lanes(s) != 1) return MISDC_OK;   // steps not in one sequence
  std::vector<cudaGraphNode_t> order = topo_order(g);
  if (order.empty()) return MISDC_OK;
  struct Member {
    cudaGraphNode_t node;
    NewtonArgs a;
    bool mixed;
    cudaKernelNodeParams p;
  };
  std::vector<std::vector<Member>> per(n);
  for (cudaGraphNode_t nd : order) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams p{};
    if (cudaGraphKernelNodeGetParams(nd, &p) != cudaSuccess || !p.kernelParams) continue;
    Member mb{nd, NewtonArgs{}, false, p};
    if (!newton_kernel_args(p.func, p.kernelParams, &mb.a, &mb.mixed)) continue;
    int f = -1;
    for (int i = 0; i < n && f < 0; ++i)
      if (b->sv[i]->st == mb.a.st) f = i;
    if (f < 0) return MISDC_OK;
    per[f].push_back(mb);
  }
  const size_t K = per[0].size();
  for (int i = 1; i < n; ++i)
    if (per[i].size() != K) return MISDC_OK;
  if (K == 0) return MISDC_OK;
  // the groups: per stage, flames of one key (kernel, N, R, ld, block, shared memory)
  std::vector<std::vector<int>> groups;   // member flames
  std::vector<size_t> stage_of;
  for (size_t k = 0; k < K; ++k) {
    std::vector<bool> used(n, false);
    for (int i = 0; i < n; ++i) {
      if (used[i]) continue;
      const Member &x = per[i][k];
      std::vector<int> grp{i};
      used[i] = true;
      for (int j = i + 1; j < n; ++j) {
        const Member &y = per[j][k];
        if (!used[j] && y.mixed == x.mixed && y.a.m.N == x.a.m.N && y.a.m.R == x.a.m.R &&
            y.a.ld == x.a.ld && y.p.blockDim.x == x.p.blockDim.x &&
            y.p.sharedMemBytes == x.p.sharedMemBytes && (int)grp.size() < kMaxGroupJobs) {
          grp.push_back(j);
          used[j] = true;
        }
      }
      if (grp.size() >= 2) {
        groups.push_back(grp);
        stage_of.push_back(k);
      }
    }
  }
  if (groups.empty()) return MISDC_OK;
  size_t jobs = 0;
  for (auto &gr : groups) jobs += gr.size();
  if (cudaMalloc(&b->d_jobs, jobs * sizeof(NewtonArgs)) != cudaSuccess ||
      cudaMalloc(&b->d_counters, groups.size() * sizeof(int)) != cudaSuccess) {
    free_groups(b);
    return fail(MISDC_E_OOM, "grouped reaction steps: job tables");
  }
  std::vector<NewtonArgs> host(jobs);
  size_t j0 = 0;
  *changed = true;
  for (size_t q = 0; q < groups.size(); ++q) {
    const std::vector<int> &gr = groups[q];
    const size_t k = stage_of[q];
    const Member &x = per[gr[0]][k];
    std::vector<cudaGraphNode_t> deps, outs;
    long long items = 0;
    for (size_t t = 0; t < gr.size(); ++t) {
      const Member &mb = per[gr[t]][k];
      host[j0 + t] = mb.a;
      items += mb.a.n;
      size_t nd = 0, no = 0;
      cudaGraphNodeGetDependencies(mb.node, nullptr, nullptr, &nd);
      cudaGraphNodeGetDependentNodes(mb.node, nullptr, nullptr, &no);
      std::vector<cudaGraphNode_t> d(nd), o(no);
      if ((nd && cudaGraphNodeGetDependencies(mb.node, d.data(), nullptr, &nd) != cudaSuccess) ||
          (no && cudaGraphNodeGetDependentNodes(mb.node, o.data(), nullptr, &no) != cudaSuccess))
        return fail(MISDC_E_CUDA, "grouped reaction steps: graph edges");
      deps.insert(deps.end(), d.begin(), d.end());
      outs.insert(outs.end(), o.begin(), o.end());
    }
    std::sort(deps.begin(), deps.end());
    deps.erase(std::unique(deps.begin(), deps.end()), deps.end());
    std::sort(outs.begin(), outs.end());
    outs.erase(std::unique(outs.begin(), outs.end()), outs.end());
    for (int f : gr)
      if (cudaGraphDestroyNode(per[f][k].node) != cudaSuccess)
        return fail(MISDC_E_CUDA, "grouped reaction steps: removing a launch");
    cudaMemsetParams ms{};
    ms.dst = b->d_counters + q;
    ms.value = 0;
    ms.elementSize = sizeof(int);
    ms.width = 1;
    ms.height = 1;
    cudaGraphNode_t mnode, knode;
    if (cudaGraphAddMemsetNode(&mnode, g, deps.data(), deps.size(), &ms) != cudaSuccess)
      return fail(MISDC_E_CUDA, "grouped reaction steps: counter reset");
    const size_t smem = x.p.sharedMemBytes;
    const void *fn = newton_group_kernel(x.mixed);
    newton_group_reserve_smem(x.mixed, smem);
    NewtonArgs *jp = b->d_jobs + j0;
    int nj = (int)gr.size();
    int *cp = b->d_counters + q;
    void *args[3] = {&jp, &nj, &cp};
    cudaKernelNodeParams kp{};
    kp.func = (void *)fn;
    kp.blockDim = x.p.blockDim;
    kp.gridDim = dim3(newton_group_grid(x.mixed, (int)(x.p.blockDim.x / 32), smem,
                                        (int)std::min<long long>(items, 1 << 30)));
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    if (cudaGraphAddKernelNode(&knode, g, &mnode, 1, &kp) != cudaSuccess)
      return fail(MISDC_E_CUDA, "grouped reaction steps: grouped launch");
    for (cudaGraphNode_t o : outs)
      if (cudaGraphAddDependencies(g, &knode, &o, nullptr, 1) != cudaSuccess)
        return fail(MISDC_E_CUDA, "grouped reaction steps: graph edges");
    j0 += gr.size();
    b->grouped_launches += 1;
    b->grouped_solves += (int)gr.size();
  }
  if (cudaMemcpy(b->d_jobs, host.data(), jobs * sizeof(NewtonArgs), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(MISDC_E_CUDA, "grouped reaction steps: job tables");
  if (topo_order(g).empty()) return fail(MISDC_E_CUDA, "grouped reaction steps: the graph has a cycle");
  return MISDC_OK;
}

}  // namespace

extern "C" {

misdc_status misdc_get_tuning(misdc_solver *s, misdc_tuning *t) {
  if (!s || !t) return fail(MISDC_E_INVALID, "null argument");
  memset(t, 0, sizeof(*t));
  t->newton_warps_per_block = s->nl.wpb;
  t->newton_blocks_per_sm = s->nl.blocks_per_sm;
  t->newton_dynamic = s->nl.dynamic;
  t->cheb_block = s->dw.cheb_block;
  t->newton_keep_factors = s->keep_factors ? 1 : 0;
  t->newton_chord_iters = s->nl.chord_iters;
  return MISDC_OK;
}

misdc_status misdc_set_tuning(misdc_solver *s, const misdc_tuning *t) {
  if (!s || !t) return fail(MISDC_E_INVALID, "null argument");
  if (t->newton_warps_per_block < 0 || t->newton_warps_per_block > 4 || t->newton_blocks_per_sm < 0 ||
      t->newton_blocks_per_sm > 32 || t->newton_chord_iters < 0 || t->newton_chord_iters > 16 ||
      (t->cheb_block && (t->cheb_block < 32 || t->cheb_block > 1024 ||
                                                         t->cheb_block % 32)))
    return fail(MISDC_E_INVALID, "tuning out of range");
  drop_graph(s);
  s->nl.wpb = t->newton_warps_per_block;
  s->nl.blocks_per_sm = t->newton_blocks_per_sm;
  s->nl.dynamic = t->newton_dynamic ? 1 : 0;
  s->dw.cheb_block = t->cheb_block;
  s->nl.chord_iters = t->newton_chord_iters;
  for (auto &L : s->lane) L.nl.chord_iters = t->newton_chord_iters;
  if (s->keep_factors != (t->newton_keep_factors != 0)) {
    s->keep_factors = t->newton_keep_factors != 0;
    for (int j = 1; j <= s->tab.M; ++j)
      if (s->cst[j].valid) cudaMemset(s->cst[j].valid, 0, (size_t)s->cs * sizeof(int));
  }
  return MISDC_OK;
}

misdc_status misdc_autotune(misdc_solver *s, const double *state, const double *T, double dt,
                            misdc_tuning *out) {
  if (!s || !state || !T) return fail(MISDC_E_INVALID, "null argument");
  if (!(dt > 0.0)) return fail(MISDC_E_INVALID, "dt must be > 0");
  configure_dt(s, dt);
  const size_t cs = s->cs, N = s->N, F = N + 1;
  cudaStream_t st = s->sD;
  CK(cudaStreamSynchronize(s->sD));
  CK(cudaStreamSynchronize(s->sR));
  double *x = nullptr, *x0 = nullptr, *FR = nullptr, *hsp = nullptr, *th = nullptr, *out_s = nullptr;
  double *Ts = nullptr, *theta = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  auto cleanup = [&]() {
    for (double *p : {x, x0, FR, hsp, th, out_s, Ts, theta}) if (p) cudaFree(p);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  };
  if (cudaMalloc(&x, F * cs * 8) || cudaMalloc(&x0, F * cs * 8) || cudaMalloc(&FR, N * cs * 8) ||
      cudaMalloc(&hsp, N * cs * 8) || cudaMalloc(&th, cs * 8) || cudaMalloc(&out_s, F * cs * 8) ||
      cudaMalloc(&Ts, cs * 8) || cudaMalloc(&theta, cs * 8) || cudaEventCreate(&a) ||
      cudaEventCreate(&b)) {
    cleanup();
    return fail(MISDC_E_OOM, "autotune scratch");
  }
  // the reaction step of the largest implicit weight from the given state:
  // b = Y, h* = h, guess (Y, T)
  double wdt = 0.0;
  for (int t = 0; t < s->tab.M; ++t) wdt = std::max(wdt, dt * s->tab.QI[t][t]);
  cudaMemcpyAsync(x0, state, N * cs * 8, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(x0 + N * cs, T, cs * 8, cudaMemcpyDeviceToDevice, st);
  const bool mixed = s->o.precision == MISDC_PREC_MIXED;
  const int wmax = newton_max_wpb(s->m, mixed);
  NewtonLaunch best = s->nl;
  float best_ms = 1e30f;
  auto run = [&](const NewtonLaunch &c) {
    cudaMemcpyAsync(x, x0, F * cs * 8, cudaMemcpyDeviceToDevice, st);
    return time_ms(st, a, b, [&] {
      launch_newton(s->m, (int)cs, (int)cs, wdt, s->o.newton_rtol, s->o.newton_maxit, state,
                    state + N * cs, x, x + N * cs, x, x + N * cs, FR, hsp, th, nullptr, s->st, st,
                    mixed, nullptr, 0, nullptr, 0.0, nullptr, nullptr, &c);
    });
  };
  // candidates (warps per block, blocks per SM, dynamic): the default shape, then
  // dynamic scheduling at 16 resident warps per SM in blocks of 4, 2 and 1 warps
  const int cand[][3] = {{0, 0, 0}, {4, 4, 1}, {2, 8, 1}, {1, 16, 1}, {2, 8, 0}, {1, 16, 0}};
  {
    NewtonLaunch c = s->nl;
    c.wpb = 0; c.blocks_per_sm = 0; c.dynamic = 0;
    run(c);   // warm-up
  }
  for (const auto &cd : cand) {
    if (cd[0] > wmax) continue;
    NewtonLaunch c = s->nl;
    c.wpb = cd[0]; c.blocks_per_sm = cd[1]; c.dynamic = cd[2];
    const float ms = run(c);
    if (ms < best_ms) { best_ms = ms; best = c; }
  }
  // smoother block size on a diffusion solve of the same size, coefficients at the state
  launch_temperature(s->m, (int)cs, (int)cs, state, state + N * cs, T, Ts, theta, hsp, s->st, st);
  int best_tb = 256;
  float best_d = 1e30f;
  for (int tb : {128, 256, 512}) {
    s->dw.cheb_block = tb;
    float ms = 0.0f;
    for (int rep = 0; rep < 2; ++rep) {
      const float t1 = time_ms(st, a, b, [&] {
        diffusion_solve(s->m, s->g, s->i0, wdt, theta, state, out_s, s->dw, s->cheb_sweeps,
                        s->rho_bound, s->o.lin_rtol, s->st, st);
      });
      if (rep) ms += t1;
    }
    if (ms < best_d) { best_d = ms; best_tb = tb; }
  }
  cudaError_t e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return fail(MISDC_E_CUDA, cudaGetErrorString(e));
  CK(cudaMemset(s->st, 0, sizeof(DevStats)));
  drop_graph(s);
  s->nl = best;
  s->dw.cheb_block = best_tb;
  if (out) {
    misdc_get_tuning(s, out);
    out->newton_ms = best_ms;
    out->cheb_ms = best_d;
  }
  return MISDC_OK;
}

misdc_status misdc_batch_create(misdc_solver *const *solvers, int n, misdc_batch **out) {
  if (!solvers || n <= 0 || !out) return fail(MISDC_E_INVALID, "bad argument");
  for (int i = 0; i < n; ++i) {
    if (!solvers[i]) return fail(MISDC_E_INVALID, "null solver");
    for (int j = 0; j < i; ++j)
      if (solvers[j] == solvers[i]) return fail(MISDC_E_INVALID, "a solver appears twice");
  }
  misdc_batch *b = new misdc_batch();
  b->sv.assign(solvers, solvers + n);
  b->evDone.assign(n, nullptr);
  bool ok = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->evIn, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->evOut, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&b->evFork, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < n; ++i)
    ok = cudaEventCreateWithFlags(&b->evDone[i], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    misdc_batch_destroy(b);
    return fail(MISDC_E_CUDA, "batch streams/events");
  }
  *out = b;
  return MISDC_OK;
}

void misdc_batch_destroy(misdc_batch *b) {
  if (!b) return;
  if (b->cs) cudaStreamSynchronize(b->cs);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  free_groups(b);
  for (cudaEvent_t e : b->evDone) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : {b->evIn, b->evOut, b->evFork}) if (e) cudaEventDestroy(e);
  if (b->cs) cudaStreamDestroy(b->cs);
  delete b;
}

misdc_status misdc_batch_step(misdc_batch *b, double *const *states, double *const *T,
                              const double *dts, int n_steps, void *stream) {
  if (!b || !states || !dts || n_steps < 0) return fail(MISDC_E_INVALID, "bad argument");
  const int n = (int)b->sv.size();
  for (int i = 0; i < n; ++i) {
    if (!states[i] || !(dts[i] > 0.0)) return fail(MISDC_E_INVALID, "bad state or dt");
    if (b->sv[i]->sg_collect) return fail(MISDC_E_INVALID, "batched steps do not record solves");
  }
  if (n_steps == 0) return MISDC_OK;
  bool stale = !b->gexec;
  for (int i = 0; i < n && !stale; ++i)
    stale = b->g_state[i] != states[i] || b->g_T[i] != (T ? T[i] : nullptr) || b->g_dt[i] != dts[i];
  if (stale) {
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    free_groups(b);
    for (int i = 0; i < n; ++i) configure_dt(b->sv[i], dts[i]);
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(b->cs, cudaStreamCaptureModeThreadLocal));
    cudaEventRecord(b->evFork, b->cs);
    for (int i = 0; i < n; ++i) {
      misdc_solver *s = b->sv[i];
      s->n_used = s->d_used = 0;
      cudaStreamWaitEvent(s->sD, b->evFork, 0);
      enqueue_step(s, states[i], T ? T[i] : nullptr, dts[i]);
      cudaEventRecord(b->evDone[i], s->sD);
      cudaStreamWaitEvent(b->cs, b->evDone[i], 0);
    }
    cudaError_t ec = cudaStreamEndCapture(b->cs, &graph);
    if (ec != cudaSuccess) return fail(MISDC_E_CUDA, std::string("batch capture: ") + cudaGetErrorString(ec));
    if (b->group) {
      bool changed = false;
      const misdc_status gs = group_newton(b, graph, &changed);
      if (gs != MISDC_OK) {
        cudaGraphDestroy(graph);
        free_groups(b);
        return gs;
      }
    }
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(graph, nodes.data(), &nn);
    b->kernels_per_step = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      cudaGraphNodeGetType(nd, &ty);
      if (ty == cudaGraphNodeTypeKernel) ++b->kernels_per_step;
    }
    ec = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ec != cudaSuccess) return fail(MISDC_E_CUDA, std::string("batch instantiate: ") + cudaGetErrorString(ec));
    for (misdc_solver *s : b->sv)
      if (s->nu_flags) CK(cudaMemcpy(s->nu_flags + 2, &s->nu_body_kernels, sizeof(int), cudaMemcpyHostToDevice));
    b->g_state.assign(states, states + n);
    b->g_T.assign(n, nullptr);
    if (T) b->g_T.assign(T, T + n);
    b->g_dt.assign(dts, dts + n);
  }
  cudaStream_t us = (cudaStream_t)stream;
  CK(cudaEventRecord(b->evIn, us));
  CK(cudaStreamWaitEvent(b->cs, b->evIn, 0));
  for (int k = 0; k < n_steps; ++k) CK(cudaGraphLaunch(b->gexec, b->cs));
  for (misdc_solver *s : b->sv)
    if (s->o.scheme == MISDC_SCHEME_CISDCQ && !s->nu_bits)
      s->nested_host += (long long)n_steps * s->o.n_sweeps * s->o.nu;
  b->kernels_launched += b->kernels_per_step * n_steps;
  CK(cudaEventRecord(b->evOut, b->cs));
  CK(cudaStreamWaitEvent(us, b->evOut, 0));
  return MISDC_OK;
}

misdc_status misdc_batch_set_grouping(misdc_batch *b, int on) {
  if (!b) return fail(MISDC_E_INVALID, "null batch");
  if ((on != 0) != b->group) {
    if (b->cs) CK(cudaStreamSynchronize(b->cs));
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    free_groups(b);
    b->group = on != 0;
  }
  return MISDC_OK;
}

misdc_status misdc_batch_grouping(misdc_batch *b, int *grouped_launches, int *grouped_solves) {
  if (!b) return fail(MISDC_E_INVALID, "null batch");
  if (grouped_launches) *grouped_launches = b->grouped_launches;
  if (grouped_solves) *grouped_solves = b->grouped_solves;
  return MISDC_OK;
}

misdc_status misdc_batch_stats(misdc_batch *b, misdc_stats *out, int reset) {
  if (!b || !out) return fail(MISDC_E_INVALID, "null argument");
  CK(cudaStreamSynchronize(b->cs));
  misdc_stats sum;
  memset(&sum, 0, sizeof(sum));
  for (misdc_solver *s : b->sv) {
    misdc_stats t;
    misdc_status st = misdc_get_stats(s, &t, reset);
    if (st) return st;
    sum.newton_solves += t.newton_solves;
    sum.newton_iters += t.newton_iters;
    sum.newton_fail += t.newton_fail;
    sum.newton_max = std::max(sum.newton_max, t.newton_max);
    if (!sum.status) sum.status = t.status;
    sum.lin_sweeps += t.lin_sweeps;
    sum.lin_resid_max = std::max(sum.lin_resid_max, t.lin_resid_max);
    sum.surrogate_used += t.surrogate_used;
    sum.surrogate_rejected += t.surrogate_rejected;
    sum.newton_fp64_fallbacks += t.newton_fp64_fallbacks;
    sum.newton_jacobians += t.newton_jacobians;
    sum.newton_lu_fp64 += t.newton_lu_fp64;
    sum.newton_certified += t.newton_certified;
    sum.newton_stored_steps += t.newton_stored_steps;
    sum.newton_floor_stops += t.newton_floor_stops;
    sum.newton_chord_cells += t.newton_chord_cells;
    sum.kernel_launches += t.kernel_launches;   // kernels in conditional bodies
    sum.nested_iterations += t.nested_iterations;
  }
  sum.kernel_launches += b->kernels_launched;
  if (reset) b->kernels_launched = 0;
  *out = sum;
  return MISDC_OK;
}

}  // extern "C"
