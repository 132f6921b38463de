// Internal declarations shared by the CUDA translation units of libmisdc.
// Not part of the C ABI (see include/misdc.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/misdc.h"

namespace misdc {

constexpr double kRu = 8.314462618;        // J/(mol K)
constexpr double kTlo = 50.0, kThi = 6000.0;   // temperature range of the one-range polynomials
constexpr int kMaxSlots = 3;               // molecules per reaction side
constexpr int kMaxSpecies = 63;
constexpr int kMaxNodes = 9;
constexpr int kMaxCheb = 512;   // cap on Chebyshev sweeps per diffusion solve
constexpr int kMaxLanes = 4;    // stream pairs for the nested iterations of CISDCQ

// Device status bits (OR-ed into DevStats::status_bits); mapped to misdc_status
enum : unsigned {
  kBitNewton = 1u, kBitSingular = 2u, kBitNan = 4u, kBitTdiag = 8u, kBitMG = 16u, kBitTimeout = 32u
};

struct DevStats {
  unsigned long long newton_solves;
  unsigned long long newton_iters;
  unsigned long long newton_fail;
  unsigned long long lin_sweeps;
  int newton_max;
  unsigned status_bits;
  unsigned long long lin_resid_bits;   // bit pattern of the largest relative residual (>= 0)
  unsigned long long sg_used;          // cells that started Newton from the learned guess
  unsigned long long sg_rejected;      // learned guesses rejected by the residual test
  unsigned long long fp64_fallbacks;   // mixed-precision solves restarted with FP64 Newton
  unsigned long long jacobians;        // Jacobian assemblies of the reaction Newton
  unsigned long long lu64;             // FP64 LU factorisations of the reaction Newton
  unsigned long long certified;        // solves whose guess was certified without rates
  unsigned long long stored_steps;     // first chord steps taken from the stored reaction term
  unsigned long long body_launches;    // kernels run inside conditional graph bodies
  unsigned long long nested_iters;     // CISDCQ nested iterations run, summed over sweeps
  unsigned long long floor_stops;      // exact Newton solves that ended on the round-off-floor test
  unsigned long long chord_cells;      // solves finished by the thread-per-cell chord pass
};

// Mechanism tables in device memory (built by the engine from misdc_mech_desc).
struct DevMech {
  int N, R;
  double rho, T_ref, theta_exp, alpha0, ln_p_over_R, ln_Tref;
  const double *invW;      // [N] 1/W
  const double *W;         // [N] W (kg/mol)
  const double *hcoef;     // [N][6]  a1, a2/2, a3/3, a4/4, a5/5, a6      (h/RT = poly + a6/T)
  const double *scoef;     // [N][6]  a1, a2, a3/2, a4/3, a5/4, a7        (s/R = a1 lnT + poly + a7)
  const double *cpcoef;    // [N][5]  a1..a5                                (cp/R)
  const double *D0;        // [N]
  const double *lnA, *beta, *TA, *dn;   // [R]   TA = Ea/R_u, dn = sum of net nu
  const signed char *fwd, *rev;         // [R][3] species of each molecule slot, -1 empty
  const int *sp_ptr;       // [N+1]  CSR of the reactions each species takes part in
  const int *sp_rx;        // [nnz]
  const double *sp_coef;   // [nnz]  W_i * nu_ri
  const double *D0_host;   // [N] host copy (launch parameters)
  // reaction-Newton assembly list: entry p adds -wdt * jc_w[p] * src[jc_pack[p] & 0xffff] to
  // J[jc_pack[p] >> 16]; entries sorted by target and cut into 32 lane segments jc_seg[0..32]
  const int *jc_pack;
  const double *jc_w;
  const int *jc_seg;
  // production rates on the FP64 tensor cores (mma m8n8k4): the nonzero tiles of
  // the (R x N) matrix [W_i nu_ri], 4 reactions by 8 species each, listed per
  // species tile (CSR mma_ptr over mma_nt species tiles, reaction block mma_kb);
  // tile p's B fragment is mma_b[32 p + lane] = entry (4 kb + lane % 4, 8 j + lane / 4)
  const double *mma_b;
  const int *mma_ptr, *mma_kb;
  int mma_nt, mma_ntiles;
};

// row stride (doubles) of the per-cell reaction rates staged for the tensor-core
// contraction: R rounded up to 4, then to 4 (mod 16) so the A-fragment loads of a
// half-warp (8 cells x 4 reactions) fall in distinct shared-memory banks
__host__ __device__ inline int mma_qld(int R) {
  const int r = (R + 3) & ~3;
  return r + ((4 - (r & 15)) & 15);
}

// leading dimension of the augmented (N+1) x (N+2) Newton matrix in shared memory (odd)
__host__ __device__ inline int newton_ld(int N) {
  int ld = N + 2;
  return (ld & 1) ? ld : ld + 1;
}

struct DevGrid {
  int dim, nx, ny, nz, cells;
  double dx;
};

// ---- chemistry kernels (misdc_chem.cu) ----
void launch_temperature(const DevMech &m, int n, int cs, const double *Y, const double *h,
                        const double *Tguess, double *T, double *theta, double *hsp,
                        DevStats *st, cudaStream_t s);
void launch_enthalpy(const DevMech &m, int n, int cs, const double *Y, const double *T,
                     double *h, cudaStream_t s);
void launch_rates(const DevMech &m, int n, int cs, const double *Y, const double *T,
                  double *FR, cudaStream_t s, bool mma = false);
// Reaction Newton (S5). b [N][cs], hstar [cs], guess Yg [N][cs], Tg [cs];
// outputs Y, T, FR (wdot/rho at the solution), hsp [N][cs] and theta at the solution.
// pred [.][ldp] (optional): learned correction, row prow[c] of cell c (prow NULL: row c;
// negative: none), applied to cells with sc[c] > s_min as
// x0 = x_p + sc p (T scaled by T_p) and kept only if the Jacobi-scaled residual at x0 is
// below that at the guess x_p, whose reaction term FRp [N][cs] and enthalpy hp [cs] give
// its residual without a rate evaluation. Mixed precision with a kept factor: a guess
// certified converged from FRp and hp alone is returned as is, with the guess's species
// enthalpies hspp [N][cs] and theta thp [cs].
// Launch shape of the reaction Newton (chosen by the autotuner): warps per block
// (0: largest that fits), resident-block cap per SM (0: default), and dynamic
// cell scheduling through the device counter `work`.
// list / list_n (mixed precision with kept factors): scratch of cs + 1 ints for the
// cells a kept factor did not certify, which the warp-per-cell kernel then takes.
struct NewtonLaunch {
  int wpb = 0, blocks_per_sm = 0, dynamic = 0;
  int *work = nullptr;
  int *list = nullptr, *list_n = nullptr;
  bool precertified = false;   // launch_certify has run: the Newton kernel takes the list
  int chord_iters = 4;         // chord iterations of the thread-per-cell pass (0: certification only)
  int *list2 = nullptr, *list2_n = nullptr;   // the cells the chord pass leaves
};
// Mixed precision: per-cell Jacobian factors kept between the solves of one SDC
// node. Per cell: fs doubles (row-major LU of the (row-scaled) (N+1)^2 Jacobian,
// pivot reciprocals, row scales, the temperature-row scale, an FP32-built flag, the
// state it was built at) and swld bytes of pivot rows; valid[c] bit 0: the factor
// may be used, bit 1: FP32 factors are too coarse for this cell.
// z32 (optional): the kept inverse rounded to FP32, element-major ([e][cs] with
// e = j (N+1) + i for entry (i, j)), which certifies converged guesses on the FP32
// pipe, one thread per cell.
// xc [N+1][cs] and sT [cs] (optional, element-major): the state each factor was
// built at and its temperature-row scale, for the certification kernel; valid bit
// 2 marks a factor built in FP32.
struct ChordStore {
  double *f = nullptr;
  unsigned char *sw = nullptr;
  int *valid = nullptr;
  float *z32 = nullptr;
  double *xc = nullptr, *sT = nullptr;
  int fs = 0, swld = 0;
};
// Arguments of one reaction-Newton solve over n cells (k_newton2): the
// right-hand side b, the enthalpy h*, the guesses (Yg, Tg) and their stored
// reaction terms, species enthalpies and theta (FRp, hp, hspp, thp), the outputs,
// the learned guess (pred rows ldp apart, scale sc, threshold s_min, row map prow),
// the kept factors, the work counter and the list of cells the certification pass
// left (list, *list_n).
struct NewtonArgs {
  DevMech m;
  int n, cs;
  double wdt, rtol;
  int maxit, ld;
  const double *b, *hstar, *Yg, *Tg;
  double *Yout, *Tout, *FR, *hsp, *theta;
  int *iters;
  DevStats *st;
  const float *pred;
  int ldp;
  const double *sc;
  double s_min;
  const double *FRp, *hp;
  int *work;
  ChordStore cst;
  const int *prow;
  const double *hspp, *thp;
  const int *list, *list_n;
};
// solves one grouped Newton launch takes at most
constexpr int kMaxGroupJobs = 256;
__host__ __device__ inline int chord_floats(int N) {
  const int nn = N + 1;
  return (nn * nn + 3 * nn + 2 + 1) / 2 * 2;
}
// table of the FP64 exponential the rate kernels use (once per device, before any
// chemistry kernel runs), and that exponential over n elements
cudaError_t init_exp_table();
cudaError_t launch_exp(const double *x, double *y, size_t n, cudaStream_t s);
void launch_newton(const DevMech &m, int n, int cs, double wdt, double rtol, int maxit,
                   const double *b, const double *hstar, const double *Yg, const double *Tg,
                   double *Y, double *T, double *FR, double *hsp, double *theta, int *iters,
                   DevStats *st, cudaStream_t s, bool mixed = false,
                   const float *pred = nullptr, int ldp = 0, const double *sc = nullptr,
                   double s_min = 0.0, const double *FRp = nullptr, const double *hp = nullptr,
                   const NewtonLaunch *cfg = nullptr, const ChordStore *store = nullptr,
                   const int *prow = nullptr, const double *hspp = nullptr,
                   const double *thp = nullptr);
int newton_max_wpb(const DevMech &m, bool mixed);
// The certification pass of a mixed reaction step alone (the cells it leaves in
// cfg->list / cfg->list_n); launch_newton with cfg->precertified then takes the list.
// Returns false (and launches nothing) when the step has no kept factors to certify from.
bool launch_certify(const DevMech &m, int n, int cs, double wdt, double rtol, int maxit, const double *b,
                    const double *hstar, const double *Yg, const double *Tg, double *Y, double *T,
                    double *FR, double *hsp, double *theta, int *iters, DevStats *st,
                    const double *FRp, const double *hp, const ChordStore *store,
                    const double *hspp, const double *thp, NewtonLaunch *cfg, cudaStream_t s);

// Grouped reaction Newton (k_newton2_group): newton_kernel_args reads the
// arguments of a captured k_newton2 launch (false for any other kernel);
// newton_group_kernel is the grouped kernel; newton_group_grid its persistent grid
// for `items` work items at wpb warps per block and `smem` dynamic bytes.
bool newton_kernel_args(const void *func, void **params, NewtonArgs *out, bool *mixed);
const void *newton_group_kernel(bool mixed);
int newton_group_grid(bool mixed, int wpb, size_t smem, int items);
// raise the grouped kernel's dynamic shared-memory limit to at least smem (never lowers it)
void newton_group_reserve_smem(bool mixed, size_t smem);

// ---- grid kernels (misdc_grid.cu) ----
struct LinComb {
  int n_out, n_in;
  double *out[8];
  const double *in[16];
  double w[8][16];
};
void launch_lincomb(const LinComb &lc, size_t n, cudaStream_t s);
// faces: scratch of operator_face_doubles(g, N) doubles (the face fluxes of the
// two-pass operator kernels)
size_t operator_face_doubles(const DevGrid &g, int N);
void launch_operators(const DevMech &m, const DevGrid &g, int i0, const double *phi,
                      const double *hsp, const double *theta_face, const double *vel,
                      double *FE, double *FD, double *faces, cudaStream_t s);
// theta at cells -> theta at the low face of every cell (harmonic mean)
void launch_theta_faces(const DevGrid &g, const double *theta, double *thf, cudaStream_t s);
void prepare_chem_kernels(const DevMech &m);
// D-step solve of every field but i0: (I - c_f L_theta) x = rhs, Chebyshev-accelerated
// Jacobi (the multigrid smoother), optional V-cycles, reconstruction and closure.
struct DiffWork {
  double *thf;       // [dim][cs] face coefficients
  double *invdiag;   // [N+1][cs]
  double *cdiag, *bdiag;   // [N+1][cs] c_f / diagonal and rhs / diagonal (Chebyshev sweep)
  double *xa, *xb, *xc;   // [N+1][cs] iterates
  double *res;       // [N+1][cs] residual (multigrid)
  unsigned long long *rho_bits;   // measured Gershgorin bound (bit pattern)
  int *kdev;                      // planned Chebyshev sweep count
  double *omega;                  // [kMaxCheb] Chebyshev weights
  // multigrid levels (level 0 = this grid, compact [solved field][cells] storage)
  int levels, cycles;
  int cheb_block;   // threads per block of the Chebyshev sweep (autotuned; 0 = 256)
  // mixed precision: refinement rounds (0: plain FP64 Chebyshev) and FP32 work
  int refine_rounds;
  float *thf32, *invdiag32, *r32, *e32[3];
  int *kdev32;
  double *omega32;
  DevGrid lg[8];
  double *lthf[8], *linvdiag[8], *lb[8], *lx[8], *lr[8], *ly[8];
  // mixed precision: the coarse levels (l >= 1) in FP32 when mg32 is set
  int mg32;
  float *lthf32[8], *linvdiag32[8], *lb32[8], *lx32[8], *lr32[8], *ly32[8];
  // V-cycle stop: flag, largest scaled fine residual of the cycle (bit pattern),
  // its target and the statistics it is counted in (set per solve)
  int *mg_done, *mg_cycle;
  unsigned long long *mg_res;
  double mg_tol;
  DevStats *mg_st;
  // inside a stream capture the V-cycles become the body of a WHILE graph node,
  // captured on this private stream (null: unrolled cycles that skip once done)
  cudaStream_t mg_stream;
};

// Inside a stream capture on s: append a conditional node (IF or WHILE, default
// value dflt at every graph launch) after the stream's capture dependencies and
// make it the stream's only dependency. Returns the body graph to capture into,
// or nullptr when s is not capturing or the node could not be added.
cudaGraph_t graph_conditional(cudaStream_t s, cudaGraphConditionalNodeType type, unsigned dflt,
                              cudaGraphConditionalHandle *h);
// the two halves of graph_conditional, for a handle that a kernel captured before
// the node sets: create it on s's capture graph (false when s is not capturing),
// then add the node that uses it
bool graph_conditional_handle(cudaStream_t s, unsigned dflt, cudaGraphConditionalHandle *h);
cudaGraph_t graph_conditional_node(cudaStream_t s, cudaGraphConditionalNodeType type,
                                   cudaGraphConditionalHandle h);

// ---- adaptive nested iterations of a CISDCQ sweep (misdc_grid.cu) ----
// After nested iteration l: delta_l = max over fields of max|now - before| / max|now|
// over the nodes' cells (now/before: the node stacks of iterations l and l-1, node
// m at [m - 1], fields [F][cs]); delta[l] = delta_l; then the rule: continue while
// l + 1 < nu and (l < 1 or (delta_l > eta delta_0 and delta_l < rho delta_{l-1})).
// *cont = the decision, *ran = l + 1; the iterations run are added to st when the
// sweep's loop ends here; with a handle, the IF node of iteration l + 1 is set;
// body_kernels (inside an IF body): the body's kernel count, added to st.
struct NodePtrs {
  const double *p[kMaxNodes];
};
void launch_nu_decide(int F, int cs, int M, NodePtrs now, NodePtrs before, int l, int nu,
                      double eta, double rho, unsigned long long *bits, double *delta, int *cont,
                      int *ran, DevStats *st, const cudaGraphConditionalHandle *h,
                      const int *body_kernels, cudaStream_t s);
// dst[k] = src[k] (n[k] doubles each, k < count) when the parity of *ran - 1 differs
// from `parity` (the nested loop ended in the other buffer of the pair)
constexpr int kMaxCopies = 7 * kMaxNodes;
struct CopyList {
  double *dst[kMaxCopies];
  const double *src[kMaxCopies];
  size_t n[kMaxCopies];
  int count;
};
void launch_copy_if_parity(const CopyList &cl, const int *ran, int parity, cudaStream_t s);
void diffusion_solve(const DevMech &m, const DevGrid &g, int i0, double wdt, const double *theta,
                     const double *rhs, double *out, DiffWork &w, int sweeps, double rho_bound,
                     double lin_rtol, DevStats *st, cudaStream_t s);
int chebyshev_sweeps(double rho_bound, double reduction);

// ---- nonlinear scalar test PDE of Sec. 5.2 (misdc_pde.cu) ----
// One CTA per instance; every node array in shared memory (pde_smem_bytes).
struct PdeLaunch {
  int scheme, M, n_sweeps, nu, n_steps, nx, n;
  double dt, dx;
  double tau[kMaxNodes + 1], Q[kMaxNodes][kMaxNodes + 1], S[kMaxNodes][kMaxNodes + 1];
  double QI[kMaxNodes][kMaxNodes], QE[kMaxNodes][kMaxNodes];
  const double *params;   // [n][5]: a, d, r, left, right
  const double *phi_in;   // [n][nx]
  double *phi_out;        // [n][nx]
  double *incr;           // [n][n_steps][n_sweeps] or null
  int *status;            // [n] or null
};
size_t pde_smem_bytes(int M, int nx);
cudaError_t launch_pde_step(const PdeLaunch &p, cudaStream_t s);
// many instances: one thread each, node arrays in a workspace of pde_batch_bytes
// laid out [array][cell][instance]
// (one warp per 32 instances is latency-bound: it pays once several warps share each SM)
constexpr int kPdeBatchMin = 4096;
size_t pde_batch_bytes(int M, int nx, int n);
cudaError_t launch_pde_batch(const PdeLaunch &p, double *ws, cudaStream_t s);

// ---- variable-density low-Mach step of independent 1D flames (misdc_lowmach.cu) ----
size_t lowmach_work_bytes(int N, int nx, int M, int n);
cudaError_t launch_lowmach(const DevMech &m, int nx, double dx, int M, const double *tau,
                           const double (*Q)[kMaxNodes + 1], const double (*QI)[kMaxNodes],
                           const double (*QE)[kMaxNodes], int scheme, int n_sweeps, int nu,
                           int i0, double rtol, int maxit, double dt, double U_in, double T_in,
                           double p0, int dchi, const double *Y_in_host, int n,
                           const double *q_in, double *q_out, double *peos, int *status,
                           double *ws, cudaStream_t s);

// ---- learned Newton guess: MLP kernels (misdc_mlp.cu) ----
namespace mlp {
// BF16 operand: element (r, k) at p[r * sm + k * sk]; rows >= rows read as zero
struct Operand {
  const __nv_bfloat16 *p;
  long long sm, sk;
  int rows;
};
enum : int { kEpiStore = 0, kEpiBiasGelu = 1, kEpiGeluGrad = 2, kEpiAtomic = 3 };
// Epilogue of the tensor-core GEMM, per output element (row, col < n_store) at row*ldo + col:
//  kEpiStore:    out_f32 = C (+ bias)
//  kEpiBiasGelu: z = C + bias; out_f32 = z (optional); out_bf16 = gelu(z)
//  kEpiGeluGrad: g = C * gelu'(zsaved); out_f32 = g (optional); out_bf16 = g
//  kEpiAtomic:   out_f32 += C (split-K)
struct Epi {
  int mode, n_store, ldo;
  const float *bias;
  float *out_f32;
  __nv_bfloat16 *out_bf16;
  const float *zsaved;
};
constexpr int kGemmSmemLaunch = 100 * 1024;
}  // namespace mlp
void mlp_prepare();
// C[M x N] (+)= A[M x K] Bt^T; splits > 1 splits K over CTAs (use kEpiAtomic). err: device flag
// set to 1 when an MMA wait gave up.
void mlp_gemm(const mlp::Operand &A, const mlp::Operand &Bt, int M, int N, int K, int splits,
              const mlp::Epi &ep, int *err, cudaStream_t s);
struct Surrogate;
// Fused inference over n rows: with m != NULL the features of cells [0, n) are
// computed from the reaction step's state (scale s written to `scale`),
// otherwise the BF16 rows X [n][ldx] are the input; out [n][ldo] FP32.
void mlp_fused_forward(const Surrogate &g, const DevMech *m, int cs, double wdt, const double *b,
                       const double *hstar, const double *Yp, const double *Tp, const double *FRp,
                       const double *hp, double *scale, const __nv_bfloat16 *X, int n, float *out,
                       cudaStream_t s, const unsigned long long *count = nullptr);
void mlp_features(const DevMech &m, int n, int cs, double wdt, const double *b,
                  const double *hstar, const double *Yp, const double *Tp, const double *FRp,
                  const double *hp, int ldx, __nv_bfloat16 *X, double *scale, double s_min,
                  unsigned long long *counter, long long cap, int *rowmap, cudaStream_t s,
                  const int *list = nullptr, const int *list_n = nullptr);
void mlp_targets(int N, int n, int cs, const double *Yp, const double *Tp, const double *Ys,
                 const double *Ts, const double *scale, const int *rowmap, int ldt, float *tgt,
                 cudaStream_t s);
void mlp_mse(int B, int n_out, int ld, const float *O, const float *Yt, float *dO,
             __nv_bfloat16 *dOb, float *loss, cudaStream_t s);
void mlp_colsum(int rows, int n, int ld, const float *in, float *out, cudaStream_t s);
void mlp_adamw(size_t n, size_t n_decay, float *P, const float *G, float *Mm, float *Vm,
               __nv_bfloat16 *Pb, float lr, float beta1, float beta2, float eps, float wd,
               float bc1, float bc2, cudaStream_t s);
void mlp_to_bf16(size_t n, const float *in, __nv_bfloat16 *out, cudaStream_t s);
void mlp_gather(int B, long long rows, unsigned long long seed, int ldx, int ldt,
                const __nv_bfloat16 *DX, const float *DT, __nv_bfloat16 *X, float *Yt,
                cudaStream_t s);

// The learned-guess network of one solver: parameters, Adam moments, activation
// buffers, and the dataset of recorded solves. Parameter vector (FP32, with a
// BF16 copy at the same offsets): W1 [H][ldx], W2 [H][H], W3 [H][H],
// W4 [ldo][H], then b1 [H], b2 [H], b3 [H], b4 [ldo]; W1 columns >= n_in and
// W4 rows / b4 entries >= n_out stay zero.
struct Surrogate {
  int N = 0, n_in = 0, ldx = 0, H = 256, n_out = 0, ldo = 0;
  size_t off[8] = {};
  size_t n_params = 0, n_weights = 0;
  float *P = nullptr, *G = nullptr, *Mm = nullptr, *Vm = nullptr;
  __nv_bfloat16 *Pb = nullptr;
  int *err = nullptr;
  long long adam_t = 0;
  bool ready = false;   // parameters initialised or loaded
  // inference over the cells of a reaction step
  int cap_inf = 0;
  __nv_bfloat16 *Xi = nullptr, *Ha = nullptr, *Hb = nullptr;
  float *Oi = nullptr;
  double *scale = nullptr;
  int *rowmap = nullptr;
  unsigned long long *inf_count = nullptr;   // rows of the compacted inference batch
  // training batch
  int cap_tr = 0;
  __nv_bfloat16 *Xt = nullptr, *H1 = nullptr, *H2 = nullptr, *H3 = nullptr, *dOb = nullptr,
                *dZa = nullptr, *dZb = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *Ot = nullptr, *dO = nullptr, *dZf = nullptr,
        *Yt = nullptr, *loss = nullptr;
  int loss_cap = 0;
  // dataset of recorded solves
  long long ds_cap = 0;
  unsigned long long *ds_count = nullptr;
  __nv_bfloat16 *DX = nullptr;
  float *DT = nullptr;
  std::vector<void *> allocs;

  ~Surrogate();
  cudaError_t setup(int n_species);                       // sizes and parameter storage
  void init_params(unsigned long long seed, std::vector<float> &host) const;
  cudaError_t upload(const float *host, cudaStream_t s);   // parameters (FP32) -> device + BF16
  cudaError_t ensure_inference(int cells);
  cudaError_t ensure_training(int batch, int steps);
  cudaError_t ensure_dataset(long long cap);
  // O [n][ldo] = MLP(X [n][ldx]); train: keep pre-activations in the training buffers
  void forward(const __nv_bfloat16 *X, int n, float *O, bool train, cudaStream_t s);
  // gradient of the mean-squared loss of the training forward pass against Yt into G
  void backward(const __nv_bfloat16 *X, int B, float *loss_slot, cudaStream_t s);
  void adamw(float lr, float wd, cudaStream_t s);

 private:
  template <typename T>
  cudaError_t alloc(T **p, size_t n);
};

}  // namespace misdc
