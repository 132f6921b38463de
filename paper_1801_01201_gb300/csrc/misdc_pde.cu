// Nonlinear scalar test problem of Sec. 5.2 (eq. nonlinear_test_pde) on the GPU:
//   phi_t = a phi_x + d phi_xx + r phi (phi - 1)(phi - 1/2)  on [0, L],
//   phi(0, t) = left, phi(L, t) = right,
// discretised by finite volumes with fourth-order advective face values and the
// fourth-order five-point Laplacian (Sec. 5.2), advanced by MISDC, MISDCQ or
// CISDCQ-nu (the update equations of Sec. 3.1-3.2) on Gauss-Lobatto nodes.
//
// Two layouts of one kernel (k_pde<BATCH>), both advancing independent instances
// (each with its own a, d, r and boundary values) through all sweeps of all time
// steps of a launch:
//  - BATCH = false, one CTA per instance: every node array in shared memory, so
//    the whole SDC node stack stays on chip and HBM carries only the initial and
//    final state. Threads own cells; the one-thread banded substitutions and the
//    block barriers make it latency-bound, which suits a few instances.
//  - BATCH = true, one thread per instance: the node arrays live in a global
//    workspace laid out [array][cell][instance], so the 32 lanes of a warp read
//    32 instances' values of the same cell in one coalesced access and every FP64
//    instruction, the substitutions included, serves 32 instances. For many
//    instances this is the throughput layout (bounded by the workspace traffic).
// The implicit diffusion matrix I - w L (L the five-point operator closed by the
// Dirichlet ghost cells) depends only on w, so each of the M weights is
// factorised once per launch (banded LU with partial pivoting) and every
// diffusion step is a forward and a back substitution over the band.
#include <math.h>

#include "misdc_internal.cuh"

namespace misdc {
namespace {

// Roles of the per-node arrays: the state and its three right-hand sides.
enum { kPhi = 0, kFA = 1, kFD = 2, kFR = 3, kRoles = 4 };

// A column of one instance: element i at p[i * s] (s = 1 in shared memory, the
// number of instances in the batched workspace).
struct Col {
  double *p;
  size_t s;
  __device__ __forceinline__ double &operator[](int i) const { return p[(size_t)i * s]; }
  __device__ __forceinline__ Col sub(size_t elems) const { return Col{p + elems * s, s}; }
};
struct ColB {
  unsigned char *p;
  size_t s;
  __device__ __forceinline__ unsigned char &operator[](int i) const { return p[(size_t)i * s]; }
  __device__ __forceinline__ ColB sub(size_t elems) const { return ColB{p + elems * s, s}; }
};

struct PdeView {
  int nx, M;
  Col node0;      // [kRoles][nx]: phi^n and its right-hand sides (I1-I4)
  Col sets;       // [3][kRoles][M][nx]: sweep k, iteration l, iteration l+1 (nodes 1..M)
  Col FAad, FDad; // lag source of iteration 0 (Sec. 3.2.2, initial lagged values)
  Col rhs, bvec, ad;
  Col U;          // [M][nx][5]: 1/pivot and the four entries right of it
  Col Lm;         // [M][nx][2]: multipliers of the two rows below
  ColB piv;       // [M][nx]: pivot row offset 0..2

  __device__ Col arr(int set, int role, int m) const {   // m in 1..M
    return sets.sub(((size_t)(set * kRoles + role) * M + (m - 1)) * nx);
  }
  __device__ Col r0(int role) const { return node0.sub((size_t)role * nx); }
  __device__ Col Ut(int t) const { return U.sub((size_t)(t - 1) * 5 * nx); }
  __device__ Col Lt(int t) const { return Lm.sub((size_t)(t - 1) * 2 * nx); }
  __device__ ColB Pt(int t) const { return piv.sub((size_t)(t - 1) * nx); }
};

// Ghost cell averages of the fourth-order Dirichlet closure: the averages over the
// first and second ghost cells of the cubic that takes the wall value and has the
// first three interior cell averages (exact rational weights of that cubic).
__device__ __forceinline__ double cell(const Col &x, int i, int nx, double L, double R) {
  if (i >= 0 && i < nx) return x[i];
  if (i == -1) return 4.0 * L + (-13.0 * x[0] + 5.0 * x[1] - x[2]) * (1.0 / 3.0);
  if (i == -2) return 16.0 * L + (-70.0 * x[0] + 32.0 * x[1] - 7.0 * x[2]) * (1.0 / 3.0);
  if (i == nx) return 4.0 * R + (-13.0 * x[nx - 1] + 5.0 * x[nx - 2] - x[nx - 3]) * (1.0 / 3.0);
  return 16.0 * R + (-70.0 * x[nx - 1] + 32.0 * x[nx - 2] - 7.0 * x[nx - 3]) * (1.0 / 3.0);
}

struct PdeCoef {
  double a, d, r, left, right;
  double ca;   // a / dx
  double cd;   // d / (12 dx^2)
};

// F_A and F_D at cell i: a (phi_{i+1/2} - phi_{i-1/2}) / dx with fourth-order face
// values (7 (phi_i + phi_{i+1}) - (phi_{i-1} + phi_{i+2})) / 12, and
// d (-phi_{i+2} + 16 phi_{i+1} - 30 phi_i + 16 phi_{i-1} - phi_{i-2}) / (12 dx^2).
__device__ __forceinline__ void ad_terms(const Col &x, int i, int nx, const PdeCoef &c,
                                         double *fa, double *fd) {
  const double em2 = cell(x, i - 2, nx, c.left, c.right), em1 = cell(x, i - 1, nx, c.left, c.right);
  const double e0 = x[i];
  const double ep1 = cell(x, i + 1, nx, c.left, c.right), ep2 = cell(x, i + 2, nx, c.left, c.right);
  const double fr = (7.0 * (e0 + ep1) - (em1 + ep2)) * (1.0 / 12.0);
  const double fl = (7.0 * (em1 + e0) - (em2 + ep1)) * (1.0 / 12.0);
  *fa = c.ca * (fr - fl);
  *fd = c.cd * (16.0 * (ep1 + em1) - 30.0 * e0 - (ep2 + em2));
}

__device__ __forceinline__ double reaction(double y, double r) { return r * y * (y - 1.0) * (y - 0.5); }

// Affine part of F_D at cell i: what the boundary values contribute through the
// ghost cells (F_D(x) = L x + g).
__device__ __forceinline__ double affine_g(int i, int nx, const PdeCoef &c) {
  double g = 0.0;
  if (i == 0) g = c.cd * (16.0 * 4.0 * c.left - 16.0 * c.left);
  else if (i == 1) g = c.cd * (-4.0 * c.left);
  else if (i == nx - 1) g = c.cd * (16.0 * 4.0 * c.right - 16.0 * c.right);
  else if (i == nx - 2) g = c.cd * (-4.0 * c.right);
  return g;
}

// Row i of the linear part L of F_D over columns i-2..i+2 (ghosts folded in).
__device__ void lap_row(int i, int nx, double cd, double row[5]) {
  const double s[5] = {-cd, 16.0 * cd, -30.0 * cd, 16.0 * cd, -cd};
  const double g1[3] = {-13.0 / 3.0, 5.0 / 3.0, -1.0 / 3.0};   // first ghost on cells 0,1,2
  const double g2[3] = {-70.0 / 3.0, 32.0 / 3.0, -7.0 / 3.0};  // second ghost
  for (int k = 0; k < 5; ++k) row[k] = 0.0;
  for (int o = -2; o <= 2; ++o) {
    const int j = i + o;
    const double w = s[o + 2];
    if (j >= 0 && j < nx) {
      row[o + 2] += w;
    } else if (j < 0) {
      const double *g = (j == -1) ? g1 : g2;
      for (int q = 0; q < 3; ++q) row[q - i + 2] += w * g[q];
    } else {
      const double *g = (j == nx) ? g1 : g2;
      for (int q = 0; q < 3; ++q) row[(nx - 1 - q) - i + 2] += w * g[q];
    }
  }
}

// Row i of I - w L over the window columns k..k+4 (k <= i <= k+2).
__device__ void sys_row(int i, int k, int nx, double w, double cd, double out[5]) {
  for (int q = 0; q < 5; ++q) out[q] = 0.0;
  if (i >= nx) return;
  double row[5];
  lap_row(i, nx, cd, row);
  for (int q = 0; q < 5; ++q) {
    const int col = i - 2 + q, slot = col - k;
    if (col >= 0 && col < nx && slot >= 0 && slot < 5) out[slot] = -w * row[q] + (q == 2 ? 1.0 : 0.0);
  }
}

// Banded LU with partial pivoting of I - w L (lower bandwidth 2, upper bandwidth 4
// after row exchanges), over a rolling window of three rows. Returns false on a
// zero pivot.
__device__ bool band_factor(int nx, double w, double cd, const Col &U, const Col &Lm, const ColB &piv) {
  double r0[5], r1[5], r2[5];
  sys_row(0, 0, nx, w, cd, r0);
  sys_row(1, 0, nx, w, cd, r1);
  sys_row(2, 0, nx, w, cd, r2);
  for (int k = 0; k < nx; ++k) {
    const int rows = min(3, nx - k);
    int p = 0;
    double best = fabs(r0[0]);
    if (rows > 1 && fabs(r1[0]) > best) { p = 1; best = fabs(r1[0]); }
    if (rows > 2 && fabs(r2[0]) > best) { p = 2; best = fabs(r2[0]); }
    if (p == 1) for (int q = 0; q < 5; ++q) { double t = r0[q]; r0[q] = r1[q]; r1[q] = t; }
    if (p == 2) for (int q = 0; q < 5; ++q) { double t = r0[q]; r0[q] = r2[q]; r2[q] = t; }
    if (!(best > 0.0)) return false;
    const double inv = 1.0 / r0[0];
    const double l1 = rows > 1 ? r1[0] * inv : 0.0, l2 = rows > 2 ? r2[0] * inv : 0.0;
    for (int q = 1; q < 5; ++q) { r1[q] -= l1 * r0[q]; r2[q] -= l2 * r0[q]; }
    U[k * 5] = inv;
    for (int q = 1; q < 5; ++q) U[k * 5 + q] = r0[q];
    Lm[k * 2] = l1;
    Lm[k * 2 + 1] = l2;
    piv[k] = (unsigned char)p;
    for (int q = 0; q < 4; ++q) { r0[q] = r1[q + 1]; r1[q] = r2[q + 1]; }
    r0[4] = 0.0;
    r1[4] = 0.0;
    sys_row(k + 3, k + 1, nx, w, cd, r2);
  }
  return true;
}

// x := (I - w L)^{-1} x with the factor of band_factor (one thread).
__device__ void band_solve(int nx, const Col &U, const Col &Lm, const ColB &piv, const Col &x) {
  double a0 = x[0], a1 = nx > 1 ? x[1] : 0.0, a2 = nx > 2 ? x[2] : 0.0;
  for (int k = 0; k < nx; ++k) {
    const int p = piv[k];
    if (p == 1) { double t = a0; a0 = a1; a1 = t; }
    if (p == 2) { double t = a0; a0 = a2; a2 = t; }
    a1 -= Lm[k * 2] * a0;
    a2 -= Lm[k * 2 + 1] * a0;
    x[k] = a0;
    a0 = a1;
    a1 = a2;
    a2 = (k + 3 < nx) ? x[k + 3] : 0.0;
  }
  double b1 = 0.0, b2 = 0.0, b3 = 0.0, b4 = 0.0;   // x[k+1..k+4]
  for (int k = nx - 1; k >= 0; --k) {
    const double v = (x[k] - U[k * 5 + 4] * b4 - U[k * 5 + 3] * b3 - U[k * 5 + 2] * b2 -
                      U[k * 5 + 1] * b1) * U[k * 5];
    x[k] = v;
    b4 = b3; b3 = b2; b2 = b1; b1 = v;
  }
}

// Scalar Newton for y - w r y (y - 1)(y - 1/2) = b from the guess y; stops once
// |dy| <= 1e-15 (1 + |y|). Returns the iterate; *st gets 1 on the iteration
// limit, 2 on a non-finite value.
__device__ __forceinline__ double reaction_solve(double w, double r, double b, double y, int *st) {
  for (int it = 0; it < 100; ++it) {
    const double f = y - w * reaction(y, r) - b;
    const double df = 1.0 - w * r * ((3.0 * y - 3.0) * y + 0.5);
    const double dy = -f / df;
    y += dy;
    if (!isfinite(y)) { *st |= 2; return y; }
    if (fabs(dy) <= 1e-15 * (1.0 + fabs(y))) return y;
  }
  *st |= 1;
  return y;
}

// block-wide sum in a fixed order (deterministic)
__device__ double block_sum(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < nw; ++q) s += red[q];
  __syncthreads();
  return s;
}

// BATCH = false: one block per instance, the views in shared memory (stride 1).
// BATCH = true: one thread per instance, the views in the workspace ws / wpiv
// (stride n); a thread past the last instance returns at once (no barriers).
template <bool BATCH>
__global__ void k_pde(PdeLaunch P, double *__restrict__ ws, unsigned char *__restrict__ wpiv) {
  extern __shared__ __align__(16) double smem[];
  const int nx = P.nx, M = P.M;
  int inst, tid, nt;
  size_t s;   // stride between the cells of one instance
  double *p;
  unsigned char *pp;
  double *red = nullptr;
  int *sflag = nullptr;
  if constexpr (BATCH) {
    inst = blockIdx.x * blockDim.x + threadIdx.x;
    if (inst >= P.n) return;
    tid = 0;
    nt = 1;
    s = (size_t)P.n;
    p = ws + inst;
    pp = wpiv + inst;
  } else {
    inst = blockIdx.x;
    tid = threadIdx.x;
    nt = blockDim.x;
    s = 1;
    p = smem;
  }
  PdeView V;
  V.nx = nx;
  V.M = M;
  V.node0 = Col{p, s}; p += (size_t)kRoles * nx * s;
  V.sets = Col{p, s}; p += (size_t)3 * kRoles * M * nx * s;
  V.FAad = Col{p, s}; p += (size_t)nx * s;
  V.FDad = Col{p, s}; p += (size_t)nx * s;
  V.rhs = Col{p, s}; p += (size_t)nx * s;
  V.bvec = Col{p, s}; p += (size_t)nx * s;
  V.ad = Col{p, s}; p += (size_t)nx * s;
  V.U = Col{p, s}; p += (size_t)5 * M * nx * s;
  V.Lm = Col{p, s}; p += (size_t)2 * M * nx * s;
  if constexpr (!BATCH) {
    red = p; p += 32;
    sflag = (int *)p; p += 1;
    pp = (unsigned char *)p;
  }
  V.piv = ColB{pp, s};
  auto sync = [&]() {
    if constexpr (!BATCH) __syncthreads();
  };

  const double *prm = P.params + (size_t)inst * 5;
  PdeCoef c;
  c.a = prm[0]; c.d = prm[1]; c.r = prm[2]; c.left = prm[3]; c.right = prm[4];
  c.ca = c.a / P.dx;
  c.cd = c.d / (12.0 * P.dx * P.dx);
  const double dt = P.dt;

  // implicit weight of the diffusion step at node t
  auto wdiff = [&](int t) -> double {
    return P.scheme == MISDC_SCHEME_MISDC ? dt * (P.tau[t] - P.tau[t - 1]) : dt * P.QI[t - 1][t - 1];
  };

  int flag = 0;   // status bits of the factorisations (BATCH) / of this thread
  if constexpr (!BATCH) {
    if (tid == 0) *sflag = 0;
  }
  sync();
  // factor I - w_t L for t = 1..M (one lane each in a block; all by the thread in a batch)
  for (int q = BATCH ? 0 : tid; q < M; q += BATCH ? 1 : M) {
    if (!band_factor(nx, wdiff(q + 1), c.cd, V.Ut(q + 1), V.Lt(q + 1), V.Pt(q + 1))) {
      if constexpr (BATCH) flag |= 4;
      else atomicOr(sflag, 4);
    }
  }
  for (int i = tid; i < nx; i += nt) V.r0(kPhi)[i] = P.phi_in[(size_t)inst * nx + i];
  sync();

  int st = 0;   // this thread's status bits
  for (int step = 0; step < P.n_steps; ++step) {
    // I1-I2, I4: every node starts at phi^n; right-hand sides at phi^n
    int sK = 0, sX = 1, sC = 2;
    for (int i = tid; i < nx; i += nt) {
      double fa, fd;
      ad_terms(V.r0(kPhi), i, nx, c, &fa, &fd);
      const double y = V.r0(kPhi)[i], fr = reaction(y, c.r);
      V.r0(kFA)[i] = fa;
      V.r0(kFD)[i] = fd;
      V.r0(kFR)[i] = fr;
      for (int m = 1; m <= M; ++m) {
        V.arr(sK, kPhi, m)[i] = y;
        V.arr(sK, kFA, m)[i] = fa;
        V.arr(sK, kFD, m)[i] = fd;
        V.arr(sK, kFR, m)[i] = fr;
      }
    }
    sync();

    for (int k = 0; k < P.n_sweeps; ++k) {
      auto K = [&](int role, int m) -> Col { return m == 0 ? V.r0(role) : V.arr(sK, role, m); };
      // Delta t Q^{0:t}(F(phi^(k))) (MISDCQ, CISDCQ) or Delta t S^{t-1:t}(F(phi^(k)))
      // (MISDC) at cell i
      auto quad = [&](int t, int i) -> double {
        double q = 0.0;
        for (int j = 0; j <= M; ++j) {
          const double w = dt * (P.scheme == MISDC_SCHEME_MISDC ? P.S[t - 1][j] : P.Q[t - 1][j]);
          q += w * (K(kFA, j)[i] + K(kFD, j)[i] + K(kFR, j)[i]);
        }
        return q;
      };
      // the diffusion solve of node t from V.rhs into V.ad (the affine part of F_D
      // moves to the right-hand side)
      auto diffusion = [&](int t) {
        const double w = wdiff(t);
        for (int i = tid; i < nx; i += nt) V.ad[i] = V.rhs[i] + w * affine_g(i, nx, c);
        sync();
        if (tid == 0) band_solve(nx, V.Ut(t), V.Lt(t), V.Pt(t), V.ad);
        sync();
      };
      // reaction step: V.bvec -> state of set ss at node t (guess: g), then S6
      auto react = [&](int t, double w, int ss, const Col &g) {
        const Col x = V.arr(ss, kPhi, t), fr = V.arr(ss, kFR, t);
        for (int i = tid; i < nx; i += nt) {
          const double b = V.bvec[i];
          const double y = reaction_solve(w, c.r, b, g[i], &st);
          x[i] = y;
          fr[i] = (y - b) / w;   // the reaction term the implicit equation assigns
        }
        sync();
        const Col fa = V.arr(ss, kFA, t), fd = V.arr(ss, kFD, t);
        for (int i = tid; i < nx; i += nt) ad_terms(x, i, nx, c, &fa[i], &fd[i]);
        sync();
      };

      int sOut;   // the set holding sweep k+1 at nodes 1..M
      if (P.scheme == MISDC_SCHEME_MISDC) {
        // eqs. update_equation_misdc_discrete_form_D / _R: node to node, backward
        // Euler for diffusion and reaction, forward Euler for advection
        for (int t = 1; t <= M; ++t) {
          const int m = t - 1;
          const double dtm = dt * (P.tau[t] - P.tau[m]);
          const Col xm = m == 0 ? V.r0(kPhi) : V.arr(sC, kPhi, m);
          const Col fam = m == 0 ? V.r0(kFA) : V.arr(sC, kFA, m);
          for (int i = tid; i < nx; i += nt)
            V.rhs[i] = xm[i] + dtm * (fam[i] - K(kFA, m)[i]) - dtm * K(kFD, t)[i] + quad(t, i);
          diffusion(t);
          for (int i = tid; i < nx; i += nt) V.bvec[i] = V.ad[i] - dtm * K(kFR, t)[i];
          sync();
          react(t, dtm, sC, K(kPhi, t));
        }
        sOut = sC;
      } else if (P.scheme == MISDC_SCHEME_MISDCQ) {
        // eqs. update_equation_misdcq_discrete_form_D / _R
        for (int t = 1; t <= M; ++t) {
          const int m = t - 1;
          const double w = dt * P.QI[t - 1][t - 1];
          for (int i = tid; i < nx; i += nt) {
            double v = V.r0(kPhi)[i] + quad(t, i) - w * K(kFD, t)[i];
            for (int j = 1; j <= m; ++j)
              v += dt * P.QE[t - 1][j - 1] * (V.arr(sC, kFA, j)[i] - K(kFA, j)[i]) +
                   dt * P.QI[t - 1][j - 1] * (V.arr(sC, kFD, j)[i] - K(kFD, j)[i]);
            V.rhs[i] = v;
          }
          diffusion(t);
          for (int i = tid; i < nx; i += nt) {
            double v = V.ad[i] - w * K(kFR, t)[i];
            for (int j = 1; j <= m; ++j)
              v += dt * P.QI[t - 1][j - 1] * (V.arr(sC, kFR, j)[i] - K(kFR, j)[i]);
            V.bvec[i] = v;
          }
          sync();
          react(t, w, sC, K(kPhi, t));
        }
        sOut = sC;
      } else {
        // CISDCQ-nu: eqs. update_equation_amisdcq_discrete_form_D and _R_alt with the
        // lagged values of iteration l; iteration 0 lags F_A, F_D at node m to the
        // advection-diffusion state of node m in the current iteration and F_R at
        // nodes m, m+1 to sweep k (initial_lagged_values_A/D/R)
        for (int l = 0; l < P.nu; ++l) {
          for (int t = 1; t <= M; ++t) {
            const int m = t - 1;
            const double w = dt * P.QI[t - 1][t - 1];
            // lagged columns (only read when m >= 1)
            const Col lagA = l == 0 ? V.FAad : V.arr(sX, kFA, m >= 1 ? m : 1);
            const Col lagD = l == 0 ? V.FDad : V.arr(sX, kFD, m >= 1 ? m : 1);
            const Col lagRm = l == 0 ? K(kFR, m) : V.arr(sX, kFR, m >= 1 ? m : 1);
            const Col lagRt = l == 0 ? K(kFR, t) : V.arr(sX, kFR, t);
            for (int i = tid; i < nx; i += nt) {
              double v = V.r0(kPhi)[i] + quad(t, i);
              for (int j = 1; j <= m - 1; ++j)
                v += dt * P.QE[t - 1][j - 1] * (V.arr(sC, kFA, j)[i] - K(kFA, j)[i]) +
                     dt * P.QI[t - 1][j - 1] * (V.arr(sC, kFD, j)[i] - K(kFD, j)[i] +
                                                V.arr(sC, kFR, j)[i] - K(kFR, j)[i]);
              if (m >= 1)
                v += dt * P.QE[t - 1][m - 1] * (lagA[i] - K(kFA, m)[i]) +
                     dt * P.QI[t - 1][m - 1] * (lagD[i] - K(kFD, m)[i] + lagRm[i] - K(kFR, m)[i]);
              v += w * (lagRt[i] - K(kFR, t)[i] - K(kFD, t)[i]);
              V.rhs[i] = v;
            }
            diffusion(t);
            if (l == 0 && t < M) {   // S4: lag source of the next node
              for (int i = tid; i < nx; i += nt) ad_terms(V.ad, i, nx, c, &V.FAad[i], &V.FDad[i]);
            }
            for (int i = tid; i < nx; i += nt) {
              double v = V.ad[i] - w * lagRt[i];
              if (m >= 1) v += dt * P.QI[t - 1][m - 1] * (V.arr(sC, kFR, m)[i] - lagRm[i]);
              V.bvec[i] = v;
            }
            sync();
            react(t, w, sC, l == 0 ? K(kPhi, t) : V.arr(sX, kPhi, t));
          }
          const int tmp = sX; sX = sC; sC = tmp;   // iteration l+1 becomes the lag source
        }
        sOut = sX;
      }
      // S7 and the sweep increment (1/nx) sum_i |phi^{M,(k+1)} - phi^{M,(k)}|
      double part = 0.0;
      for (int i = tid; i < nx; i += nt) part += fabs(V.arr(sOut, kPhi, M)[i] - V.arr(sK, kPhi, M)[i]);
      double inc;
      if constexpr (BATCH) inc = part / nx;
      else inc = block_sum(part, red) / nx;
      if (P.incr && tid == 0) P.incr[((size_t)inst * P.n_steps + step) * P.n_sweeps + k] = inc;
      const int old = sK;
      sK = sOut;
      if (sX == sOut) sX = old; else sC = old;
    }
    // phi^{n+1} = phi^M of the last sweep becomes the next step's phi^n
    for (int i = tid; i < nx; i += nt) V.r0(kPhi)[i] = V.arr(sK, kPhi, M)[i];
    sync();
  }
  for (int i = tid; i < nx; i += nt) P.phi_out[(size_t)inst * nx + i] = V.r0(kPhi)[i];
  if constexpr (BATCH) {
    if (P.status) P.status[inst] = flag | st;
  } else {
    if (st) atomicOr(sflag, st);
    __syncthreads();
    if (tid == 0 && P.status) P.status[inst] = *sflag;
  }
}

}  // namespace

size_t pde_smem_bytes(int M, int nx) {
  const size_t dbl = (size_t)kRoles * nx + (size_t)3 * kRoles * M * nx + 5 * (size_t)nx +
                     7 * (size_t)M * nx + 32 + 1;
  return dbl * sizeof(double) + (size_t)M * nx;
}

size_t pde_batch_bytes(int M, int nx, int n) {
  const size_t dbl = (size_t)kRoles * nx + (size_t)3 * kRoles * M * nx + 5 * (size_t)nx +
                     7 * (size_t)M * nx;
  return ((dbl * sizeof(double) + (size_t)M * nx) * (size_t)n + 255) / 256 * 256 + 256;
}

cudaError_t launch_pde_step(const PdeLaunch &p, cudaStream_t s) {
  const size_t smem = pde_smem_bytes(p.M, p.nx);
  cudaError_t e = cudaFuncSetAttribute(k_pde<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int threads = min(512, max(64, (p.nx + 31) / 32 * 32));
  k_pde<false><<<p.n, threads, smem, s>>>(p, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_pde_batch(const PdeLaunch &p, double *ws, cudaStream_t s) {
  const size_t dbl = ((size_t)kRoles * p.nx + (size_t)3 * kRoles * p.M * p.nx + 5 * (size_t)p.nx +
                      7 * (size_t)p.M * p.nx) * (size_t)p.n;
  unsigned char *wpiv = reinterpret_cast<unsigned char *>(ws + dbl);
  // one warp per block (about 230 registers a thread): the warps spread over the SMs
  k_pde<true><<<(p.n + 31) / 32, 32, 0, s>>>(p, ws, wpiv);
  return cudaGetLastError();
}

}  // namespace misdc
