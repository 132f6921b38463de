// Variable-density low-Mach coupling on the GPU: one time step of CISDCQ-nu (or
// the serial MISDCQ) for many independent 1D flames with open boundaries, one
// thread block per flame (Sec. 2: eqs. continuity_equation, species_equation,
// enthalpy_equation, p_eos_definition, divergence_constraint, S_def; Sec. 3.3:
// I1-I4 and S1-S7, with S2 the density update, S3/S4 the species and enthalpy
// diffusion solved against the new density, S5 the reaction Newton at the new
// density, S6 the volume-discrepancy correction delta_chi and the velocity from
// div U = S + delta_chi).
//
// State per flame: q = [rho, rho Y_1..rho Y_N, rho h] ([N+2][nx], cells left to
// right). Boundaries: at x = 0 an inflow Dirichlet state (Y_in, T_in, rho from
// the EOS at p0) and velocity U_in; at x = L zero-gradient outflow and no
// diffusive flux. Closures (the paper gives none for them):
//  - advection: fourth-order centred face values of the conserved quantity,
//    (7 (a + b) - (c + d))/12, the inflow value on the inflow face and as the
//    first face's outer ghost, the last cell's value beyond the outflow;
//  - diffusion: second-order fluxes with harmonic-mean (rho theta) coefficients;
//    on the inflow face the gradient is taken to the inflow value half a cell
//    away with the first cell's coefficient; the dominant species' flux is
//    minus the others';
//  - S (eq. S_def) with Gamma_i = rho D_i grad Y_i (the sign the EOS held at p0
//    along particle paths gives), lambda/cp = rho alpha(T), lambda = rho cp
//    alpha(T), the differential-diffusion flux of h explicit with face means of
//    h_i;
//  - delta_chi per cell and node, incremented every sweep from the previous
//    sweep's value by (2/p0)(p_EOS - p0)/dt_m;
//  - the lag source of iteration 0 at node m is the node's advection-diffusion
//    state with the velocity of its own S and the current delta_chi.
// Every phase spreads its work over the block's threads (cells, faces, or one
// thread per field for the tridiagonal diffusion solves); the node stacks live in
// a workspace in global memory (about 0.3 MB per flame of 64 cells and 9 species).
#include <math.h>

#include <string>

#include "misdc_internal.cuh"

namespace misdc {
namespace {

constexpr int kLmThreads = 256;

struct LmLaunch {
  DevMech m;
  int nx, M, n_sweeps, nu, scheme, i0, maxit, dchi, n;
  double dx, dt, U_in, T_in, p0, rtol;
  double tau[kMaxNodes + 1], Q[kMaxNodes][kMaxNodes + 1], QI[kMaxNodes][kMaxNodes],
      QE[kMaxNodes][kMaxNodes];
  // inflow state (device): Y_in [N], rho_in, h_in, h_i(T_in) [N]
  const double *Y_in, *hsp_in;
  const double *rho_h_in;
  const double *q_in;     // [n][N+2][nx]
  double *q_out, *peos;   // [n][N+2][nx], [n][nx] (may be null)
  int *status;            // [n] (may be null): bit 1 Newton, 2 temperature, 4 non-finite
  double *ws;
  size_t per_flame;       // doubles of workspace per flame
};

// ---- thread-level thermodynamics and kinetics --------------------------------
__device__ __forceinline__ double lm_hRT(const DevMech &m, int i, double T, double invT) {
  const double *a = m.hcoef + 6 * i;
  return fma(a[5], invT, a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4]))));
}
__device__ __forceinline__ double lm_cpR(const DevMech &m, int i, double T) {
  const double *c = m.cpcoef + 5 * i;
  return c[0] + T * (c[1] + T * (c[2] + T * (c[3] + T * c[4])));
}
__device__ __forceinline__ double lm_sR(const DevMech &m, int i, double T, double lnT) {
  const double *s = m.scoef + 6 * i;
  return fma(s[0], lnT, T * (s[1] + T * (s[2] + T * (s[3] + T * s[4])))) + s[5];
}
// species enthalpy (J/kg) and heat capacity (J/kg/K)
__device__ __forceinline__ double lm_h(const DevMech &m, int i, double T) {
  return kRu * m.invW[i] * T * lm_hRT(m, i, T, 1.0 / T);
}
__device__ __forceinline__ double lm_cp(const DevMech &m, int i, double T) {
  return kRu * m.invW[i] * lm_cpR(m, i, T);
}
// mixture h and cp of cell k (mass fractions Y[i * ys + k])
__device__ void lm_mix(const DevMech &m, const double *Y, int ys, int k, double T, double &h,
                       double &cp) {
  double hs = 0.0, cs = 0.0;
  const double invT = 1.0 / T;
  for (int i = 0; i < m.N; ++i) {
    const double y = Y[(size_t)i * ys + k] * m.invW[i];
    hs = fma(y, lm_hRT(m, i, T, invT), hs);
    cs = fma(y, lm_cpR(m, i, T), cs);
  }
  h = kRu * T * hs;
  cp = kRu * cs;
}
// temperature of cell k from sum Y_i h_i(T) = h: Newton from the guess, kept inside a
// bisection bracket on [50, 6000] K; false when the bracket holds no root
__device__ bool lm_temperature(const DevMech &m, const double *Y, int ys, int k, double h, double guess,
                               double &T) {
  double lo = kTlo, hi = kThi, f, cp;
  lm_mix(m, Y, ys, k, lo, f, cp);
  if (f - h > 0.0) { T = NAN; return false; }
  lm_mix(m, Y, ys, k, hi, f, cp);
  if (f - h < 0.0) { T = NAN; return false; }
  T = (guess > lo && guess < hi) ? guess : 1000.0;
  for (int it = 0; it < 200; ++it) {
    lm_mix(m, Y, ys, k, T, f, cp);
    f -= h;
    if (f > 0.0) hi = T; else lo = T;
    double Tn = T - f / cp;
    if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
    const double dT = Tn - T;
    T = Tn;
    if (fabs(dT) <= 1e-14 * T) break;
  }
  return true;
}
// ---- per-flame workspace ----------------------------------------------------
struct LmWork {
  double *q[3][kMaxNodes + 1], *FA[3][kMaxNodes + 1], *FD[3][kMaxNodes + 1], *FR[3][kMaxNodes + 1];
  double *Tn[3][kMaxNodes + 1], *dch[3][kMaxNodes + 1];
  double *qad, *lagA, *lagD, *rhs, *bb;                 // [F][nx]
  double *S, *U, *pe, *Tad, *hm;                        // [nx], [nx+1], [nx], [nx], [nx+1]
  double *Y, *h, *hsp, *cpm;                            // [N][nx], [nx], [N][nx], [nx]
  double *G, *gY, *hf, *gh, *Qf, *Kf, *Lc;              // [N][nx+1] x4, [nx+1] x3
  double *cp, *dp;                                      // [F][nx] Thomas scratch
  double *J, *xr, *rr;                                  // Newton: [n^2][nx], [n][nx], [n][nx]
};

__host__ __device__ inline size_t lm_work_doubles(int N, int nx, int M) {
  const size_t F = N + 2, n = N + 1, X = nx, Xp = nx + 1;
  return 3 * (size_t)(M + 1) * (4 * F * X + 2 * X) + 5 * F * X + 4 * X + 2 * Xp + 2 * N * X + 2 * X +
         4 * (size_t)N * Xp + 3 * Xp + 2 * F * X + n * n * X + 2 * n * X;
}

__device__ LmWork lm_carve(double *p, int N, int nx, int M) {
  LmWork w;
  const size_t F = N + 2, n = N + 1, X = nx, Xp = nx + 1;
  for (int s = 0; s < 3; ++s)
    for (int j = 0; j <= M; ++j) {
      w.q[s][j] = p; p += F * X;
      w.FA[s][j] = p; p += F * X;
      w.FD[s][j] = p; p += F * X;
      w.FR[s][j] = p; p += F * X;
      w.Tn[s][j] = p; p += X;
      w.dch[s][j] = p; p += X;
    }
  w.qad = p; p += F * X;
  w.lagA = p; p += F * X;
  w.lagD = p; p += F * X;
  w.rhs = p; p += F * X;
  w.bb = p; p += F * X;
  w.S = p; p += X;
  w.U = p; p += Xp;
  w.pe = p; p += X;
  w.Tad = p; p += X;
  w.hm = p; p += Xp;
  w.Y = p; p += (size_t)N * X;
  w.h = p; p += X;
  w.hsp = p; p += (size_t)N * X;
  w.cpm = p; p += X;
  w.G = p; p += (size_t)N * Xp;
  w.gY = p; p += (size_t)N * Xp;
  w.hf = p; p += (size_t)N * Xp;
  w.gh = p; p += (size_t)N * Xp;
  w.Qf = p; p += Xp;
  w.Kf = p; p += Xp;
  w.Lc = p; p += Xp;
  w.cp = p; p += F * X;
  w.dp = p; p += F * X;
  w.J = p; p += n * n * X;
  w.xr = p; p += n * X;
  w.rr = p; p += n * X;
  return w;
}

__device__ __forceinline__ double lm_theta(const LmLaunch &P, double T) {
  return pow(T / P.m.T_ref, P.m.theta_exp);
}

// fourth-order face value x 12 on interior face j (1..nx-1) of field f (inflow
// value fin as the outer ghost of face 1, the last cell beyond the outflow)
__device__ __forceinline__ double lm_face12(const double *f, double fin, int j, int nx) {
  const double a = (j - 2 >= 0) ? f[j - 2] : fin;
  const double e = (j + 1 < nx) ? f[j + 1] : f[nx - 1];
  return 7.0 * (f[j - 1] + f[j]) - (a + e);
}

// Right-hand sides, S, velocity and p_EOS of state q (block-wide):
//  FA = -div(U q) for every row plus the explicit differential diffusion of h;
//  FD = div(rho D_i grad Y_i) (dominant species closed), div(lambda/cp grad h), 0 for rho;
//  FR = wdot_i for the species rows, 0 for rho and h;
//  S (eq. S_def), U[0] = U_in, U[k+1] = U[k] + dx (S[k] + dchi[k]), p_EOS = rho R T / W.
// Uadv (may be null) is the face velocity of the advection (else U). T: in guess,
// out temperature. Returns (in *bad) the temperature-diagnosis failures.
__device__ void lm_terms(const LmLaunch &P, const LmWork &w, const double *q, const double *dchi,
                         const double *Uadv, double *FA, double *FD, double *FR, double *T,
                         unsigned *bad) {
  const DevMech &m = P.m;
  const int nx = P.nx, N = m.N, i0 = P.i0, tid = threadIdx.x, nt = blockDim.x;
  const double dx = P.dx, inv = 1.0 / dx;
  // primitives, species enthalpies, mixture cp
  for (int k = tid; k < nx; k += nt) {
    const double rho = q[k];
    for (int i = 0; i < N; ++i) w.Y[(size_t)i * nx + k] = q[(size_t)(1 + i) * nx + k] / rho;
    w.h[k] = q[(size_t)(N + 1) * nx + k] / rho;
    double Tk;
    if (!lm_temperature(m, w.Y, nx, k, w.h[k], T[k], Tk)) atomicOr(bad, 2u);
    T[k] = Tk;
    double hh, cpk;
    lm_mix(m, w.Y, nx, k, Tk, hh, cpk);
    w.cpm[k] = cpk;
    for (int i = 0; i < N; ++i) w.hsp[(size_t)i * nx + k] = lm_h(m, i, Tk);
  }
  __syncthreads();
  // diffusive fluxes on the nx+1 faces
  const int Xp = nx + 1;
  for (int j = tid; j <= nx; j += nt) {
    if (j == nx) {   // outflow: no diffusive flux
      for (int i = 0; i < N; ++i) {
        w.G[(size_t)i * Xp + j] = 0.0;
        w.gY[(size_t)i * Xp + j] = 0.0;
        w.gh[(size_t)i * Xp + j] = 0.0;
        w.hf[(size_t)i * Xp + j] = w.hsp[(size_t)i * nx + nx - 1];
      }
      w.Qf[j] = w.Kf[j] = w.Lc[j] = 0.0;
      continue;
    }
    const int r = j;
    const bool in = (j == 0);
    const double dist = in ? 0.5 * dx : dx;
    const double rho_r = q[r], T_r = T[r], h_r = w.h[r], cp_r = w.cpm[r];
    const double th_r = lm_theta(P, T_r);
    double T_l, h_l, rho_l, cp_l;
    if (in) {
      T_l = P.T_in; h_l = P.rho_h_in[1]; rho_l = P.rho_h_in[0];
      double hh;
      lm_mix(m, P.Y_in, 1, 0, P.T_in, hh, cp_l);
    } else {
      T_l = T[j - 1]; h_l = w.h[j - 1]; rho_l = q[j - 1]; cp_l = w.cpm[j - 1];
    }
    const double th_l = lm_theta(P, T_l);
    // on the inflow face the coefficients are those of the first cell
    const double a_l = in ? rho_r * th_r : rho_l * th_l, a_r = rho_r * th_r;
    const double hmf = 2.0 * a_l * a_r / (a_l + a_r);
    const double lam_l = in ? rho_r * cp_r * m.alpha0 * th_r : rho_l * cp_l * m.alpha0 * th_l;
    const double lam_r = rho_r * cp_r * m.alpha0 * th_r;
    w.Lc[j] = m.alpha0 * hmf;
    w.Qf[j] = w.Lc[j] * (h_r - h_l) / dist;
    w.Kf[j] = (2.0 * lam_l * lam_r / (lam_l + lam_r)) * (T_r - T_l) / dist;
    double sum = 0.0;
    for (int i = 0; i < N; ++i) {
      const double yl = in ? P.Y_in[i] : w.Y[(size_t)i * nx + j - 1];
      const double yr = w.Y[(size_t)i * nx + r];
      const double g = (yr - yl) / dist;
      w.gY[(size_t)i * Xp + j] = g;
      const double hl = in ? P.hsp_in[i] : w.hsp[(size_t)i * nx + j - 1];
      const double hr = w.hsp[(size_t)i * nx + r];
      w.hf[(size_t)i * Xp + j] = 0.5 * (hl + hr);
      w.gh[(size_t)i * Xp + j] = (hr - hl) / dist;
      if (i == i0) continue;
      const double v = m.D0[i] * hmf * g;
      w.G[(size_t)i * Xp + j] = v;
      sum += v;
    }
    w.G[(size_t)i0 * Xp + j] = -sum;
  }
  __syncthreads();
  // per cell: wdot, FD, FR, S, p_EOS
  for (int k = tid; k < nx; k += nt) {
    const double rho = q[k], Tk = T[k], lnT = log(Tk), invT = 1.0 / Tk;
    double sw = 0.0;
    for (int i = 0; i < N; ++i) sw += w.Y[(size_t)i * nx + k] * m.invW[i];
    const double Wmix = 1.0 / sw, cpk = w.cpm[k];
    double s2 = 0.0, s3 = 0.0, ghl = 0.0, ghr = 0.0;
    // production rates: every reaction once, scattered to its species
    double wdot[kMaxSpecies];
    for (int i = 0; i < N; ++i) wdot[i] = 0.0;
    for (int r = 0; r < m.R; ++r) {
      // c_i = rho Y_i / W_i, taken by slot
      const signed char *fs = m.fwd + kMaxSlots * r, *rs = m.rev + kMaxSlots * r;
      double qr;
      {
        double dg = 0.0, cf[kMaxSlots], cr[kMaxSlots];
        for (int p2 = 0; p2 < kMaxSlots; ++p2) {
          cf[p2] = cr[p2] = 1.0;
          if (fs[p2] >= 0) {
            const int i = fs[p2];
            dg -= lm_hRT(m, i, Tk, invT) - lm_sR(m, i, Tk, lnT);
            cf[p2] = rho * w.Y[(size_t)i * nx + k] * m.invW[i];
          }
          if (rs[p2] >= 0) {
            const int i = rs[p2];
            dg += lm_hRT(m, i, Tk, invT) - lm_sR(m, i, Tk, lnT);
            cr[p2] = rho * w.Y[(size_t)i * nx + k] * m.invW[i];
          }
        }
        const double lnkf = m.lnA[r] + m.beta[r] * lnT - m.TA[r] * invT;
        const double lnKc = -dg + m.dn[r] * (m.ln_p_over_R - lnT);
        qr = exp(lnkf) * cf[0] * cf[1] * cf[2] - exp(lnkf - lnKc) * cr[0] * cr[1] * cr[2];
      }
      for (int p2 = 0; p2 < kMaxSlots; ++p2) {
        if (fs[p2] >= 0) wdot[fs[p2]] -= qr;
        if (rs[p2] >= 0) wdot[rs[p2]] += qr;
      }
    }
    for (int i = 0; i < N; ++i) wdot[i] *= 1.0 / m.invW[i];   // W_i sum_r nu_ri q_r
    for (int i = 0; i < N; ++i) {
      const double dY = (w.G[(size_t)i * Xp + k + 1] - w.G[(size_t)i * Xp + k]) * inv;
      if (FD) FD[(size_t)(1 + i) * nx + k] = dY;
      if (FR) FR[(size_t)(1 + i) * nx + k] = wdot[i];
      s2 += Wmix * m.invW[i] * dY;
      s3 += (Wmix * m.invW[i] - w.hsp[(size_t)i * nx + k] / (cpk * Tk)) * wdot[i];
      ghl += w.G[(size_t)i * Xp + k] * w.gh[(size_t)i * Xp + k];
      ghr += w.G[(size_t)i * Xp + k + 1] * w.gh[(size_t)i * Xp + k + 1];
    }
    if (FD) {
      FD[k] = 0.0;
      FD[(size_t)(N + 1) * nx + k] = (w.Qf[k + 1] - w.Qf[k]) * inv;
    }
    if (FR) {
      FR[k] = 0.0;
      FR[(size_t)(N + 1) * nx + k] = 0.0;
    }
    const double divK = (w.Kf[k + 1] - w.Kf[k]) * inv;
    w.S[k] = (divK + 0.5 * (ghl + ghr)) / (rho * cpk * Tk) + s2 / rho + s3 / rho;
    w.pe[k] = rho * kRu * Tk * sw;
  }
  __syncthreads();
  // velocity from the constraint, integrated from the inflow face (one thread, in
  // the order of the faces)
  if (tid == 0) {
    w.U[0] = P.U_in;
    for (int k = 0; k < nx; ++k) w.U[k + 1] = w.U[k] + dx * (w.S[k] + (dchi ? dchi[k] : 0.0));
  }
  __syncthreads();
  if (FA) {
    const double *Ua = Uadv ? Uadv : w.U;
    const int F = N + 2;
    for (int e = tid; e < F * nx; e += nt) {
      const int f = e / nx, k = e - f * nx;
      const double *x = q + (size_t)f * nx;
      const double rin = P.rho_h_in[0];
      const double fin = (f == 0) ? rin : (f <= N ? rin * P.Y_in[f - 1] : rin * P.rho_h_in[1]);
      const double Fl = (k == 0) ? Ua[0] * fin : Ua[k] * lm_face12(x, fin, k, nx) / 12.0;
      const double Fr = (k + 1 < nx) ? Ua[k + 1] * lm_face12(x, fin, k + 1, nx) / 12.0
                                     : Ua[nx] * x[nx - 1];
      double v = -(Fr - Fl) * inv;
      if (f == N + 1) {   // explicit differential diffusion of h
        double fl = 0.0, fr = 0.0;
        for (int i = 0; i < N; ++i) {
          const size_t a = (size_t)i * Xp + k, b = a + 1;
          fl += w.hf[a] * (w.G[a] - w.Lc[k] * w.gY[a]);
          fr += w.hf[b] * (w.G[b] - w.Lc[k + 1] * w.gY[b]);
        }
        v += (fr - fl) * inv;
      }
      FA[e] = v;
    }
  }
  __syncthreads();
}

// (rho theta) on the faces of a state: harmonic means inside, the first cell's value
// on the inflow face, 0 on the outflow face
__device__ void lm_face_coef(const LmLaunch &P, const double *q, const double *T, double *hm) {
  const int nx = P.nx;
  for (int j = threadIdx.x; j <= nx; j += blockDim.x) {
    if (j == nx) { hm[j] = 0.0; continue; }
    const double ar = q[j] * lm_theta(P, T[j]);
    if (j == 0) { hm[j] = ar; continue; }
    const double al = q[j - 1] * lm_theta(P, T[j - 1]);
    hm[j] = 2.0 * al * ar / (al + ar);
  }
}

// rho_new x - w div(f0 hm grad x) = rhs for field row f (inflow value xin on the
// inflow face, no flux through the outflow face): tridiagonal, diagonally
// dominant, solved by elimination without pivoting (the Thomas algorithm, one
// thread per field), then the flux-form reconstruction
// out = rhs + w div(f0 hm grad x) (conserved exactly); x in the scratch dp row.
__device__ void lm_tridiag(const LmLaunch &P, const LmWork &w, int f, double wgt, double f0,
                           const double *rho_new, const double *rhs, double xin) {
  const int nx = P.nx;
  const double dx = P.dx, dx2 = dx * dx;
  double *cpr = w.cp + (size_t)f * nx, *x = w.dp + (size_t)f * nx;
  double cprev = 0.0, dprev = 0.0;
  for (int k = 0; k < nx; ++k) {
    const double kl = f0 * w.hm[k] / ((k == 0 ? 0.5 : 1.0) * dx2);
    const double kr = f0 * w.hm[k + 1] / dx2;
    const double diag = rho_new[k] + wgt * (kl + kr);
    const double sub = (k > 0) ? -wgt * kl : 0.0, sup = (k + 1 < nx) ? -wgt * kr : 0.0;
    const double r = rhs[k] + (k == 0 ? wgt * kl * xin : 0.0);
    const double den = diag - sub * cprev;
    cprev = sup / den;
    dprev = (r - sub * dprev) / den;
    cpr[k] = cprev;
    x[k] = dprev;
  }
  for (int k = nx - 2; k >= 0; --k) x[k] -= cpr[k] * x[k + 1];
}

__device__ void lm_reconstruct(const LmLaunch &P, const LmWork &w, int f, double wgt, double f0,
                               const double *rhs, double xin, double *out) {
  const int nx = P.nx;
  const double dx = P.dx;
  const double *x = w.dp + (size_t)f * nx;
  for (int k = threadIdx.x; k < nx; k += blockDim.x) {
    const double fl = f0 * w.hm[k] * (x[k] - (k == 0 ? xin : x[k - 1])) / ((k == 0 ? 0.5 : 1.0) * dx);
    const double fr = (k + 1 < nx) ? f0 * w.hm[k + 1] * (x[k + 1] - x[k]) / dx : 0.0;
    out[k] = rhs[k] + wgt * (fr - fl) / dx;
  }
}

// S5 of cell k at density rho: Y - wgt wdot(rho, Y, T)/rho = bY, sum Y_i h_i(T) = hst;
// Newton with the analytic Jacobian and partial-pivot LU; x = (Y, T) in/out. Stops
// once d = max(max|dY|, |dT|/T) <= rtol (or, as a guard, once d <= 1e-8 no longer
// halves). Returns the iterations, or -1 (limit), -2 (singular), -3 (non-finite).
__device__ int lm_newton(const LmLaunch &P, const LmWork &w, int k, double rho, double wgt,
                         const double *bY, int bs, double hst, double *x, int xs) {
  const DevMech &m = P.m;
  const int N = m.N, n = N + 1, nx = P.nx;
  double *J = w.J + k;          // entry (i, j) at J[(i * n + j) * nx]
  double *rr = w.rr + k;        // [n] stride nx
  const size_t js = nx;
  auto Jat = [&](int i, int j) -> double & { return J[((size_t)i * n + j) * js]; };
  double dprev = INFINITY;
  const double wr = wgt / rho;
  for (int it = 1; it <= P.maxit; ++it) {
    const double T = x[(size_t)N * xs];
    if (!(T > 0.0)) return -3;
    const double lnT = log(T), invT = 1.0 / T;
    // residual and Jacobian
    double hsum = 0.0, cpsum = 0.0;
    for (int i = 0; i < N; ++i) {
      const double y = x[(size_t)i * xs];
      const double hi = kRu * m.invW[i] * T * lm_hRT(m, i, T, invT);
      hsum = fma(y, hi, hsum);
      cpsum = fma(y, kRu * m.invW[i] * lm_cpR(m, i, T), cpsum);
      for (int j = 0; j < n; ++j) Jat(i, j) = (i == j) ? 1.0 : 0.0;
      rr[(size_t)i * js] = y - bY[(size_t)i * bs];
      Jat(N, i) = hi;
    }
    Jat(N, N) = cpsum;
    rr[(size_t)N * js] = hsum - hst;
    for (int r = 0; r < m.R; ++r) {
      const signed char *fs = m.fwd + kMaxSlots * r, *rs = m.rev + kMaxSlots * r;
      double dg = 0.0, dh = 0.0, cf[kMaxSlots], cr[kMaxSlots];
      for (int p = 0; p < kMaxSlots; ++p) {
        cf[p] = cr[p] = 1.0;
        if (fs[p] >= 0) {
          const int i = fs[p];
          const double hr = lm_hRT(m, i, T, invT);
          dg -= hr - lm_sR(m, i, T, lnT);
          dh -= hr;
          cf[p] = rho * x[(size_t)i * xs] * m.invW[i];
        }
        if (rs[p] >= 0) {
          const int i = rs[p];
          const double hr = lm_hRT(m, i, T, invT);
          dg += hr - lm_sR(m, i, T, lnT);
          dh += hr;
          cr[p] = rho * x[(size_t)i * xs] * m.invW[i];
        }
      }
      const double lnkf = m.lnA[r] + m.beta[r] * lnT - m.TA[r] * invT;
      const double lnKc = -dg + m.dn[r] * (m.ln_p_over_R - lnT);
      const double kf = exp(lnkf), kr = exp(lnkf - lnKc);
      const double Ff = cf[0] * cf[1] * cf[2], Fr = cr[0] * cr[1] * cr[2];
      const double qr = kf * Ff - kr * Fr;
      const double dlnkf = (m.beta[r] + m.TA[r] * invT) * invT;
      const double dlnKc = (dh - m.dn[r]) * invT;
      const double dqdT = kf * Ff * dlnkf - kr * Fr * (dlnkf - dlnKc);
      // derivative of q by the concentration of each slot's species
      const double ds[6] = {kf * cf[1] * cf[2], kf * cf[0] * cf[2], kf * cf[0] * cf[1],
                            -kr * cr[1] * cr[2], -kr * cr[0] * cr[2], -kr * cr[0] * cr[1]};
      const int sp[6] = {fs[0], fs[1], fs[2], rs[0], rs[1], rs[2]};
      // rows: the species of every slot, with nu = -1 per reactant slot, +1 per product slot
      for (int a = 0; a < 6; ++a) {
        const int i = sp[a];
        if (i < 0) continue;
        const double s = (a < 3 ? -1.0 : 1.0) / m.invW[i];   // W_i nu per slot
        rr[(size_t)i * js] -= wr * s * qr;
        for (int b2 = 0; b2 < 6; ++b2) {
          const int j = sp[b2];
          if (j < 0) continue;
          Jat(i, j) -= wr * s * ds[b2] * rho * m.invW[j];
        }
        Jat(i, N) -= wr * s * dqdT;
      }
    }
    // LU with partial pivoting on the augmented system J dx = -r
    for (int i = 0; i < n; ++i) rr[(size_t)i * js] = -rr[(size_t)i * js];
    for (int c = 0; c < n; ++c) {
      int p = c;
      double best = fabs(Jat(c, c));
      for (int i = c + 1; i < n; ++i)
        if (fabs(Jat(i, c)) > best) { best = fabs(Jat(i, c)); p = i; }
      if (!(best > 0.0) || !isfinite(best)) return -2;
      if (p != c) {
        for (int j = c; j < n; ++j) { const double t = Jat(c, j); Jat(c, j) = Jat(p, j); Jat(p, j) = t; }
        const double t = rr[(size_t)c * js]; rr[(size_t)c * js] = rr[(size_t)p * js]; rr[(size_t)p * js] = t;
      }
      const double piv = 1.0 / Jat(c, c);
      for (int i = c + 1; i < n; ++i) {
        const double l = Jat(i, c) * piv;
        if (l == 0.0) continue;
        for (int j = c + 1; j < n; ++j) Jat(i, j) -= l * Jat(c, j);
        rr[(size_t)i * js] -= l * rr[(size_t)c * js];
      }
    }
    for (int c = n - 1; c >= 0; --c) {
      double v = rr[(size_t)c * js];
      for (int j = c + 1; j < n; ++j) v -= Jat(c, j) * rr[(size_t)j * js];
      rr[(size_t)c * js] = v / Jat(c, c);
    }
    double dmax = 0.0;
    for (int i = 0; i < N; ++i) {
      const double d = rr[(size_t)i * js];
      x[(size_t)i * xs] += d;
      dmax = fmax(dmax, fabs(d));
    }
    x[(size_t)N * xs] += rr[(size_t)N * js];
    const double Tn = x[(size_t)N * xs];
    if (!(Tn > 0.0) || !isfinite(Tn)) return -3;
    const double d = fmax(dmax, fabs(rr[(size_t)N * js]) / Tn);
    if (!isfinite(d)) return -3;
    if (d <= P.rtol || (d <= 1e-8 && d >= 0.5 * dprev)) return it;
    dprev = d;
  }
  return -1;
}

__global__ void __launch_bounds__(kLmThreads) k_lowmach(LmLaunch P) {
  const int inst = blockIdx.x;
  if (inst >= P.n) return;
  const DevMech &m = P.m;
  const int nx = P.nx, N = m.N, F = N + 2, nF = F * nx, M = P.M, tid = threadIdx.x, nt = blockDim.x;
  const int i0 = P.i0;
  const bool cisdc = P.scheme == MISDC_SCHEME_CISDCQ;
  const int nu = cisdc ? P.nu : 1;
  const double dt = P.dt;
  LmWork w = lm_carve(P.ws + (size_t)inst * P.per_flame, N, nx, M);
  __shared__ unsigned bad;
  if (tid == 0) bad = 0u;
  const double *qn = P.q_in + (size_t)inst * nF;
  enum { KS = 0, XS = 1, CS = 2 };
  __syncthreads();
  // I1, I2, I4: node 0 and every node of sweep 0 hold q^n and its terms
  for (int k = tid; k < nx; k += nt) w.Tn[KS][0][k] = 1000.0;
  for (int e = tid; e < nF; e += nt) w.q[KS][0][e] = qn[e];
  __syncthreads();
  lm_terms(P, w, w.q[KS][0], nullptr, nullptr, w.FA[KS][0], w.FD[KS][0], w.FR[KS][0], w.Tn[KS][0], &bad);
  for (int s = 0; s < 3; ++s)
    for (int j = 0; j <= M; ++j) {
      if (s == KS && j == 0) continue;
      if (s != KS && j != 0) continue;
      for (int e = tid; e < nF; e += nt) {
        w.q[s][j][e] = qn[e];
        w.FA[s][j][e] = w.FA[KS][0][e];
        w.FD[s][j][e] = w.FD[KS][0][e];
        w.FR[s][j][e] = w.FR[KS][0][e];
      }
      for (int k = tid; k < nx; k += nt) {
        w.Tn[s][j][k] = w.Tn[KS][0][k];
        w.dch[s][j][k] = 0.0;
      }
    }
  for (int k = tid; k < nx; k += nt) w.dch[KS][0][k] = 0.0;
  __syncthreads();
  int sK = KS, sX = XS, sC = CS;
  for (int kk = 0; kk < P.n_sweeps; ++kk) {
    for (int l = 0; l < nu; ++l) {
      for (int mm = 0; mm < M; ++mm) {
        const int t = mm + 1;
        const double wgt = dt * P.QI[t - 1][t - 1], dtm = dt * (P.tau[t] - P.tau[mm]);
        const double *lA = nullptr, *lD = nullptr, *lRm = nullptr;
        if (mm >= 1 && cisdc) {
          lA = (l == 0) ? w.lagA : w.FA[sX][mm];
          lD = (l == 0) ? w.lagD : w.FD[sX][mm];
          lRm = (l == 0) ? w.FR[sK][mm] : w.FR[sX][mm];
        }
        const double *lRt = (l == 0) ? w.FR[sK][t] : w.FR[sX][t];
        // right-hand side of the D update (the CISDCQ form on q; MISDCQ: the serial one)
        for (int e = tid; e < nF; e += nt) {
          double v = qn[e];
          for (int j = 0; j <= M; ++j) {
            const double qw = dt * P.Q[t - 1][j];
            v += qw * w.FA[sK][j][e];
            v += qw * w.FD[sK][j][e];
            v += qw * w.FR[sK][j][e];
          }
          if (!cisdc) {
            for (int j = 1; j <= mm; ++j)
              v += dt * P.QE[t - 1][j - 1] * (w.FA[sC][j][e] - w.FA[sK][j][e]) +
                   dt * P.QI[t - 1][j - 1] * (w.FD[sC][j][e] - w.FD[sK][j][e]);
            v -= wgt * w.FD[sK][t][e];
          } else {
            for (int j = 1; j <= mm - 1; ++j)
              v += dt * P.QE[t - 1][j - 1] * (w.FA[sC][j][e] - w.FA[sK][j][e]) +
                   dt * P.QI[t - 1][j - 1] *
                       (w.FD[sC][j][e] - w.FD[sK][j][e] + w.FR[sC][j][e] - w.FR[sK][j][e]);
            if (mm >= 1)
              v += dt * P.QE[t - 1][mm - 1] * (lA[e] - w.FA[sK][mm][e]) +
                   dt * P.QI[t - 1][mm - 1] * (lD[e] - w.FD[sK][mm][e] + lRm[e] - w.FR[sK][mm][e]);
            v += wgt * (-w.FD[sK][t][e] + lRt[e] - w.FR[sK][t][e]);
          }
          w.rhs[e] = v;
        }
        __syncthreads();
        // S2: the density row has no diffusion or reaction
        for (int k = tid; k < nx; k += nt) w.qad[k] = w.rhs[k];
        // S3, S4: diffusion against rho_new, coefficients lagged (eq.
        // lagged_diffusion_flux: sweep k at l = 0, iteration l otherwise)
        const double *qc = (l == 0) ? w.q[sK][t] : w.q[sX][t];
        const double *Tc = (l == 0) ? w.Tn[sK][t] : w.Tn[sX][t];
        lm_face_coef(P, qc, Tc, w.hm);
        __syncthreads();
        // one thread per solved field: the N-1 species but i0, then h (row N+1)
        for (int f = tid; f < N + 1; f += nt) {
          const int i = (f < N) ? f : -1;   // species index, or h
          if (i == i0) continue;
          const int row = (i >= 0) ? 1 + i : N + 1;
          const double f0 = (i >= 0) ? m.D0[i] : m.alpha0;
          const double xin = (i >= 0) ? P.Y_in[i] : P.rho_h_in[1];
          lm_tridiag(P, w, row, wgt, f0, w.qad, w.rhs + (size_t)row * nx, xin);
        }
        __syncthreads();
        for (int f = 0; f < N + 1; ++f) {
          const int i = (f < N) ? f : -1;
          if (i == i0) continue;
          const int row = (i >= 0) ? 1 + i : N + 1;
          const double f0 = (i >= 0) ? m.D0[i] : m.alpha0;
          const double xin = (i >= 0) ? P.Y_in[i] : P.rho_h_in[1];
          lm_reconstruct(P, w, row, wgt, f0, w.rhs + (size_t)row * nx, xin, w.qad + (size_t)row * nx);
        }
        __syncthreads();
        for (int k = tid; k < nx; k += nt) {   // closure: rho Y_i0 = rho - sum of the others
          double v = w.qad[k];
          for (int i = 0; i < N; ++i)
            if (i != i0) v -= w.qad[(size_t)(1 + i) * nx + k];
          w.qad[(size_t)(1 + i0) * nx + k] = v;
        }
        __syncthreads();
        // S5: rho_new Y - wgt wdot(Y) = b (R_alt form), enthalpy fixed
        for (int e = tid; e < nF; e += nt) {
          double v = w.qad[e];
          if (!cisdc) {
            for (int j = 1; j <= mm; ++j) v += dt * P.QI[t - 1][j - 1] * (w.FR[sC][j][e] - w.FR[sK][j][e]);
          } else if (mm >= 1) {
            v += dt * P.QI[t - 1][mm - 1] * (w.FR[sC][mm][e] - lRm[e]);
          }
          w.bb[e] = v - wgt * lRt[e];
        }
        __syncthreads();
        {
          const double *qg = (l == 0) ? w.q[sK][t] : w.q[sX][t];
          const double *Tg = (l == 0) ? w.Tn[sK][t] : w.Tn[sX][t];
          double *qo = w.q[sC][t], *FRo = w.FR[sC][t];
          for (int k = tid; k < nx; k += nt) {
            const double rho = w.qad[k];
            double *x = w.xr + k;   // [n] stride nx: (Y, T)
            double *bY = w.dp + nx + k;   // b / rho (the diffusion scratch is free here)
            for (int i = 0; i < N; ++i) {
              x[(size_t)i * nx] = qg[(size_t)(1 + i) * nx + k] / qg[k];
              bY[(size_t)i * nx] = w.bb[(size_t)(1 + i) * nx + k] / rho;
            }
            x[(size_t)N * nx] = Tg[k];
            const double hst = w.qad[(size_t)(N + 1) * nx + k] / rho;
            const int it = lm_newton(P, w, k, rho, wgt, bY, nx, hst, x, nx);
            if (it < 0) atomicOr(&bad, it == -1 ? 1u : 4u);
            qo[k] = rho;
            for (int i = 0; i < N; ++i) {
              const double y = x[(size_t)i * nx];
              qo[(size_t)(1 + i) * nx + k] = rho * y;
              FRo[(size_t)(1 + i) * nx + k] = (rho * y - w.bb[(size_t)(1 + i) * nx + k]) / wgt;
            }
            FRo[k] = 0.0;
            FRo[(size_t)(N + 1) * nx + k] = 0.0;
            qo[(size_t)(N + 1) * nx + k] = w.qad[(size_t)(N + 1) * nx + k];
            w.Tn[sC][t][k] = x[(size_t)N * nx];
          }
        }
        __syncthreads();
        // S6: delta_chi from the thermodynamic-pressure discrepancy, velocity and the
        // advection / diffusion terms at the new state
        for (int k = tid; k < nx; k += nt) w.Tad[k] = w.Tn[sC][t][k];
        __syncthreads();
        lm_terms(P, w, w.q[sC][t], nullptr, nullptr, nullptr, nullptr, nullptr, w.Tad, &bad);
        for (int k = tid; k < nx; k += nt)
          w.dch[sC][t][k] = P.dchi ? w.dch[sK][t][k] + 2.0 / P.p0 * (w.pe[k] - P.p0) / dtm : 0.0;
        __syncthreads();
        lm_terms(P, w, w.q[sC][t], w.dch[sC][t], nullptr, w.FA[sC][t], w.FD[sC][t], nullptr,
                 w.Tn[sC][t], &bad);
        if (l == 0 && t < M && cisdc) {   // S4: lag source of the next node
          for (int k = tid; k < nx; k += nt) w.Tad[k] = w.Tn[sC][t][k];
          __syncthreads();
          lm_terms(P, w, w.qad, w.dch[sC][t], nullptr, w.lagA, w.lagD, nullptr, w.Tad, &bad);
        }
      }
      const int tmp = sX; sX = sC; sC = tmp;   // iteration l+1 becomes the lag source
    }
    const int old = sK; sK = sX; sX = old;     // S7
  }
  double *qo = P.q_out + (size_t)inst * nF;
  for (int e = tid; e < nF; e += nt) qo[e] = w.q[sK][M][e];
  __syncthreads();
  if (P.peos) {
    for (int k = tid; k < nx; k += nt) w.Tad[k] = w.Tn[sK][M][k];
    __syncthreads();
    lm_terms(P, w, w.q[sK][M], nullptr, nullptr, nullptr, nullptr, nullptr, w.Tad, &bad);
    for (int k = tid; k < nx; k += nt) P.peos[(size_t)inst * nx + k] = w.pe[k];
  }
  __syncthreads();
  if (tid == 0 && P.status) P.status[inst] = (int)bad;
}

// the inflow state: rho_in from the EOS at p0, h_in, and the species enthalpies at
// T_in (hdr = [Y_in (N), rho_in, h_in, h_i(T_in) (N)])
__global__ void k_lm_inflow(DevMech m, double T_in, double p0, double *hdr) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int N = m.N;
  double sw = 0.0, h = 0.0;
  for (int i = 0; i < N; ++i) {
    const double hi = lm_h(m, i, T_in);
    hdr[N + 2 + i] = hi;
    sw += hdr[i] * m.invW[i];
    h += hdr[i] * hi;
  }
  hdr[N] = p0 / (kRu * T_in * sw);
  hdr[N + 1] = h;
}

}  // namespace

// workspace of the low-Mach step: the inflow header, then n flames' node stacks
size_t lowmach_work_bytes(int N, int nx, int M, int n) {
  return (128 + lm_work_doubles(N, nx, M) * (size_t)n) * sizeof(double);
}

cudaError_t launch_lowmach(const DevMech &m, int nx, double dx, int M, const double *tau,
                           const double (*Q)[kMaxNodes + 1], const double (*QI)[kMaxNodes],
                           const double (*QE)[kMaxNodes], int scheme, int n_sweeps, int nu,
                           int i0, double rtol, int maxit, double dt, double U_in, double T_in,
                           double p0, int dchi, const double *Y_in_host, int n,
                           const double *q_in, double *q_out, double *peos, int *status,
                           double *ws, cudaStream_t s) {
  LmLaunch P;
  memset(&P, 0, sizeof(P));
  P.m = m;
  P.nx = nx; P.M = M; P.n_sweeps = n_sweeps; P.nu = nu; P.scheme = scheme; P.i0 = i0;
  P.maxit = maxit; P.dchi = dchi; P.n = n;
  P.dx = dx; P.dt = dt; P.U_in = U_in; P.T_in = T_in; P.p0 = p0;
  P.rtol = rtol;
  for (int j = 0; j <= M; ++j) P.tau[j] = tau[j];
  for (int t = 0; t < M; ++t) {
    for (int j = 0; j <= M; ++j) P.Q[t][j] = Q[t][j];
    for (int j = 0; j < M; ++j) { P.QI[t][j] = QI[t][j]; P.QE[t][j] = QE[t][j]; }
  }
  const int N = m.N;
  cudaError_t e = cudaMemcpyAsync(ws, Y_in_host, N * sizeof(double), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  k_lm_inflow<<<1, 32, 0, s>>>(m, T_in, p0, ws);
  P.Y_in = ws; P.rho_h_in = ws + N; P.hsp_in = ws + N + 2;
  P.q_in = q_in; P.q_out = q_out; P.peos = peos;
  P.status = status; P.ws = ws + 128; P.per_flame = lm_work_doubles(N, nx, M);
  k_lowmach<<<n, kLmThreads, 0, s>>>(P);
  return cudaGetLastError();
}

}  // namespace misdc
