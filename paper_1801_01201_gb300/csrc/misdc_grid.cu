// Grid kernels: spectral-integration / right-hand-side linear combinations,
// the advection-diffusion right-hand sides (Sec. 2 operators, steps S3, S4, S6)
// and the implicit diffusion solve of steps S3-S4 (Chebyshev-accelerated
// Jacobi smoother, multigrid V-cycles, flux-form reconstruction, closure).
//
// Layout: field-major [field][cells], cells x-fastest, periodic grid.
#include <math.h>

#include <algorithm>
#include <vector>

#include "misdc_internal.cuh"

namespace misdc {

namespace {

struct FieldMap {
  int nfs;                  // number of solved fields (all but the dominant species)
  int fld[kMaxSpecies + 1]; // physical field of each solved field
  double cf[kMaxSpecies + 1];   // wdt * diffusivity / dx^2
};

struct Nbr {
  int cm2[3], cm[3], cp[3], cp2[3];
};

__device__ __forceinline__ unsigned long long dbits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__device__ __forceinline__ Nbr neighbours(const DevGrid &g, int c) {
  Nbr b;
  const int x = c % g.nx, y = (c / g.nx) % g.ny, z = c / (g.nx * g.ny);
  const int sx = 1, sy = g.nx, sz = g.nx * g.ny;
  const int base[3] = {c - x * sx, c - y * sy, c - z * sz};
  const int pos[3] = {x, y, z}, n[3] = {g.nx, g.ny, g.nz}, str[3] = {sx, sy, sz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int p = pos[d], nn = n[d];
    b.cm2[d] = base[d] + wrapi(wrapi(p - 2, nn), nn) * str[d];
    b.cm[d] = base[d] + wrapi(p - 1, nn) * str[d];
    b.cp[d] = base[d] + wrapi(p + 1, nn) * str[d];
    b.cp2[d] = base[d] + wrapi(wrapi(p + 2, nn), nn) * str[d];
  }
  return b;
}

// ---------------------------------------------------------------------------
// out[o][e] = sum_k w[o][k] in[k][e] with the input and output counts fixed at
// compile time (NI inputs, NO outputs): exactly NI x NO FMAs and NI loads per
// element, every load of a thread issued before its first FMA
template <int NO, int NI>
__global__ void __launch_bounds__(256) k_lincomb_t(LinComb lc, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    double v[NI];
#pragma unroll
    for (int k = 0; k < NI; ++k) v[k] = lc.in[k][e];
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < NI; ++k) acc = fma(lc.w[o][k], v[k], acc);
      lc.out[o][e] = acc;
    }
  }
}

// any other count (at most 8 outputs, 16 inputs)
__global__ void k_lincomb(LinComb lc, size_t n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n;
       e += (size_t)gridDim.x * blockDim.x) {
    double v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = (k < lc.n_in) ? lc.in[k][e] : 0.0;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      if (o < lc.n_out) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (k < lc.n_in) s = fma(lc.w[o][k], v[k], s);
        lc.out[o][e] = s;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// F_E (advection of every field + explicit differential diffusion of h) and
// F_D (implicit diffusion, dominant species closed by minus the sum), in two
// passes so that every face is evaluated once (FP64 instructions bound these
// kernels): k_faces writes, for the low face of every cell along every used
// direction, the advective flux, the diffusive flux and the differential-diffusion
// flux of h; k_divergence differences them.
//
// Face buffer (per direction d, quantity q, cell c at fb[(d * (2N+3) + q) * cs + c]):
//   q = f (0..N):       A_f = u (7 (x_{c-1} + x_c) - (x_{c-2} + x_{c+1}))   (12 x the
//                        fourth-order face value times the face velocity)
//   q = N + 1 + f:      D_f = theta_face (x_c - x_{c-1})                  (f != i0)
//   q = 2N + 2:         Q = theta_face (hbar0 G + q), the differential diffusion of h
//                        of eq. enthalpy_equation with the dominant species' flux
//                        minus the others':  q = sum_i (h_i,l + h_i,r)(Y_i,r - Y_i,l)
//                        (alpha0 - D_i) (D_i -> 0 for i0), G = sum_{i != i0} D_i
//                        (Y_i,r - Y_i,l), hbar0 = h_i0,l + h_i0,r
// The 1/12, 1/dx, 1/dx^2, 1/2 and the per-field D0 are applied in k_divergence.
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void k_faces(DevMech m, DevGrid g, int i0, const double *__restrict__ phi,
                        const double *__restrict__ hsp, const double *__restrict__ thf,
                        const double *__restrict__ vel, double *__restrict__ fb) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int cs = g.cells;
  if (c >= cs) return;
  const int N = m.N, FB = 2 * N + 3;
  const Nbr nb = neighbours(g, c);
  double u[DIM], th[DIM], sq[DIM], sg[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    u[d] = vel[(size_t)d * cs + c];
    th[d] = thf[(size_t)d * cs + c];
    sq[d] = sg[d] = 0.0;
  }
  for (int f = 0; f <= N; ++f) {
    const double *x = phi + (size_t)f * cs;
    const double xc = x[c];
    const bool sp = f < N;
    const double *hs = hsp + (size_t)f * cs;
    const double hc = sp ? hs[c] : 0.0;
    const double wf = sp ? (f != i0 ? m.alpha0 - m.D0[f] : m.alpha0) : 0.0;
    const double Df = (sp && f != i0) ? m.D0[f] : 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int cm = nb.cm[d];
      const double xm = x[cm];
      const double face12 = fma(7.0, xm + xc, -(x[nb.cm2[d]] + x[nb.cp[d]]));
      double *o = fb + (size_t)d * FB * cs + c;
      o[(size_t)f * cs] = u[d] * face12;
      const double dl = xc - xm;
      if (f != i0) o[(size_t)(N + 1 + f) * cs] = th[d] * dl;
      if (sp) {
        sq[d] = fma((hs[cm] + hc) * dl, wf, sq[d]);
        sg[d] = fma(Df, dl, sg[d]);
      }
    }
  }
  const double *hs0 = hsp + (size_t)i0 * cs;
  const double h0 = hs0[c];
#pragma unroll
  for (int d = 0; d < DIM; ++d)
    fb[((size_t)d * FB + 2 * N + 2) * cs + c] = th[d] * fma(hs0[nb.cm[d]] + h0, sg[d], sq[d]);
}

template <int DIM>
__global__ void k_divergence(DevMech m, DevGrid g, int i0, const double *__restrict__ fb,
                             double *__restrict__ FE, double *__restrict__ FD) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int cs = g.cells;
  if (c >= cs) return;
  const int N = m.N, FB = 2 * N + 3;
  const Nbr nb = neighbours(g, c);
  const double invdx = 1.0 / g.dx, invdx2 = invdx * invdx;
  const double adv = invdx / 12.0;
  int cp[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) cp[d] = nb.cp[d];
  // sum over directions of (value at the high face) - (value at the low face)
  auto div = [&](int q) {
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const double *a = fb + ((size_t)d * FB + q) * cs;
      s += a[cp[d]] - a[c];
    }
    return s;
  };
  double fd_i0 = 0.0;
  for (int f = 0; f <= N; ++f) {
    const double fa = div(f);
    if (f < N) {
      if (FE) FE[(size_t)f * cs + c] = -fa * adv;
      if (f != i0) {
        const double v = m.D0[f] * div(N + 1 + f) * invdx2;
        if (FD) FD[(size_t)f * cs + c] = v;
        fd_i0 -= v;
      }
    } else {
      if (FD) FD[(size_t)N * cs + c] = m.alpha0 * div(N + 1 + N) * invdx2;
      if (FE) FE[(size_t)N * cs + c] = -fa * adv - 0.5 * div(2 * N + 2) * invdx2;
    }
  }
  if (FD) FD[(size_t)i0 * cs + c] = fd_i0;
}

// theta at cells -> harmonic mean at the low face of each cell; inverse
// diagonal of I - c_f L_theta for every solved field; and (if rho_bits) the
// largest Gershgorin bound c S/(1 + c S) of the Jacobi iteration matrix over
// cells, for the largest c_f (bit pattern of a non-negative double).
__global__ void k_face_coef(DevGrid g, FieldMap fm, const double *__restrict__ theta,
                            double *__restrict__ thf, double *__restrict__ invdiag, double cmax,
                            unsigned long long *rho_bits, float *__restrict__ thf32,
                            float *__restrict__ invdiag32, double *__restrict__ cdiag) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int cs = g.cells;
  double ratio = 0.0;
  if (c < cs) {
    const Nbr nb = neighbours(g, c);
    const double tc = theta[c];
    double S = 0.0;
    for (int d = 0; d < g.dim; ++d) {
      const double a = theta[nb.cm[d]], b = theta[nb.cp[d]];
      const double lo = 2.0 * a * tc / (a + tc), hi = 2.0 * tc * b / (tc + b);
      thf[(size_t)d * cs + c] = lo;
      if (thf32) thf32[(size_t)d * cs + c] = (float)lo;
      S += lo + hi;
    }
    if (invdiag) {
      for (int k = 0; k < fm.nfs; ++k) {
        const double di = 1.0 / (1.0 + fm.cf[k] * S);
        invdiag[(size_t)k * cs + c] = di;
        if (invdiag32) invdiag32[(size_t)k * cs + c] = (float)di;
        if (cdiag) cdiag[(size_t)k * cs + c] = fm.cf[k] * di;
      }
    } else if (invdiag32) {
      // FP32 inner solves only (mixed precision): the diagonal in FP32
      const float Sf = (float)S;
      for (int k = 0; k < fm.nfs; ++k)
        invdiag32[(size_t)k * cs + c] = 1.0f / fmaf((float)fm.cf[k], Sf, 1.0f);
    }
    ratio = cmax * S / (1.0 + cmax * S);
  }
  if (rho_bits) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ratio = fmax(ratio, __shfl_xor_sync(0xffffffffu, ratio, o));
    if ((threadIdx.x & 31) == 0 && ratio > 0.0)
      atomicMax(rho_bits, (unsigned long long)__double_as_longlong(ratio));
  }
}

// Chebyshev plan from the measured bound: sweep count K (at most kmax) for an
// error reduction `red`, and the weights omega_k of the semi-iterative method.
__global__ void k_cheb_plan(const unsigned long long *rho_bits, int kmax, double red, int *kdev,
                            double *omega, DevStats *st, int solves) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double rho = __longlong_as_double((long long)*rho_bits) * (1.0 + 1e-12);
  int K = 1;
  if (rho > 0.0) {
    if (rho >= 1.0) rho = 1.0 - 1e-12;
    K = (int)ceil(acosh(1.0 / red) / acosh(1.0 / rho));
  }
  K = max(1, min(K, kmax));
  *kdev = K;
  if (st) atomicAdd(&st->lin_sweeps, (unsigned long long)K * solves);   // sweeps per field
  const double r2 = rho * rho;
  double om = 1.0;
  for (int k = 0; k < K; ++k) {
    if (k == 1) om = 1.0 / (1.0 - 0.5 * r2);
    else if (k > 1) om = 1.0 / (1.0 - 0.25 * r2 * om);
    omega[k] = om;
  }
}

// ---- mixed precision: iterative refinement with FP32 inner Chebyshev solves
// x_{j+1} = x_j + e_j, A e_j = r_j = b - A x_j solved approximately in FP32 from
// e_j = 0; r_j and the update in FP64.

// r32 = b - A x (A = I - c_f L_theta) for every solved field: the FP64 residual
// of the round's iterate x, rounded to FP32 for the inner solve. In the last
// round (q != NULL) also q = b + c_f L_theta x in FP64: the flux-form
// reconstruction of x, to which the finish adds that of the round's correction.
template <int DIM>
__global__ void k_refine_residual(DevGrid g, FieldMap fm, const double *__restrict__ thf,
                                  const double *__restrict__ rhs, const double *__restrict__ x,
                                  float *__restrict__ r32, double *__restrict__ q) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int cs = g.cells;
  if (c >= cs) return;
  const Nbr nb = neighbours(g, c);
  double tlo[DIM], thi[DIM];
  int cm[DIM], cp[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    cm[d] = nb.cm[d];
    cp[d] = nb.cp[d];
    tlo[d] = thf[(size_t)d * cs + c];
    thi[d] = thf[(size_t)d * cs + cp[d]];
  }
  const int k0 = blockIdx.y * 4, k1 = min(fm.nfs, k0 + 4);
  for (int k = k0; k < k1; ++k) {
    const size_t off = (size_t)fm.fld[k] * cs;
    const double *xf = x + off;
    const double xc = xf[c];
    double L = thi[0] * (xf[cp[0]] - xc);
    L = fma(-tlo[0], xc - xf[cm[0]], L);
#pragma unroll
    for (int d = 1; d < DIM; ++d) {
      L = fma(thi[d], xf[cp[d]] - xc, L);
      L = fma(-tlo[d], xc - xf[cm[d]], L);
    }
    const double qv = fma(fm.cf[k], L, rhs[off + c]);
    r32[off + c] = (float)(qv - xc);
    if (q) q[off + c] = qv;
  }
}

// one FP32 Chebyshev-accelerated Jacobi sweep of A e = r from e = 0 (same method
// as k_cheb; weights from the FP64 plan of the inner reduction)
template <int DIM>
__global__ void k_cheb32(DevGrid g, FieldMap fm, const float *__restrict__ thf,
                         const float *__restrict__ invdiag, const float *__restrict__ rhs,
                         const float *__restrict__ xk, const float *__restrict__ xkm1,
                         float *__restrict__ xkp1, int it, const int *__restrict__ kdev,
                         const double *__restrict__ omega, const double *__restrict__ xbase,
                         double *__restrict__ xnext) {
  const int K = *kdev;
  if (it >= K) return;
  const bool last = (it == K - 1);   // the last planned sweep also forms x + e in FP64
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int cs = g.cells;
  if (c >= cs) return;
  const Nbr nb = neighbours(g, c);
  float tlo[DIM], thi[DIM];
  int cm[DIM], cp[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    cm[d] = nb.cm[d];
    cp[d] = nb.cp[d];
    tlo[d] = thf[(size_t)d * cs + c];
    thi[d] = thf[(size_t)d * cs + cp[d]];
  }
  const float om = (float)omega[it];
  const int k0 = blockIdx.y * 4, k1 = min(fm.nfs, k0 + 4);
  for (int k = k0; k < k1; ++k) {
    const size_t off = (size_t)fm.fld[k] * cs;
    const float cf = (float)fm.cf[k];
    float y, v;
    if (it == 0) {   // e_0 = 0: the first sweep is D^{-1} r
      y = rhs[off + c] * invdiag[(size_t)k * cs + c];
      v = y;
    } else {
      const float *x = xk + off;
      float sx = 0.0f;
#pragma unroll
      for (int d = 0; d < DIM; ++d) sx += thi[d] * x[cp[d]] + tlo[d] * x[cm[d]];
      y = (rhs[off + c] + cf * sx) * invdiag[(size_t)k * cs + c];
      const float prev = xkm1 ? xkm1[off + c] : 0.0f;
      v = fmaf(om, y - prev, prev);
    }
    xkp1[off + c] = v;
    if (last && xnext) xnext[off + c] = xbase[off + c] + (double)v;
  }
}

// First sweep of the first refinement round, whose iterate is the right-hand
// side itself: its residual b - A b = c_f L_theta b is formed here in FP32 from
// the FP64 differences of b rounded to FP32 (relative error ~1e-7 of c L b, below
// the inner solve's own 1e-6 reduction; the FP64 residual of the next round
// corrects both), stored for the later sweeps, and
// the sweep from e_0 = 0 is e_1 = D^{-1} r. A single planned sweep also writes
// x + e in FP64.
template <int DIM>
__global__ void k_cheb32_first(DevGrid g, FieldMap fm, const float *__restrict__ thf,
                               const float *__restrict__ invdiag, const double *__restrict__ b,
                               float *__restrict__ r32, float *__restrict__ e1,
                               const int *__restrict__ kdev, double *__restrict__ xnext) {
  const bool last = (*kdev == 1);
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int cs = g.cells;
  if (c >= cs) return;
  const Nbr nb = neighbours(g, c);
  float tlo[DIM], thi[DIM];
  int cm[DIM], cp[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    cm[d] = nb.cm[d];
    cp[d] = nb.cp[d];
    tlo[d] = thf[(size_t)d * cs + c];
    thi[d] = thf[(size_t)d * cs + cp[d]];
  }
  const int k0 = blockIdx.y * 4, k1 = min(fm.nfs, k0 + 4);
  for (int k = k0; k < k1; ++k) {
    const size_t off = (size_t)fm.fld[k] * cs;
    const double *x = b + off;
    const double xd = x[c];
    // differences in FP64, rounded after: a field of large offset and small
    // variation (the enthalpy) keeps its differences to FP32 precision
    float L = 0.0f;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      L = fmaf(thi[d], (float)(x[cp[d]] - xd), L);
      L = fmaf(-tlo[d], (float)(xd - x[cm[d]]), L);
    }
    const float r = (float)fm.cf[k] * L;
    r32[off + c] = r;
    const float v = r * invdiag[(size_t)k * cs + c];
    e1[off + c] = v;
    if (last && xnext) xnext[off + c] = xd + (double)v;
  }
}

// Finish of the mixed-precision solve: with the last round's iterate x_r, its
// reconstruction q = b + c_f L x_r (FP64) and the round's correction e (FP32,
// the buffer of the last planned sweep), the solution x = x_r + e is
// reconstructed in flux form as v = q + c_f L e (L e in FP32: e is the small
// correction of an FP32 inner solve), its residual r = v - x checked against
// |b| + |c_f L x| + |x|, and the dominant species closed by 1 - sum.
template <int DIM>
__global__ void k_finish32(DevGrid g, FieldMap fm, int N, int i0, double tol,
                           const float *__restrict__ thf, const double *__restrict__ rhs,
                           const double *__restrict__ q, const double *__restrict__ xr,
                           const float *e0, const float *e1, const float *e2,
                           const int *__restrict__ kdev, double *__restrict__ out, DevStats *st) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int cs = g.cells;
  const int sl = (*kdev - 1) % 3;
  const float *e = sl == 0 ? e0 : (sl == 1 ? e1 : e2);
  float rmax = 0.0f;
  if (c < cs) {
    int cm[DIM], cp[DIM];
    float tlo[DIM], thi[DIM];
    {
      const Nbr nb = neighbours(g, c);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        cm[d] = nb.cm[d];
        cp[d] = nb.cp[d];
        tlo[d] = thf[(size_t)d * cs + c];
        thi[d] = thf[(size_t)d * cs + cp[d]];
      }
    }
    double sum = 0.0;
    for (int k = 0; k < fm.nfs; ++k) {
      const int f = fm.fld[k];
      const size_t off = (size_t)f * cs;
      const float *ef = e + off;
      const float ec = ef[c];
      float Le = 0.0f;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        Le = fmaf(thi[d], ef[cp[d]] - ec, Le);
        Le = fmaf(-tlo[d], ec - ef[cm[d]], Le);
      }
      const double v = q[off + c] + (double)((float)fm.cf[k] * Le);
      const double x = xr[off + c] + (double)ec;
      const double b = rhs[off + c];
      const double r = v - x;
      const double scale = fabs(b) + fabs(v - b) + fabs(x) + 1e-300;
      rmax = fmaxf(rmax, __double2float_ru(fabs(r)) / fmaxf(__double2float_rd(scale), 1e-30f));
      out[off + c] = v;
      if (f < N) sum += v;
    }
    out[(size_t)i0 * cs + c] = 1.0 - sum;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0 && rmax > 0.0f) {
    atomicMax(&st->lin_resid_bits, dbits((double)rmax));
    if (!((double)rmax <= tol)) atomicOr(&st->status_bits, kBitMG);
  }
}

template <class T>
__device__ __forceinline__ T lap_theta(const DevGrid &g, const Nbr &nb, int c, int cs,
                                       const T *__restrict__ thf, const T *__restrict__ x) {
  const T xc = x[c];
  T s = 0;
  for (int d = 0; d < g.dim; ++d)
    s += thf[(size_t)d * cs + nb.cp[d]] * (x[nb.cp[d]] - xc) - thf[(size_t)d * cs + c] * (xc - x[nb.cm[d]]);
  return s;
}

// One Chebyshev-accelerated Jacobi sweep for every solved field:
// y = D^{-1} (b + c_f * offdiag(x_k)), x_{k+1} = omega (y - x_{k-1}) + x_{k-1}.
// A thread takes one cell and kChebFields fields (neighbour indices and face
// coefficients loaded once). Sweeps it >= *kdev (the device-planned count) do nothing.
constexpr int kChebFields = 4;
template <int DIM>
__global__ void k_cheb(DevGrid g, FieldMap fm, const double *__restrict__ thf,
                       const double *__restrict__ invdiag, const double *__restrict__ cdiag,
                       double *__restrict__ bdiag, const double *__restrict__ rhs,
                       const double *__restrict__ xk, const double *__restrict__ xkm1,
                       double *__restrict__ xkp1, int it, const int *__restrict__ kdev,
                       const double *__restrict__ omega) {
  if (it >= *kdev) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int cs = g.cells;
  if (c >= cs) return;
  const Nbr nb = neighbours(g, c);
  double tlo[DIM], thi[DIM];
  int cm[DIM], cp[DIM];
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    cm[d] = nb.cm[d];
    cp[d] = nb.cp[d];
    tlo[d] = thf[(size_t)d * cs + c];
    thi[d] = thf[(size_t)d * cs + cp[d]];
  }
  const double om = omega[it];
  const int k0 = blockIdx.y * kChebFields, k1 = min(fm.nfs, k0 + kChebFields);
  for (int k = k0; k < k1; ++k) {
    const size_t off = (size_t)fm.fld[k] * cs, kc = (size_t)k * cs + c;
    const double *x = xk + off;
    // neighbour sum as one FMA chain (FP64 instructions, not bytes, bound this sweep)
    double s = thi[0] * x[cp[0]];
    s = fma(tlo[0], x[cm[0]], s);
#pragma unroll
    for (int d = 1; d < DIM; ++d) {
      s = fma(thi[d], x[cp[d]], s);
      s = fma(tlo[d], x[cm[d]], s);
    }
    // Jacobi value D^{-1} (rhs + c_f s) = b~ + c~ s: c~ = c_f D^{-1} comes with the
    // diagonal, b~ = D^{-1} rhs is formed by sweep 0 and kept for the later sweeps
    double bt;
    if (it == 0) {
      bt = rhs[off + c] * invdiag[kc];
      bdiag[kc] = bt;
    } else {
      bt = bdiag[kc];
    }
    const double y = fma(cdiag[kc], s, bt);
    xkp1[off + c] = (it == 0) ? y : fma(om, y - xkm1[off + c], xkm1[off + c]);
  }
}


// Residual check, flux-form reconstruction x := rhs + c_f L x, and closure of
// the dominant species. Writes the advection-diffusion state.
template <int DIM>
__global__ void k_finish(DevGrid g, FieldMap fm, int N, int i0, double tol,
                         const double *__restrict__ thf, const double *__restrict__ rhs,
                         const double *x0, const double *x1, const double *x2,
                         const int *kdev, double *__restrict__ out, DevStats *st) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int cs = g.cells;
  double rmax = 0.0;
  // final iterate: x0 alone, or the buffer the last planned sweep wrote
  const double *x = x0;
  if (kdev) {
    const int K = *kdev, sl = (K - 1) % 3;
    x = sl == 0 ? x0 : (sl == 1 ? x1 : x2);
  }
  if (c < cs) {
    // neighbour indices and face coefficients once per cell (not per field)
    int cm[DIM], cp[DIM];
    double tlo[DIM], thi[DIM];
    {
      const Nbr nb = neighbours(g, c);
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        cm[d] = nb.cm[d];
        cp[d] = nb.cp[d];
        tlo[d] = thf[(size_t)d * cs + c];
        thi[d] = thf[(size_t)d * cs + cp[d]];
      }
    }
    double sum = 0.0;
    for (int k = 0; k < fm.nfs; ++k) {
      const int f = fm.fld[k];
      const size_t off = (size_t)f * cs;
      const double *xf = x + off;
      const double xc = xf[c];
      double L = 0.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) L += thi[d] * (xf[cp[d]] - xc) - tlo[d] * (xc - xf[cm[d]]);
      const double b = rhs[off + c];
      const double cl = fm.cf[k] * L;
      const double scale = fabs(b) + fabs(cl) + fabs(xc) + 1e-300;
      const double r = b - (xc - cl);
      // diagnostic ratio in FP32 (FP64 divisions are scarce on this part)
      rmax = fmax(rmax, (double)(__double2float_ru(fabs(r)) / fmaxf(__double2float_rd(scale), 1e-30f)));
      const double v = b + cl;
      out[off + c] = v;
      if (f < N) sum += v;
    }
    out[(size_t)i0 * cs + c] = 1.0 - sum;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  if ((threadIdx.x & 31) == 0 && rmax > 0.0) {
    atomicMax(&st->lin_resid_bits, dbits(rmax));
    if (!(rmax <= tol)) atomicOr(&st->status_bits, kBitMG);
  }
}

void launch_finish(const DevGrid &g, const FieldMap &fm, int N, int i0, double tol, const double *thf,
                   const double *rhs, const double *x0, const double *x1, const double *x2,
                   const int *kdev, double *out, DevStats *st, cudaStream_t s) {
  const int blocks = (g.cells + 255) / 256;
  if (g.dim == 1)
    k_finish<1><<<blocks, 256, 0, s>>>(g, fm, N, i0, tol, thf, rhs, x0, x1, x2, kdev, out, st);
  else if (g.dim == 2)
    k_finish<2><<<blocks, 256, 0, s>>>(g, fm, N, i0, tol, thf, rhs, x0, x1, x2, kdev, out, st);
  else
    k_finish<3><<<blocks, 256, 0, s>>>(g, fm, N, i0, tol, thf, rhs, x0, x1, x2, kdev, out, st);
}

// ---- multigrid (cell-centred, coarsening by 2 in every used direction) on
// compact [solved field][cells] storage. Level kernels are templated on the
// storage type: FP64 everywhere in FP64 mode; in mixed precision the fine level
// stays FP64 (its residual decides convergence) and the coarse levels run in FP32.
// Every level kernel returns at once when *done is set (the fine residual met the
// target); smoothing counts are even, so a skipped pair leaves the iterate in the
// buffer the host expects.

// restriction: coarse residual = mean of the 2^dim fine residuals
template <class TF, class TC>
__global__ void k_restrict(DevGrid gf, DevGrid gc, const TF *__restrict__ rf, TC *__restrict__ rc,
                           const int *__restrict__ done) {
  if (*done) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (c >= gc.cells) return;
  const int X = c % gc.nx, Y = (c / gc.nx) % gc.ny, Z = c / (gc.nx * gc.ny);
  const int sx = gf.dim > 0 ? 2 : 1, sy = gf.dim > 1 ? 2 : 1, sz = gf.dim > 2 ? 2 : 1;
  TF s = 0;
  for (int dz = 0; dz < sz; ++dz)
    for (int dy = 0; dy < sy; ++dy)
      for (int dx = 0; dx < sx; ++dx)
        s += rf[(size_t)k * gf.cells + (size_t)(X * sx + dx) + gf.nx * ((size_t)(Y * sy + dy) + (size_t)gf.ny * (Z * sz + dz))];
  rc[(size_t)k * gc.cells + c] = (TC)(s * ((TF)1 / (TF)(sx * sy * sz)));   // 1/2^d: exact
}

// prolongation: fine correction += coarse value of the parent cell
template <class TC, class TF>
__global__ void k_prolong(DevGrid gf, DevGrid gc, const TC *__restrict__ xc, TF *__restrict__ xf,
                          const int *__restrict__ done) {
  if (*done) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (c >= gf.cells) return;
  const int x = c % gf.nx, y = (c / gf.nx) % gf.ny, z = c / (gf.nx * gf.ny);
  const int X = gf.dim > 0 ? x / 2 : x, Y = gf.dim > 1 ? y / 2 : y, Z = gf.dim > 2 ? z / 2 : z;
  xf[(size_t)k * gf.cells + c] += (TF)xc[(size_t)k * gc.cells + X + gc.nx * (Y + gc.ny * Z)];
}

// coarse face coefficient: mean of the fine faces that tile the coarse face
template <class TF, class TC>
__global__ void k_coarsen_faces(DevGrid gf, DevGrid gc, const TF *__restrict__ tf,
                                TC *__restrict__ tc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= gc.cells) return;
  const int X = c % gc.nx, Y = (c / gc.nx) % gc.ny, Z = c / (gc.nx * gc.ny);
  for (int d = 0; d < gf.dim; ++d) {
    TF s = 0;
    int cnt = 0;
    const int ox = (d == 0) ? 1 : 2, oy = (gf.dim > 1) ? ((d == 1) ? 1 : 2) : 1,
              oz = (gf.dim > 2) ? ((d == 2) ? 1 : 2) : 1;
    for (int dz = 0; dz < oz; ++dz)
      for (int dy = 0; dy < oy; ++dy)
        for (int dx = 0; dx < ox; ++dx) {
          const int fx = (gf.dim > 0 ? 2 * X : X) + dx, fy = (gf.dim > 1 ? 2 * Y : Y) + dy,
                    fz = (gf.dim > 2 ? 2 * Z : Z) + dz;
          s += tf[(size_t)d * gf.cells + fx + (size_t)gf.nx * (fy + (size_t)gf.ny * fz)];
          ++cnt;
        }
    tc[(size_t)d * gc.cells + c] = (TC)(s / (TF)cnt);
  }
}

// residual r = b - (I - c L) x on one level for the solved fields; on the fine
// level (res_bits set) also the largest scaled residual |r| / (|b| + |c L x| + |x|)
// of the launch (the scale of the final check), the convergence measure of the
// V-cycles
template <class T>
__global__ void k_residual(DevGrid g, FieldMap fm, const T *__restrict__ thf,
                           const T *__restrict__ b, const T *__restrict__ x, T *__restrict__ r,
                           const int *__restrict__ done, unsigned long long *res_bits) {
  if (*done) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  float q = 0.0f;
  if (c < g.cells) {
    const Nbr nb = neighbours(g, c);
    const size_t off = (size_t)k * g.cells;
    const T xc = x[off + c], bc = b[off + c];
    const T cl = (T)fm.cf[k] * lap_theta<T>(g, nb, c, g.cells, thf, x + off);
    const T rc = bc - (xc - cl);
    r[off + c] = rc;
    // the ratio in FP32, rounded up (FP64 divisions are scarce on this part)
    if (res_bits)
      q = __double2float_ru(fabs((double)rc)) /
          fmaxf(__double2float_rd(fabs((double)bc) + fabs((double)cl) + fabs((double)xc)), 1e-30f);
  }
  if (!res_bits) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) q = fmaxf(q, __shfl_xor_sync(0xffffffffu, q, o));
  if ((threadIdx.x & 31) == 0 && q > 0.0f) atomicMax(res_bits, dbits((double)q));
}

// after the fine residual of a V-cycle: stop the cycles once it meets the target;
// counts the fine smoothing sweeps that ran (two before the residual, two after
// it unless the cycles stop here)
// (in a WHILE graph body: also ends the loop once done or after `cap` cycles, and
// counts the body's kernels)
__global__ void k_mg_check(unsigned long long *res_bits, double tol, int *done, DevStats *st,
                           int *cycle, int cap, cudaGraphConditionalHandle h, int body_kernels) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (body_kernels) {
    atomicAdd(&st->body_launches, (unsigned long long)body_kernels);
    if (*done || ++*cycle >= cap) cudaGraphSetConditional(h, 0);
  }
  if (*done) return;
  const double r = __longlong_as_double((long long)*res_bits);
  *res_bits = 0ull;
  const bool stop = r <= tol;
  if (stop) {
    *done = 1;
    if (body_kernels) cudaGraphSetConditional(h, 0);
  }
  atomicAdd(&st->lin_sweeps, stop ? 2ull : 4ull);
}

// damped Jacobi on one level: y = x + w D^{-1} (b - A x)
template <class T>
__global__ void k_jacobi_level(DevGrid g, FieldMap fm, const T *__restrict__ thf,
                               const T *__restrict__ invdiag, const T *__restrict__ b,
                               const T *__restrict__ x, T *__restrict__ y, T w,
                               const int *__restrict__ done) {
  if (*done) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (c >= g.cells) return;
  const Nbr nb = neighbours(g, c);
  const size_t off = (size_t)k * g.cells;
  const T r = b[off + c] - (x[off + c] - (T)fm.cf[k] * lap_theta<T>(g, nb, c, g.cells, thf, x + off));
  y[off + c] = fma(w * invdiag[off + c], r, x[off + c]);
}

template <class T>
__global__ void k_diag_level(DevGrid g, FieldMap fm, const T *__restrict__ thf,
                             T *__restrict__ invdiag) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= g.cells) return;
  const Nbr nb = neighbours(g, c);
  T S = 0;
  for (int d = 0; d < g.dim; ++d) S += thf[(size_t)d * g.cells + c] + thf[(size_t)d * g.cells + nb.cp[d]];
  for (int k = 0; k < fm.nfs; ++k) invdiag[(size_t)k * g.cells + c] = (T)1 / ((T)1 + (T)fm.cf[k] * S);
}

// ---- adaptive nested iterations: per field, max |now - before| and max |now|
// over the nodes' cells (bit patterns of non-negative doubles, so integer max)
__global__ void k_nu_incr(int cs, int M, NodePtrs now, NodePtrs before,
                          unsigned long long *__restrict__ bits) {
  const int f = blockIdx.y;
  double dm = 0.0, sm = 0.0;
  for (int m = 0; m < M; ++m) {
    const double *a = now.p[m] + (size_t)f * cs, *b = before.p[m] + (size_t)f * cs;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cs; c += gridDim.x * blockDim.x) {
      const double x = a[c];
      dm = fmax(dm, fabs(x - b[c]));
      sm = fmax(sm, fabs(x));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    sm = fmax(sm, __shfl_xor_sync(0xffffffffu, sm, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (dm > 0.0) atomicMax(&bits[2 * f], dbits(dm));
    if (sm > 0.0) atomicMax(&bits[2 * f + 1], dbits(sm));
  }
}

__global__ void k_nu_decide(int F, int l, int nu, double eta, double rho,
                            unsigned long long *bits, double *delta, int *cont, int *ran,
                            DevStats *st, cudaGraphConditionalHandle h, int has_h,
                            const int *body_kernels) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (body_kernels) atomicAdd(&st->body_launches, (unsigned long long)*body_kernels);
  double d = 0.0;
  for (int f = 0; f < F; ++f) {
    const double dm = __longlong_as_double((long long)bits[2 * f]);
    const double sm = __longlong_as_double((long long)bits[2 * f + 1]);
    if (sm > 0.0) d = fmax(d, dm / sm);
    bits[2 * f] = bits[2 * f + 1] = 0ull;
  }
  delta[l] = d;
  const bool go = l + 1 < nu && (l < 1 || (d > eta * delta[0] && d < rho * delta[l - 1]));
  *cont = go ? 1 : 0;
  *ran = l + 1;
  if (!go) atomicAdd(&st->nested_iters, (unsigned long long)(l + 1));
  if (has_h) cudaGraphSetConditional(h, go ? 1u : 0u);
}

__global__ void k_copy_if_parity(CopyList cl, const int *ran, int parity) {
  if (((*ran - 1) & 1) == parity) return;
  const int k = blockIdx.y;
  const size_t n = cl.n[k];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    cl.dst[k][i] = cl.src[k][i];
}

// gather the solved fields of a full-layout array into compact storage and back
// (with kdev: from the buffer the last planned Chebyshev sweep wrote)
__global__ void k_gather(int cs, FieldMap fm, const double *f0, const double *f1, const double *f2,
                         const int *kdev, double *__restrict__ compact) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (c >= cs) return;
  const double *full = f0;
  if (kdev) {
    const int sl = (*kdev - 1) % 3;
    full = sl == 0 ? f0 : (sl == 1 ? f1 : f2);
  }
  compact[(size_t)k * cs + c] = full[(size_t)fm.fld[k] * cs + c];
}
__global__ void k_scatter_set(int cs, FieldMap fm, const double *__restrict__ compact, double *__restrict__ full) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (c >= cs) return;
  full[(size_t)fm.fld[k] * cs + c] = compact[(size_t)k * cs + c];
}

inline dim3 grid2(int cells, int nf) { return dim3((cells + 255) / 256, nf); }

FieldMap make_map(const DevMech &m, const double *D0h, double alpha0, int i0, double wdt, double dx) {
  FieldMap fm;
  fm.nfs = 0;
  for (int f = 0; f <= m.N; ++f) {
    if (f == i0) continue;
    fm.fld[fm.nfs] = f;
    fm.cf[fm.nfs] = wdt * ((f < m.N) ? D0h[f] : alpha0) / (dx * dx);
    ++fm.nfs;
  }
  return fm;
}

}  // namespace

int chebyshev_sweeps(double rho_bound, double reduction) {
  if (rho_bound <= 0.0) return 1;
  const double a = acosh(1.0 / rho_bound);
  const double need = acosh(1.0 / reduction);
  return std::max(1, (int)ceil(need / a));
}

namespace {
template <int NO, int NI>
bool lincomb_fixed(const LinComb &lc, size_t n, unsigned blocks, cudaStream_t s) {
  if (lc.n_in == NI) {
    k_lincomb_t<NO, NI><<<blocks, 256, 0, s>>>(lc, n);
    return true;
  }
  if constexpr (NI > 1) return lincomb_fixed<NO, NI - 1>(lc, n, blocks, s);
  return false;
}
}  // namespace

void launch_lincomb(const LinComb &lc, size_t n, cudaStream_t s) {
  if (!n) return;
  size_t blocks = (n + 255) / 256;
  if (blocks > 65535 * 8) blocks = 65535 * 8;
  const unsigned b = (unsigned)blocks;
  bool done = false;
  if (lc.n_out == 1) done = lincomb_fixed<1, 12>(lc, n, b, s);
  else if (lc.n_out == 2) done = lincomb_fixed<2, 12>(lc, n, b, s);
  if (!done) k_lincomb<<<b, 256, 0, s>>>(lc, n);
}

size_t operator_face_doubles(const DevGrid &g, int N) {
  return (size_t)g.dim * (2 * N + 3) * g.cells;
}

void launch_operators(const DevMech &m, const DevGrid &g, int i0, const double *phi,
                      const double *hsp, const double *theta_face, const double *vel,
                      double *FE, double *FD, double *faces, cudaStream_t s) {
  const int blocks = (g.cells + 127) / 128;
  if (g.dim == 1) {
    k_faces<1><<<blocks, 128, 0, s>>>(m, g, i0, phi, hsp, theta_face, vel, faces);
    k_divergence<1><<<blocks, 128, 0, s>>>(m, g, i0, faces, FE, FD);
  } else if (g.dim == 2) {
    k_faces<2><<<blocks, 128, 0, s>>>(m, g, i0, phi, hsp, theta_face, vel, faces);
    k_divergence<2><<<blocks, 128, 0, s>>>(m, g, i0, faces, FE, FD);
  } else {
    k_faces<3><<<blocks, 128, 0, s>>>(m, g, i0, phi, hsp, theta_face, vel, faces);
    k_divergence<3><<<blocks, 128, 0, s>>>(m, g, i0, faces, FE, FD);
  }
}

void launch_theta_faces(const DevGrid &g, const double *theta, double *thf, cudaStream_t s) {
  FieldMap fm;
  fm.nfs = 0;
  k_face_coef<<<(g.cells + 255) / 256, 256, 0, s>>>(g, fm, theta, thf, nullptr, 0.0, nullptr,
                                                     nullptr, nullptr, nullptr);
}

namespace {

// the storage of level l: FP32 for the coarse levels of a mixed-precision solve
template <class T> T *lv(double *d, float *f);
template <> double *lv<double>(double *d, float *) { return d; }
template <> float *lv<float>(double *, float *f) { return f; }

// n (even) damped-Jacobi sweeps on level l; the iterate ends in lx[l] again
template <class T>
void mg_smooth(DiffWork &w, const FieldMap &fm, int l, int n, cudaStream_t s) {
  const DevGrid &g = w.lg[l];
  T *x = lv<T>(w.lx[l], w.lx32[l]), *y = lv<T>(w.ly[l], w.ly32[l]);
  for (int sw = 0; sw < n; ++sw) {
    k_jacobi_level<T><<<grid2(g.cells, fm.nfs), 256, 0, s>>>(
        g, fm, lv<T>(w.lthf[l], w.lthf32[l]), lv<T>(w.linvdiag[l], w.linvdiag32[l]),
        lv<T>(w.lb[l], w.lb32[l]), x, y, (T)0.8, w.mg_done);
    std::swap(x, y);
  }
}

// residual of level l (with the convergence measure on the fine level), restricted
// into the right-hand side of level l+1, whose iterate starts from zero
struct CycleLoop {   // the WHILE node the cycles run in (body_kernels = 0: none)
  cudaGraphConditionalHandle h;
  int body_kernels;
};

template <class TF, class TC>
void mg_down(DiffWork &w, const FieldMap &fm, int l, const CycleLoop &loop, cudaStream_t s) {
  const DevGrid &gl = w.lg[l], &gc = w.lg[l + 1];
  TF *r = lv<TF>(w.lr[l], w.lr32[l]);
  k_residual<TF><<<grid2(gl.cells, fm.nfs), 256, 0, s>>>(
      gl, fm, lv<TF>(w.lthf[l], w.lthf32[l]), lv<TF>(w.lb[l], w.lb32[l]), lv<TF>(w.lx[l], w.lx32[l]),
      r, w.mg_done, l == 0 ? w.mg_res : nullptr);
  if (l == 0)
    k_mg_check<<<1, 32, 0, s>>>(w.mg_res, w.mg_tol, w.mg_done, w.mg_st, w.mg_cycle, w.cycles,
                                loop.h, loop.body_kernels);
  k_restrict<TF, TC><<<grid2(gc.cells, fm.nfs), 256, 0, s>>>(gl, gc, r, lv<TC>(w.lb[l + 1], w.lb32[l + 1]),
                                                             w.mg_done);
  cudaMemsetAsync(lv<TC>(w.lx[l + 1], w.lx32[l + 1]), 0, sizeof(TC) * (size_t)fm.nfs * gc.cells, s);
}

template <class TC, class TF>
void mg_up(DiffWork &w, const FieldMap &fm, int l, cudaStream_t s) {
  k_prolong<TC, TF><<<grid2(w.lg[l].cells, fm.nfs), 256, 0, s>>>(
      w.lg[l], w.lg[l + 1], lv<TC>(w.lx[l + 1], w.lx32[l + 1]), lv<TF>(w.lx[l], w.lx32[l]), w.mg_done);
}

template <class TF, class TC>
void mg_coarsen(DiffWork &w, const FieldMap &fc, int l, cudaStream_t s) {
  const DevGrid &gf = w.lg[l - 1], &gc = w.lg[l];
  TC *tc = lv<TC>(w.lthf[l], w.lthf32[l]);
  k_coarsen_faces<TF, TC><<<(gc.cells + 255) / 256, 256, 0, s>>>(gf, gc, lv<TF>(w.lthf[l - 1], w.lthf32[l - 1]), tc);
  k_diag_level<TC><<<(gc.cells + 255) / 256, 256, 0, s>>>(gc, fc, tc, lv<TC>(w.linvdiag[l], w.linvdiag32[l]));
}

// Multigrid solve of (I - c L) x = rhs for every solved field: V-cycles of the
// correction scheme from x0 = rhs, two damped-Jacobi sweeps before and after the
// coarse correction on every level and eight on the coarsest, mean-value
// restriction, piecewise-constant prolongation and coefficients re-discretised
// from the fine face coefficients (c / 4 per level). The cycles stop on the device
// once the scaled fine residual is below 10 lin_rtol, at most w.cycles of them; the
// solution goes to w.xa (full layout, the dominant-species row untouched).
void multigrid_solve(const DevGrid &g, const FieldMap &fm, const double *rhs, DiffWork &w,
                     double lin_rtol, DevStats *st, cudaStream_t s) {
  const int cs = g.cells, L = w.levels;
  const dim3 gr = grid2(cs, fm.nfs);
  auto f32 = [&](int l) { return w.mg32 && l >= 1; };
  w.lthf[0] = w.thf;
  w.linvdiag[0] = w.invdiag;
  FieldMap fl[8];
  fl[0] = fm;
  for (int l = 1; l < L; ++l) {
    fl[l] = fm;
    for (int k = 0; k < fm.nfs; ++k) fl[l].cf[k] = fm.cf[k] / (double)(1 << (2 * l));
    if (!f32(l)) mg_coarsen<double, double>(w, fl[l], l, s);
    else if (!f32(l - 1)) mg_coarsen<double, float>(w, fl[l], l, s);
    else mg_coarsen<float, float>(w, fl[l], l, s);
  }
  // the stop target sits 10x below the final check (100 lin_rtol, same measure):
  // the scaled residual bottoms out at round-off near lin_rtol itself
  w.mg_tol = 10.0 * lin_rtol;
  w.mg_st = st;
  cudaMemsetAsync(w.mg_done, 0, sizeof(int), s);
  cudaMemsetAsync(w.mg_res, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(w.mg_cycle, 0, sizeof(int), s);
  k_gather<<<gr, 256, 0, s>>>(cs, fm, rhs, nullptr, nullptr, nullptr, w.lb[0]);
  k_gather<<<gr, 256, 0, s>>>(cs, fm, rhs, nullptr, nullptr, nullptr, w.lx[0]);
  auto cycle = [&](const CycleLoop &loop, cudaStream_t q) {
    for (int l = 0; l + 1 < L; ++l) {          // down-leg
      if (f32(l)) {
        mg_smooth<float>(w, fl[l], l, 2, q);
        mg_down<float, float>(w, fl[l], l, loop, q);
      } else {
        mg_smooth<double>(w, fl[l], l, 2, q);
        if (f32(l + 1)) mg_down<double, float>(w, fl[l], l, loop, q);
        else mg_down<double, double>(w, fl[l], l, loop, q);
      }
    }
    if (f32(L - 1)) mg_smooth<float>(w, fl[L - 1], L - 1, 8, q);   // coarsest level
    else mg_smooth<double>(w, fl[L - 1], L - 1, 8, q);
    for (int l = L - 2; l >= 0; --l) {         // up-leg
      if (f32(l)) {
        mg_up<float, float>(w, fl[l], l, q);
        mg_smooth<float>(w, fl[l], l, 2, q);
      } else {
        if (f32(l + 1)) mg_up<float, double>(w, fl[l], l, q);
        else mg_up<double, double>(w, fl[l], l, q);
        mg_smooth<double>(w, fl[l], l, 2, q);
      }
    }
  };
  // kernels in one cycle: smoothing 2 per level above the coarsest and back, 8 on
  // the coarsest, residual + restriction + prolongation per level above it, the check
  const int per_cycle = 4 * (L - 1) + 8 + 3 * (L - 1) + 1;
  CycleLoop loop{0, 0};
  cudaGraph_t body = w.mg_stream ? graph_conditional(s, cudaGraphCondTypeWhile, 1, &loop.h) : nullptr;
  if (body) {
    // captured: one cycle is the body of a WHILE node that the check ends
    loop.body_kernels = per_cycle;
    cudaStreamBeginCaptureToGraph(w.mg_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    cycle(loop, w.mg_stream);
    cudaStreamEndCapture(w.mg_stream, &body);
  } else {
    for (int cyc = 0; cyc < w.cycles; ++cyc) cycle(loop, s);
  }
  k_scatter_set<<<gr, 256, 0, s>>>(cs, fm, w.lx[0], w.xa);
}

}  // namespace

bool graph_conditional_handle(cudaStream_t s, unsigned dflt, cudaGraphConditionalHandle *h) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess ||
      cs != cudaStreamCaptureStatusActive)
    return false;
  return cudaGraphConditionalHandleCreate(h, g, dflt, cudaGraphCondAssignDefault) == cudaSuccess;
}

cudaGraph_t graph_conditional(cudaStream_t s, cudaGraphConditionalNodeType type, unsigned dflt,
                              cudaGraphConditionalHandle *h) {
  if (!graph_conditional_handle(s, dflt, h)) return nullptr;
  return graph_conditional_node(s, type, *h);
}

cudaGraph_t graph_conditional_node(cudaStream_t s, cudaGraphConditionalNodeType type,
                                   cudaGraphConditionalHandle h) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess ||
      cs != cudaStreamCaptureStatusActive)
    return nullptr;
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = type;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, g, deps, nullptr, nd, &p) != cudaSuccess) return nullptr;
  if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) !=
      cudaSuccess)
    return nullptr;
  return p.conditional.phGraph_out[0];
}

void diffusion_solve(const DevMech &m, const DevGrid &g, int i0, double wdt, const double *theta,
                     const double *rhs, double *out, DiffWork &w, int sweeps, double rho_bound,
                     double lin_rtol, DevStats *st, cudaStream_t s) {
  const double reduction = std::max(1e-3 * lin_rtol, 1e-17);
  const FieldMap fm = make_map(m, m.D0_host, m.alpha0, i0, wdt, g.dx);
  const int cs = g.cells;
  double cmax = 0.0;
  for (int k = 0; k < fm.nfs; ++k) cmax = std::max(cmax, fm.cf[k]);
  cudaMemsetAsync(w.rho_bits, 0, sizeof(unsigned long long), s);
  const bool refine = w.refine_rounds > 0 && w.levels <= 1;   // FP32 inner Chebyshev solves
  k_face_coef<<<(cs + 255) / 256, 256, 0, s>>>(g, fm, theta, w.thf, refine ? nullptr : w.invdiag, cmax,
                                               w.rho_bits, w.thf32, w.invdiag32,
                                               refine ? nullptr : w.cdiag);
  if (refine) {
    // mixed precision: FP32 inner Chebyshev solves (reduction 1e-6 each) of the
    // residual of each round's iterate; the first round's residual (of x_0 = b)
    // in FP32 inside its first sweep, the later rounds' in FP64
    const int k32 = std::min(sweeps, chebyshev_sweeps(rho_bound, 1e-6));
    const int R = w.refine_rounds;
    k_cheb_plan<<<1, 32, 0, s>>>(w.rho_bits, k32, 1e-6, w.kdev32, w.omega32, st, R);
    const dim3 gr4((cs + 255) / 256, (fm.nfs + 3) / 4);
    // round r: the residual of x_r, the inner sweeps for e, and (all but the last
    // round) x_{r+1} = x_r + e written by the last planned sweep; the last round's
    // residual pass also stores its reconstruction q in xc, and the finish forms
    // the solution from x_r, q and e
    const double *xcur = rhs;
    double *xr[2] = {w.xa, w.xb};
    for (int round = 0; round < R; ++round) {
      const bool lastr = round == R - 1;
      double *xnext = lastr ? nullptr : xr[round & 1];
      double *q = lastr ? w.xc : nullptr;
      const bool fused = round == 0 && !lastr;
      if (!fused) {
        if (g.dim == 1)
          k_refine_residual<1><<<gr4, 256, 0, s>>>(g, fm, w.thf, rhs, xcur, w.r32, q);
        else if (g.dim == 2)
          k_refine_residual<2><<<gr4, 256, 0, s>>>(g, fm, w.thf, rhs, xcur, w.r32, q);
        else
          k_refine_residual<3><<<gr4, 256, 0, s>>>(g, fm, w.thf, rhs, xcur, w.r32, q);
      }
      for (int it = 0; it < k32; ++it) {
        const float *ek = w.e32[(it + 2) % 3];
        const float *ekm1 = (it >= 2) ? w.e32[(it + 1) % 3] : nullptr;   // e_0 = 0
        if (fused && it == 0) {
          if (g.dim == 1)
            k_cheb32_first<1><<<gr4, 256, 0, s>>>(g, fm, w.thf32, w.invdiag32, rhs, w.r32, w.e32[0],
                                                  w.kdev32, xnext);
          else if (g.dim == 2)
            k_cheb32_first<2><<<gr4, 256, 0, s>>>(g, fm, w.thf32, w.invdiag32, rhs, w.r32, w.e32[0],
                                                  w.kdev32, xnext);
          else
            k_cheb32_first<3><<<gr4, 256, 0, s>>>(g, fm, w.thf32, w.invdiag32, rhs, w.r32, w.e32[0],
                                                  w.kdev32, xnext);
        } else if (g.dim == 1)
          k_cheb32<1><<<gr4, 256, 0, s>>>(g, fm, w.thf32, w.invdiag32, w.r32, ek, ekm1,
                                          w.e32[it % 3], it, w.kdev32, w.omega32, xcur, xnext);
        else if (g.dim == 2)
          k_cheb32<2><<<gr4, 256, 0, s>>>(g, fm, w.thf32, w.invdiag32, w.r32, ek, ekm1,
                                          w.e32[it % 3], it, w.kdev32, w.omega32, xcur, xnext);
        else
          k_cheb32<3><<<gr4, 256, 0, s>>>(g, fm, w.thf32, w.invdiag32, w.r32, ek, ekm1,
                                          w.e32[it % 3], it, w.kdev32, w.omega32, xcur, xnext);
      }
      if (!lastr) xcur = xnext;
    }
    // solution, reconstruction and residual check from x_r, q and the last e
    const int blocks = (cs + 255) / 256;
    const double tol = lin_rtol * 100.0;
    if (g.dim == 1)
      k_finish32<1><<<blocks, 256, 0, s>>>(g, fm, m.N, i0, tol, w.thf32, rhs, w.xc, xcur, w.e32[0],
                                           w.e32[1], w.e32[2], w.kdev32, out, st);
    else if (g.dim == 2)
      k_finish32<2><<<blocks, 256, 0, s>>>(g, fm, m.N, i0, tol, w.thf32, rhs, w.xc, xcur, w.e32[0],
                                           w.e32[1], w.e32[2], w.kdev32, out, st);
    else
      k_finish32<3><<<blocks, 256, 0, s>>>(g, fm, m.N, i0, tol, w.thf32, rhs, w.xc, xcur, w.e32[0],
                                           w.e32[1], w.e32[2], w.kdev32, out, st);
    return;
  }
  if (w.levels > 1) {
    multigrid_solve(g, fm, rhs, w, lin_rtol, st, s);
    launch_finish(g, fm, m.N, i0, lin_rtol * 100.0, w.thf, rhs, w.xa, w.xb, w.xc, nullptr, out, st, s);
    return;
  }
  // sweeps: planned on the device from the measured Gershgorin bound, at most
  // `sweeps` (the a-priori bound with theta at the 6000 K cap)
  (void)rho_bound;
  k_cheb_plan<<<1, 32, 0, s>>>(w.rho_bits, sweeps, reduction, w.kdev, w.omega, st, 1);
  const int tb = (w.cheb_block >= 32 && w.cheb_block <= 1024) ? w.cheb_block : 256;
  // Chebyshev-accelerated Jacobi from x0 = rhs (the operator is I - c L)
  double *bufs[3] = {w.xa, w.xb, w.xc};
  for (int it = 0; it < sweeps; ++it) {
    const double *xk = (it == 0) ? rhs : bufs[(it - 1) % 3];
    const double *xkm1 = (it <= 1) ? rhs : bufs[(it - 2) % 3];
    const dim3 grid((cs + tb - 1) / tb, (fm.nfs + kChebFields - 1) / kChebFields);
    if (g.dim == 1)
      k_cheb<1><<<grid, tb, 0, s>>>(g, fm, w.thf, w.invdiag, w.cdiag, w.bdiag, rhs, xk, xkm1,
                                    bufs[it % 3], it, w.kdev, w.omega);
    else if (g.dim == 2)
      k_cheb<2><<<grid, tb, 0, s>>>(g, fm, w.thf, w.invdiag, w.cdiag, w.bdiag, rhs, xk, xkm1,
                                    bufs[it % 3], it, w.kdev, w.omega);
    else
      k_cheb<3><<<grid, tb, 0, s>>>(g, fm, w.thf, w.invdiag, w.cdiag, w.bdiag, rhs, xk, xkm1,
                                    bufs[it % 3], it, w.kdev, w.omega);
  }
  const int *kdev = w.kdev;
  const double *xfin = w.xa;
  launch_finish(g, fm, m.N, i0, lin_rtol * 100.0, w.thf, rhs, xfin, w.xb, w.xc, kdev, out, st, s);
}

void launch_nu_decide(int F, int cs, int M, NodePtrs now, NodePtrs before, int l, int nu,
                      double eta, double rho, unsigned long long *bits, double *delta, int *cont,
                      int *ran, DevStats *st, const cudaGraphConditionalHandle *h,
                      const int *body_kernels, cudaStream_t s) {
  const int bx = std::max(1, std::min((cs + 255) / 256, 64));
  k_nu_incr<<<dim3(bx, F), 256, 0, s>>>(cs, M, now, before, bits);
  k_nu_decide<<<1, 32, 0, s>>>(F, l, nu, eta, rho, bits, delta, cont, ran, st, h ? *h : 0, h ? 1 : 0,
                               body_kernels);
}

void launch_copy_if_parity(const CopyList &cl, const int *ran, int parity, cudaStream_t s) {
  if (cl.count <= 0) return;
  k_copy_if_parity<<<dim3(64, cl.count), 256, 0, s>>>(cl, ran, parity);
}

}  // namespace misdc
