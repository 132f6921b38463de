// Chemistry kernels: temperature diagnosis, production rates and the per-cell
// reaction Newton solve of step S5 (Sec. 3.3, eq.
// reaction_step_numerical_methodology), one warp per cell.
//
// Layout: every per-cell array is field-major, [field][cs] with a cell stride cs.
#include <math.h>

#include <mutex>

#include "misdc_internal.cuh"

namespace misdc {

namespace {

// 2^(j/32), j = 0..31, rounded to double; written once per device by
// init_exp_table() from an extended-precision evaluation on the host.
__device__ double g_exp2_32[32];

// e^x by Tang's table-driven method (P. T. P. Tang, ACM TOMS 15(2), 1989):
// x = (32 m + j) ln2/32 + r with |r| <= ln2/64, so e^x = 2^m 2^(j/32) e^r. The
// reduction rounds x 32/ln2 to an integer by adding 1.5 2^52 (whose low word is
// then the integer), subtracts it times ln2/32 split into a leading and a trailing
// double (the leading product is exact here); e^r - 1 is the Taylor polynomial of
// degree 6 (truncation below 4e-18 relative for |r| <= ln2/64); 2^m goes into the
// exponent field. Error about 1 ulp, in about twelve FP64 instructions, where the
// general-purpose exp() costs roughly twice that on the FP64 pipe. Arguments
// outside (-700, 700), and NaN, take exp().
__device__ __forceinline__ double exp_tab(double x) {
  if (!(fabs(x) < 700.0)) return exp(x);
  const double shift = 6755399441055744.0;                 // 1.5 * 2^52
  const double t = fma(x, 46.16624130844683, shift);       // x * 32 / ln2, rounded
  const int k = __double2loint(t);
  const double kd = t - shift;
  double r = fma(-kd, 0.02166084939249829, x);             // ln2/32, leading part
  r = fma(-kd, 7.247021293269686e-19, r);                  // ln2/32, trailing part
  double q = fma(r, 1.0 / 720.0, 1.0 / 120.0);
  q = fma(q, r, 1.0 / 24.0);
  q = fma(q, r, 1.0 / 6.0);
  q = fma(q, r, 0.5);
  const double p = fma(q, r * r, r);                        // e^r - 1
  const double tj = g_exp2_32[k & 31];
  const double v = fma(tj, p, tj);
  return __longlong_as_double(__double_as_longlong(v) + ((long long)(k >> 5) << 52));
}

__global__ void k_exp(const double *__restrict__ x, double *__restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = exp_tab(x[i]);
}

// h/RT and g/RT of species i (NASA-7); cp/R separately where it is needed
__device__ __forceinline__ void species_hg(const DevMech &m, int i, double T, double lnT,
                                           double invT, double &hRT, double &gRT) {
  const double *a = m.hcoef + 6 * i;
  hRT = fma(a[5], invT, a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4]))));
  const double *s = m.scoef + 6 * i;
  double sR = fma(s[0], lnT, T * (s[1] + T * (s[2] + T * (s[3] + T * s[4])))) + s[5];
  gRT = hRT - sR;
}

__device__ __forceinline__ double species_cpR(const DevMech &m, int i, double T) {
  const double *c = m.cpcoef + 5 * i;
  return c[0] + T * (c[1] + T * (c[2] + T * (c[3] + T * c[4])));
}

__device__ __forceinline__ void species_thermo(const DevMech &m, int i, double T, double lnT,
                                               double invT, double &hRT, double &gRT,
                                               double &cpR) {
  species_hg(m, i, T, lnT, invT, hRT, gRT);
  cpR = species_cpR(m, i, T);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// Temperature from (Y, h): Newton safeguarded by bisection on [kTlo, kThi].
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mix_h_cp(const DevMech &m, const double *Y, int cs, int c,
                                         double T, double &h, double &cp) {
  double lnT = 0.0, invT = 1.0 / T;
  double hs = 0.0, cps = 0.0;
  for (int i = 0; i < m.N; ++i) {
    double hRT, gRT, cpR;
    const double *a = m.hcoef + 6 * i;
    hRT = fma(a[5], invT, a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4]))));
    const double *cc = m.cpcoef + 5 * i;
    cpR = cc[0] + T * (cc[1] + T * (cc[2] + T * (cc[3] + T * cc[4])));
    double wy = Y[(size_t)i * cs + c] * m.invW[i];
    hs = fma(wy, hRT, hs);
    cps = fma(wy, cpR, cps);
    (void)gRT;
  }
  (void)lnT;
  h = kRu * T * hs;
  cp = kRu * cps;
}

__global__ void k_temperature(DevMech m, int n, int cs, const double *__restrict__ Y,
                              const double *__restrict__ hin, const double *__restrict__ Tg,
                              double *__restrict__ Tout, double *__restrict__ theta,
                              double *__restrict__ hsp, DevStats *st) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double h = hin[c];
  double lo = kTlo, hi = kThi, fl, fh, d;
  double T = (Tg && Tg[c] > lo && Tg[c] < hi) ? Tg[c] : 1000.0;
  // plain Newton from the guess first (h is monotone in T: cp > 0); the bracketed
  // iteration below, with its check that [50, 6000] K holds the root, runs only
  // when Newton leaves the range or does not settle
  bool done = false;
  for (int it = 0; it < 12; ++it) {
    double f, df;
    mix_h_cp(m, Y, cs, c, T, f, df);
    const double Tn = T - (f - h) / df;
    if (!(Tn > lo && Tn < hi)) break;
    const double dT = Tn - T;
    T = Tn;
    if (fabs(dT) <= 1e-14 * T) { done = true; break; }
  }
  if (!done) {
  T = (Tg && Tg[c] > lo && Tg[c] < hi) ? Tg[c] : 1000.0;
  mix_h_cp(m, Y, cs, c, lo, fl, d);
  mix_h_cp(m, Y, cs, c, hi, fh, d);
  if (!(fl - h <= 0.0 && fh - h >= 0.0)) {
    atomicOr(&st->status_bits, kBitTdiag);
    T = NAN;
  } else {
    for (int it = 0; it < 200; ++it) {
      double f, df;
      mix_h_cp(m, Y, cs, c, T, f, df);
      f -= h;
      if (f > 0.0) hi = T; else lo = T;
      double Tn = T - f / df;
      if (!(Tn > lo && Tn < hi)) Tn = 0.5 * (lo + hi);
      double dT = Tn - T;
      T = Tn;
      if (fabs(dT) <= 1e-14 * T) break;
    }
  }
  }
  Tout[c] = T;
  if (theta) theta[c] = pow(T / m.T_ref, m.theta_exp);
  if (hsp) {
    double invT = 1.0 / T;
    for (int i = 0; i < m.N; ++i) {
      const double *a = m.hcoef + 6 * i;
      double hRT = fma(a[5], invT, a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4]))));
      hsp[(size_t)i * cs + c] = kRu * m.invW[i] * T * hRT;
    }
  }
}

__global__ void k_enthalpy(DevMech m, int n, int cs, const double *__restrict__ Y,
                           const double *__restrict__ T, double *__restrict__ h) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double hh, cp;
  mix_h_cp(m, Y, cs, c, T[c], hh, cp);
  h[c] = hh;
}

// ---------------------------------------------------------------------------
// Warp-level chemistry state in shared memory
// ---------------------------------------------------------------------------
struct WarpChem {
  double *c, *g, *hRT, *hm, *cpm;   // [N] concentration, g/RT, h/RT, h (J/kg), cp (J/kg/K)
  double *q, *kf, *kr, *dqdT;       // [R]
};

// thermo of every species at T, then every reaction's rate of progress (and
// what the Jacobian needs); concentrations w.c must be set.
__device__ void eval_chem(const DevMech &m, const WarpChem &w, int lane, double T, bool jac) {
  double lnT = 0.0, invT = 0.0;   // warp-uniform: computed on one lane, broadcast
  if (lane == 0) { lnT = log(T); invT = 1.0 / T; }
  lnT = __shfl_sync(0xffffffffu, lnT, 0);
  invT = __shfl_sync(0xffffffffu, invT, 0);
  for (int i = lane; i < m.N; i += 32) {
    double hRT, gRT, cpR;
    species_thermo(m, i, T, lnT, invT, hRT, gRT, cpR);
    w.g[i] = gRT;
    w.hRT[i] = hRT;
    w.hm[i] = kRu * m.invW[i] * T * hRT;
    w.cpm[i] = kRu * m.invW[i] * cpR;
  }
  __syncwarp();
  for (int r = lane; r < m.R; r += 32) {
    const signed char *fs = m.fwd + kMaxSlots * r, *rs = m.rev + kMaxSlots * r;
    double dg = 0.0, dh = 0.0, Ff = 1.0, Fr = 1.0;
#pragma unroll
    for (int p = 0; p < kMaxSlots; ++p) {
      int sf = fs[p], sr = rs[p];
      if (sf >= 0) { dg -= w.g[sf]; dh -= w.hRT[sf]; Ff *= w.c[sf]; }
      if (sr >= 0) { dg += w.g[sr]; dh += w.hRT[sr]; Fr *= w.c[sr]; }
    }
    const double beta = m.beta[r], TA = m.TA[r], dn = m.dn[r];
    const double lnkf = m.lnA[r] + beta * lnT - TA * invT;
    const double lnKc = -dg + dn * (m.ln_p_over_R - lnT);
    const double kf = exp_tab(lnkf);
    const double kr = exp_tab(lnkf - lnKc);
    w.q[r] = kf * Ff - kr * Fr;
    if (jac) {
      const double dlnkf = (beta + TA * invT) * invT;
      const double dlnKc = (dh - dn) * invT;
      w.kf[r] = kf;
      w.kr[r] = kr;
      w.dqdT[r] = kf * Ff * dlnkf - kr * Fr * (dlnkf - dlnKc);
    }
  }
  __syncwarp();
}

// Production rates with the contraction wdot = diag(W) nu^T q on the FP64 tensor
// cores. A block takes 32 cells at a time: each warp evaluates the reaction
// rates q of 8 cells (lanes over reactions, as above) into a [32][qld] tile in
// shared memory; then each warp takes every 4th species tile and, per nonzero
// (4 reactions x 8 species) tile of [W_i nu_ri], loads the B fragment once and
// issues one m8n8k4 FP64 MMA for each of the four 8-cell row tiles.
constexpr int kMmaCells = 32;

__device__ __forceinline__ void dmma_8x8x4(double &d0, double &d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(128) k_rates_mma(DevMech m, int n, int cs,
                                                   const double *__restrict__ Y,
                                                   const double *__restrict__ T,
                                                   double *__restrict__ FR) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int N = m.N, R = m.R, qld = mma_qld(R), R4 = (R + 3) & ~3;
  double *Q = smem;                                        // [32][qld]
  double *scratch = smem + (size_t)kMmaCells * qld + (size_t)wib * 5 * N;
  WarpChem w;
  w.c = scratch; w.g = scratch + N; w.hRT = scratch + 2 * N; w.hm = scratch + 3 * N;
  w.cpm = scratch + 4 * N;
  w.kf = w.kr = w.dqdT = nullptr;
  const double invrho = 1.0 / m.rho;
  const int row = lane >> 2, col = lane & 3;
  const int groups = (n + kMmaCells - 1) / kMmaCells;
  for (int grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const int c0 = grp * kMmaCells;
    for (int j = wib; j < kMmaCells; j += wpb) {
      const int cell = c0 + j;
      w.q = Q + (size_t)j * qld;
      if (cell < n) {
        for (int i = lane; i < N; i += 32) w.c[i] = m.rho * Y[(size_t)i * cs + cell] * m.invW[i];
        __syncwarp();
        eval_chem(m, w, lane, T[cell], false);
        for (int r = R + lane; r < R4; r += 32) w.q[r] = 0.0;   // reaction padding
      } else {
        for (int r = lane; r < R4; r += 32) w.q[r] = 0.0;       // ragged tail
      }
      __syncwarp();
    }
    __syncthreads();
    for (int jt = wib; jt < m.mma_nt; jt += wpb) {
      double d[4][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}};
      for (int p = m.mma_ptr[jt]; p < m.mma_ptr[jt + 1]; ++p) {
        const double b = __ldg(m.mma_b + (size_t)p * 32 + lane);
        const int k = 4 * m.mma_kb[p] + col;
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) dmma_8x8x4(d[mt][0], d[mt][1], Q[(size_t)(8 * mt + row) * qld + k], b);
      }
      const int sp = 8 * jt + 2 * col;
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const int cell = c0 + 8 * mt + row;
        if (cell < n) {
          if (sp < N) FR[(size_t)sp * cs + cell] = d[mt][0] * invrho;
          if (sp + 1 < N) FR[(size_t)(sp + 1) * cs + cell] = d[mt][1] * invrho;
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Reaction Newton, lane-balanced form: one warp per cell; the iterate, the
// augmented Jacobian and the per-reaction quantities live in shared memory and
// every phase spreads its work over all 32 lanes:
//  * thermo over species, rates and slot derivatives over reactions;
//  * Jacobian and residual assembly from a host-built list of contributions
//    (target entry, source value, weight) sorted by target and cut into 32
//    segments of whole targets, so each lane owns its targets (deterministic,
//    no atomics) and the lanes carry equal work;
//  * partial pivoting by a warp argmax on the integer bit patterns of |J_ik|;
//    elimination of the trailing block spread element-wise over the lanes.
// The temperature row is scaled by 1/(c_p T) (the solution is unchanged).
// ---------------------------------------------------------------------------
struct NW {
  double *J, *src, *xs, *bs, *c, *g, *hRT, *hm, *cpm, *piv, *dx;
  // mixed precision: FP32 factor, FP64 right-hand side and residual
  float *Jf, *zf, *pivf;
  int *sw;
  double *r64, *res, *xg, *zd;
};

// doubles of shared memory one warp needs
__host__ __device__ inline size_t newton_warp_doubles(int N, int R, int ld, bool mixed) {
  const size_t nn = N + 1;
  size_t d = nn * ld + 8 * (size_t)R + 6 * (size_t)N + 4 * nn;
  if (mixed) d += (nn * ld + 1) / 2 + 3 * nn + (3 * nn + 1) / 2 + 1;
  return d;
}

__device__ __forceinline__ NW carve2(double *p, int N, int R, int ld, bool mixed) {
  const int nn = N + 1;
  NW w;
  w.J = p; p += (size_t)nn * ld;
  w.src = p; p += 8 * R;
  w.xs = p; p += nn;
  w.bs = p; p += N;
  w.c = p; p += N;
  w.g = p; p += N;
  w.hRT = p; p += N;
  w.hm = p; p += N;
  w.cpm = p; p += N;
  w.piv = p; p += nn;
  w.dx = p; p += nn;
  w.xg = p; p += nn;
  if (mixed) {
    w.r64 = p; p += nn;
    w.res = p; p += nn;
    w.zd = p; p += nn;
    w.Jf = reinterpret_cast<float *>(p); p += ((size_t)nn * ld + 1) / 2;
    float *f = reinterpret_cast<float *>(p);
    w.zf = f; w.pivf = f + nn;
    w.sw = reinterpret_cast<int *>(f + 2 * nn);
  } else {
    w.r64 = w.res = w.zd = nullptr; w.Jf = w.zf = w.pivf = nullptr; w.sw = nullptr;
  }
  return w;
}


// Kept factors are stored as explicit inverses, so that a chord step is one
// matrix-vector product (nn FMA warp instructions) instead of a forward and a
// back substitution (about 3 nn, each on a shrinking set of lanes).
//
// invert_lu: Z = U^{-1} L^{-1} P in place of the factor in J (L unit lower below
// the diagonal, U on and above it, piv = 1/U_kk, row exchanges sw taken in order
// k = 0..nn-1): the inverse of the factored matrix. Steps: U^{-1} column by
// column; then, from the last column to the first, the columns of U^{-1} L^{-1}
// from those to their right; then the column exchanges in reverse order. T is
// the precision of the factor (an FP32 factor is inverted in FP32: it carries
// no more accuracy than that, and the FP32 pipe is 60x faster). z: nn scratch.
template <class T>
__device__ void invert_lu(T *J, int ld, int nn, int lane, const T *piv, T *z, const int *sw) {
  for (int j = 0; j < nn; ++j) {   // U^{-1}: X[0:j, j] = -X[j][j] X[0:j, 0:j] U[0:j, j]
    const T xjj = piv[j];
    T t0 = 0, t1 = 0;
    if (lane < j)
      for (int k = lane; k < j; ++k) t0 = fma(J[(size_t)lane * ld + k], J[(size_t)k * ld + j], t0);
    if (lane + 32 < j)
      for (int k = lane + 32; k < j; ++k) t1 = fma(J[(size_t)(lane + 32) * ld + k], J[(size_t)k * ld + j], t1);
    __syncwarp();
    if (lane < j) J[(size_t)lane * ld + j] = -xjj * t0;
    if (lane + 32 < j) J[(size_t)(lane + 32) * ld + j] = -xjj * t1;
    if (lane == 0) J[(size_t)j * ld + j] = xjj;
    __syncwarp();
  }
  for (int j = nn - 2; j >= 0; --j) {   // X[:, j] -= X[:, j+1:] L[j+1:, j]
    for (int i = j + 1 + lane; i < nn; i += 32) {
      z[i] = J[(size_t)i * ld + j];
      J[(size_t)i * ld + j] = 0;
    }
    __syncwarp();
    for (int i = lane; i < nn; i += 32) {
      T s = J[(size_t)i * ld + j];
      for (int k = j + 1; k < nn; ++k) s = fma(-J[(size_t)i * ld + k], z[k], s);
      J[(size_t)i * ld + j] = s;
    }
    __syncwarp();
  }
  for (int j = nn - 2; j >= 0; --j) {   // column exchanges, last first
    const int jp = sw[j];
    if (jp != j)
      for (int i = lane; i < nn; i += 32) {
        const T t = J[(size_t)i * ld + j];
        J[(size_t)i * ld + j] = J[(size_t)i * ld + jp];
        J[(size_t)i * ld + jp] = t;
      }
  }
  __syncwarp();
}

// out = Z r with the inverse kept in J; warp-wide
__device__ __forceinline__ void apply_kept(const double *J, int ld, int nn, int lane,
                                           const double *r, double *out) {
  for (int i = lane; i < nn; i += 32) {
    double s = 0.0;
    for (int j = 0; j < nn; ++j) s = fma(J[(size_t)i * ld + j], r[j], s);
    out[i] = s;
  }
  __syncwarp();
}

// Certification of converged guesses, one thread per cell (mixed precision with
// kept factors). A cell whose guess x_p has a kept FP64-built factor, built within
// 1e-4 of x_p, is solved when the step through that factor's inverse Z of the
// residual r = b - Y_p + wdt F_p (and (h* - h_p) times the temperature-row scale),
// formed from the stored reaction term F_p without evaluating any rate, is below
// 0.09 rtol (|dY|, |dT|/T). r is formed in FP64 (a difference of nearly equal
// values), rounded to FP32 and multiplied by the FP32 copy of Z on the FP32 pipe
// (the product only has to be compared with the threshold). A certified cell keeps
// x_p, its species enthalpies and theta; its reaction term is (Y - b)/wdt. Every
// other cell (no usable factor, a learned guess to vet, a step above the
// threshold) is appended to `list` for the warp-per-cell Newton kernel.
__global__ void __launch_bounds__(256) k_certify(DevMech m, int n, int cs, double wdt, double rtol,
                                                 const double *__restrict__ b,
                                                 const double *__restrict__ hstar,
                                                 const double *__restrict__ Yg,
                                                 const double *__restrict__ Tg,
                                                 double *__restrict__ Yout, double *__restrict__ Tout,
                                                 double *__restrict__ FR, double *__restrict__ hsp,
                                                 double *__restrict__ theta, int *__restrict__ iters,
                                                 DevStats *st, const double *__restrict__ sc,
                                                 double s_min, const int *__restrict__ prow,
                                                 const double *__restrict__ FRp,
                                                 const double *__restrict__ hp, ChordStore cst,
                                                 const double *__restrict__ hspp,
                                                 const double *__restrict__ thp,
                                                 int *__restrict__ list, int *__restrict__ list_n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int N = m.N, nn = N + 1;
  bool done = false;
  if (c < n) {
    const int v = cst.valid[c];
    bool ok = (v & 1) != 0 && (v & 4) == 0;   // a kept factor, built in FP64
    if (ok && sc) {   // a learned guess goes to the Newton kernel, which vets it
      const int prw = prow ? prow[c] : c;
      const double s0 = sc[c];
      ok = !(prw >= 0 && s0 > s_min && isfinite(s0));
    }
    const double T = Tg[c];
    if (ok) {   // the factor was built near x_p (without dividing by T); no early
                // exit, so that the loads of all species are in flight together
      double dev = 0.0;
      for (int i = 0; i < N; ++i) {
        const double e = fabs(Yg[(size_t)i * cs + c] - cst.xc[(size_t)i * cs + c]);
        dev = (e <= dev) ? dev : e;   // a NaN deviation propagates (fmax would drop it)
      }
      ok = dev <= 1e-4 && fabs(T - cst.xc[(size_t)N * cs + c]) <= 1e-4 * T;
    }
    if (ok) {
      float r32[kMaxSpecies + 1];
      for (int i = 0; i < N; ++i)
        r32[i] = __double2float_rn(b[(size_t)i * cs + c] - Yg[(size_t)i * cs + c] +
                                   wdt * FRp[(size_t)i * cs + c]);
      r32[N] = __double2float_rn((hstar[c] - hp[c]) * cst.sT[c]);
      // every row (most cells are certified and need them all): the rows' loads
      // are independent of the earlier rows' outcome
      const float thr = (float)(0.09 * rtol), thrT = thr * (float)T;
      bool small = true;
      for (int i = 0; i < nn; ++i) {
        float z = 0.0f;
        for (int j = 0; j < nn; ++j) z = fmaf(cst.z32[((size_t)j * nn + i) * cs + c], r32[j], z);
        small = small && fabsf(z) <= (i < N ? thr : thrT);
      }
      ok = small;
    }
    if (ok) {
      const double invw = (wdt > 0.0) ? 1.0 / wdt : 0.0;
      for (int i = 0; i < N; ++i) {
        const double y = Yg[(size_t)i * cs + c];
        Yout[(size_t)i * cs + c] = y;
        if (FR) FR[(size_t)i * cs + c] = (y - b[(size_t)i * cs + c]) * invw;
        if (hsp) hsp[(size_t)i * cs + c] = hspp[(size_t)i * cs + c];
      }
      Tout[c] = T;
      if (theta) theta[c] = thp[c];
      if (iters) iters[c] = 1;
      done = true;
    } else {
      list[atomicAdd(list_n, 1)] = c;
    }
  }
  // statistics: one atomic per warp
  const unsigned cert = __ballot_sync(0xffffffffu, done);
  if ((threadIdx.x & 31) == 0 && cert) {
    const unsigned long long k = __popc(cert);
    atomicAdd(&st->newton_solves, k);
    atomicAdd(&st->newton_iters, k);
    atomicAdd(&st->certified, k);
    atomicMax(&st->newton_max, 1);
  }
}

// One thread's rates of progress q_r = k_f prod c^nu' - k_r prod c^nu'' of its
// cell, scattered into wd_i += (nu''_ri - nu'_ri) q_r (wd zeroed by the caller).
// Per-thread arrays in shared memory as [species][thread] (B threads): cc the
// concentrations, gg g/RT, wd the sums.
__device__ __forceinline__ void thread_rates(const DevMech &m, double lnT, double invT,
                                             const double *cc, const double *gg, double *wd, int B,
                                             int tid) {
  for (int r = 0; r < m.R; ++r) {
    const signed char *fs = m.fwd + kMaxSlots * r, *rs = m.rev + kMaxSlots * r;
    double dg = 0.0, Ff = 1.0, Fr = 1.0;
#pragma unroll
    for (int q = 0; q < kMaxSlots; ++q) {
      const int sf = fs[q], sr = rs[q];
      if (sf >= 0) { dg -= gg[(size_t)sf * B + tid]; Ff *= cc[(size_t)sf * B + tid]; }
      if (sr >= 0) { dg += gg[(size_t)sr * B + tid]; Fr *= cc[(size_t)sr * B + tid]; }
    }
    const double lnkf = m.lnA[r] + m.beta[r] * lnT - m.TA[r] * invT;
    const double lnKc = -dg + m.dn[r] * (m.ln_p_over_R - lnT);
    const double qr = exp_tab(lnkf) * Ff - exp_tab(lnkf - lnKc) * Fr;
#pragma unroll
    for (int q = 0; q < kMaxSlots; ++q) {
      const int sf = fs[q], sr = rs[q];
      if (sf >= 0) wd[(size_t)sf * B + tid] -= qr;
      if (sr >= 0) wd[(size_t)sr * B + tid] += qr;
    }
  }
}

// Production rates F_R = wdot / rho, one thread per cell (grid-stride): thermo and
// concentrations of the cell, then thread_rates; wdot_i = W_i wd_i.
__global__ void __launch_bounds__(64) k_rates_t(DevMech m, int n, int cs, const double *__restrict__ Y,
                                                const double *__restrict__ T,
                                                double *__restrict__ FR) {
  extern __shared__ double rates_sm[];
  const int B = blockDim.x, tid = threadIdx.x, N = m.N;
  double *cc = rates_sm, *gg = cc + (size_t)N * B, *wd = gg + (size_t)N * B;
  const double invrho = 1.0 / m.rho;
  for (int c = blockIdx.x * B + tid; c < n; c += gridDim.x * B) {
    const double Tc = T[c], lnT = log(Tc), invT = 1.0 / Tc;
    for (int i = 0; i < N; ++i) {
      double hRT, gRT;
      species_hg(m, i, Tc, lnT, invT, hRT, gRT);
      cc[(size_t)i * B + tid] = m.rho * Y[(size_t)i * cs + c] * m.invW[i];
      gg[(size_t)i * B + tid] = gRT;
      wd[(size_t)i * B + tid] = 0.0;
    }
    thread_rates(m, lnT, invT, cc, gg, wd, B, tid);
    for (int i = 0; i < N; ++i) FR[(size_t)i * cs + c] = m.W[i] * wd[(size_t)i * B + tid] * invrho;
  }
}

// Chord iterations, one thread per cell, over the cells certification left
// (in_list; mixed precision with kept factors), persistent blocks taking rounds
// of them. A cell with a usable FP64-built factor near its guess, whose step
// through the kept inverse is at most 1e-4 (certification found it above
// 0.09 rtol), takes that step as iteration 1 (from the stored reaction term, as
// the warp kernel's stored first step does) and then up to max_chord chord
// iterations: the FP64 residual r = b - Y + (wdt/rho) W nu^T q at the iterate,
// every rate of progress evaluated by the cell's own thread, and the step Z r
// through the kept FP64 inverse, as in the warp kernel. (The FP32 copy that
// certification uses is too coarse a chord inverse for stiff cells: its rounding
// misled the stopping test by up to 1e-5 on the 9-species flames.) It stops as
// the warp kernel's chord iteration does, once th = d/d_prev < 0.1 and
// d th / (1 - th) <= rtol. A step above 1e-4, a contraction of less than 10 or a
// non-finite value hands the cell, from its original guess, to the
// warp-per-cell Newton kernel through `list`, as do the cells certification
// cannot take (no usable FP64-built factor, a learned guess to vet). Per-thread
// arrays live in shared memory as [element][thread].
__global__ void __launch_bounds__(64) k_chord(DevMech m, int n, int cs, double wdt, double rtol,
                                              int maxit, int max_chord,
                                              const double *__restrict__ b,
                                              const double *__restrict__ hstar,
                                              const double *__restrict__ Yg,
                                              const double *__restrict__ Tg,
                                              double *__restrict__ Yout, double *__restrict__ Tout,
                                              double *__restrict__ FR, double *__restrict__ hsp,
                                              double *__restrict__ theta, int *__restrict__ iters,
                                              DevStats *st, const double *__restrict__ sc,
                                              double s_min, const int *__restrict__ prow,
                                              const double *__restrict__ FRp,
                                              const double *__restrict__ hp, ChordStore cst,
                                              const double *__restrict__ hspp,
                                              const double *__restrict__ thp,
                                              const int *__restrict__ in_list,
                                              const int *__restrict__ in_n,
                                              int *__restrict__ list, int *__restrict__ list_n) {
  extern __shared__ double chord_sm[];
  const int B = blockDim.x, tid = threadIdx.x;
  const int N = m.N, nn = N + 1;
  const int total = *in_n;
  double *xs = chord_sm;                         // [nn][B] iterate
  double *cc = xs + (size_t)nn * B;              // [nn][B] concentrations, then the residual
  double *gg = cc + (size_t)nn * B;              // [N][B]  g/RT
  double *wd = gg + (size_t)N * B;               // [N][B]  sum_r nu_ri q_r
  double *rr = cc;   // the residual reuses the concentrations, dead after the rates
#define TH(a, k) a[(size_t)(k) * B + tid]
  // rounds of B items per block (uniform per block, so the statistics below see
  // every lane of a warp)
  for (int base = blockIdx.x * B; base < total; base += gridDim.x * B) {
  const int item = base + tid;
  const int c = item < total ? in_list[item] : -1;
  bool conv = false;
  int it = 0;
  if (c >= 0) {
    const int v = cst.valid[c];
    bool ok = (v & 1) != 0 && (v & 4) == 0;   // a kept factor, built in FP64
    if (ok && sc) {   // a learned guess goes to the Newton kernel, which vets it
      const int prw = prow ? prow[c] : c;
      const double s0 = sc[c];
      ok = !(prw >= 0 && s0 > s_min && isfinite(s0));
    }
    const double T0 = Tg[c];
    if (ok) {   // the factor was built near x_p (without dividing by T)
      double dev = 0.0;
      for (int i = 0; i < N; ++i) {
        const double e = fabs(Yg[(size_t)i * cs + c] - cst.xc[(size_t)i * cs + c]);
        dev = (e <= dev) ? dev : e;   // a NaN deviation propagates (fmax would drop it)
      }
      ok = dev <= 1e-4 && fabs(T0 - cst.xc[(size_t)N * cs + c]) <= 1e-4 * T0;
    }
    const double sT = ok ? cst.sT[c] : 0.0;
    const double hst = hstar[c];
    // the step Z r through the kept FP64 inverse (row-major, the cell's own block
    // of the factor store), added to the iterate (a first step that is not taken
    // sends the cell, from its guess, to the warp kernel); d = max(max|dY|, |dT|/T)
    const double *Zc = cst.f + (size_t)c * cst.fs;
    auto step = [&](double T, double &d, bool &fin) {
      double dm = 0.0, dT = 0.0;
      fin = true;
      for (int i = 0; i < nn; ++i) {
        const double *Zi = Zc + (size_t)i * nn;
        double z = 0.0;
        for (int j = 0; j < nn; ++j) z = fma(Zi[j], TH(rr, j), z);
        TH(xs, i) += z;
        fin = fin && isfinite(z);
        if (i < N) dm = fmax(dm, fabs(z));
        else dT = fabs(z);
      }
      d = fmax(dm, dT / T);
    };
    if (ok) {
      for (int i = 0; i < N; ++i) {
        const double y = Yg[(size_t)i * cs + c];
        TH(xs, i) = y;
        TH(rr, i) = b[(size_t)i * cs + c] - y + wdt * FRp[(size_t)i * cs + c];
      }
      TH(xs, N) = T0;
      TH(rr, N) = (hst - hp[c]) * sT;
      double d0;
      bool fin;
      step(T0, d0, fin);
      if (fin && max_chord > 0 && maxit >= 2 && d0 <= 1e-4) {
        // iteration 1: the step from the stored reaction term (taken by step())
        double dprev = d0;
        it = 1;
        const double wr = wdt / m.rho;
        while (it < maxit && it <= max_chord) {
          ++it;
          const double T = TH(xs, N);
          if (!(T > 0.0)) break;
          const double lnT = log(T), invT = 1.0 / T;
          double sh = 0.0;
          for (int i = 0; i < N; ++i) {
            double hRT, gRT;
            species_hg(m, i, T, lnT, invT, hRT, gRT);
            const double y = TH(xs, i);
            TH(cc, i) = m.rho * y * m.invW[i];
            TH(gg, i) = gRT;
            TH(wd, i) = 0.0;
            sh = fma(y, kRu * m.invW[i] * T * hRT, sh);
          }
          thread_rates(m, lnT, invT, cc, gg, wd, B, tid);
          for (int i = 0; i < N; ++i)
            TH(rr, i) = fma(wr, m.W[i] * TH(wd, i), b[(size_t)i * cs + c] - TH(xs, i));
          TH(rr, N) = -(sh - hst) * sT;
          double d;
          step(T, d, fin);
          if (!fin) break;
          if (d > 1e-4 || !(d < 0.1 * dprev)) break;   // not contracting: a new factor is due
          if (d * d <= rtol * (dprev - d)) { conv = true; break; }
          dprev = d;
        }
      }
    }
    if (conv) {
      // species enthalpies and theta at the solution; reaction term (Y - b)/wdt
      const double invw = (wdt > 0.0) ? 1.0 / wdt : 0.0;
      const double T = TH(xs, N), lnT = log(T), invT = 1.0 / T;
      for (int i = 0; i < N; ++i) {
        double hRT, gRT;
        species_hg(m, i, T, lnT, invT, hRT, gRT);
        const double y = TH(xs, i);
        Yout[(size_t)i * cs + c] = y;
        if (FR) FR[(size_t)i * cs + c] = (y - b[(size_t)i * cs + c]) * invw;
        if (hsp) hsp[(size_t)i * cs + c] = kRu * m.invW[i] * T * hRT;
      }
      Tout[c] = T;
      if (theta) theta[c] = exp_tab(m.theta_exp * (lnT - m.ln_Tref));
      if (iters) iters[c] = it;
    } else {
      list[atomicAdd(list_n, 1)] = c;
    }
  }
  // statistics: one atomic per warp and counter
  const unsigned vb = __ballot_sync(0xffffffffu, conv);
  int itv = conv ? it : 0;
  unsigned mx = conv ? (unsigned)it : 0u;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    itv += __shfl_xor_sync(0xffffffffu, itv, o);
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0 && vb) {
    const unsigned long long kv = __popc(vb);
    atomicAdd(&st->newton_solves, kv);
    atomicAdd(&st->newton_iters, (unsigned long long)itv);
    atomicAdd(&st->stored_steps, kv);
    atomicAdd(&st->chord_cells, kv);
    atomicMax(&st->newton_max, (int)mx);
  }
  }   // rounds
#undef TH
}

size_t chord_smem_bytes(int N, int threads) {
  const size_t nn = N + 1;
  return (size_t)threads * (2 * nn + 2 * (size_t)N) * sizeof(double);
}

// The reaction Newton of a run of work items of one solve (one warp per cell);
// `first` is the warp's first item, next(item) its next one (>= items ends the
// run). wsm: the warp's shared-memory scratch. Per-warp counters go to A.st at the
// end of the run.
template <bool MIXED, class Next>
__device__ __forceinline__ void newton_items(const NewtonArgs &A, double *wsm, int first, int items,
                                             Next next_item) {
  const DevMech &m = A.m;
  const int cs = A.cs, maxit = A.maxit, ld = A.ld, ldp = A.ldp;
  const double wdt = A.wdt, rtol = A.rtol, s_min = A.s_min;
  const double *__restrict__ b = A.b;
  const double *__restrict__ hstar = A.hstar;
  const double *Yg = A.Yg, *Tg = A.Tg;
  double *Yout = A.Yout, *Tout = A.Tout;
  double *__restrict__ FR = A.FR;
  double *__restrict__ hsp = A.hsp;
  double *__restrict__ theta = A.theta;
  int *__restrict__ iters = A.iters;
  DevStats *st = A.st;
  const float *__restrict__ pred = A.pred;
  const double *__restrict__ sc = A.sc;
  const double *__restrict__ FRp = A.FRp;
  const double *__restrict__ hp = A.hp;
  const ChordStore &cst = A.cst;
  const int *__restrict__ prow = A.prow;
  const double *__restrict__ hspp = A.hspp;
  const double *__restrict__ thp = A.thp;
  const int *__restrict__ list = A.list;
  const int lane = threadIdx.x & 31;
  const int N = m.N, R = m.R, nn = N + 1, na = nn + 1;   // na: columns of the augmented matrix
  NW w = carve2(wsm, N, R, ld, MIXED);
  double *J = w.J;
  const int seg0 = m.jc_seg[lane], seg1 = m.jc_seg[lane + 1];
  // per-launch constants (an FP64 division is a long instruction sequence on this
  // part: formed once, not per cell)
  const double invw = (wdt > 0.0) ? 1.0 / wdt : 0.0;
  const double wr = wdt / m.rho;
  unsigned long long my_solves = 0, my_iters = 0, my_fail = 0, my_sg = 0, my_rej = 0, my_fb = 0,
                     my_jac = 0, my_lu64 = 0, my_cert = 0, my_stored = 0, my_floor = 0;
  int my_max = 0;
  unsigned bits = 0;

  // an item is a cell, or with `list` the list's entry (the cells that the
  // certification kernel left)
  for (int item = first; item < items; item = next_item(item)) {
    const int cell = list ? list[item] : item;
    for (int i = lane; i < N; i += 32) {
      w.xs[i] = Yg[(size_t)i * cs + cell];
      w.bs[i] = b[(size_t)i * cs + cell];
    }
    if (lane == 0) w.xs[N] = Tg[cell];
    const double hst = hstar[cell];
    // learned guess: x0 = x_p + s p, judged below by its residual against the
    // residual at x_p (whose scaled max-norm is s); x_p is kept in dx until then
    bool vet = false;
    double s0 = 0.0;
    int prw = cell;
    if (pred) {
      s0 = sc[cell];
      if (prow) prw = prow[cell];
      vet = prw >= 0 && s0 > s_min && isfinite(s0);
    }
    __syncwarp();
    if (MIXED && vet && cst.valid && (cst.valid[cell] & 1)) {
      // a cell with a kept factor built within 1e-4 of x_p iterates from x_p on that
      // factor without a new Jacobian; a guess elsewhere would cost one, so the
      // learned guess is kept for the cells that need a new Jacobian anyway
      const double *xf = cst.f + (size_t)cell * cst.fs + nn * nn + 2 * nn + 2;
      bool near = true;
      for (int i = lane; i < nn; i += 32)
        near = near && fabs(w.xs[i] - xf[i]) <= ((i < N) ? 1e-4 : 1e-4 * w.xs[i]);
      if (__all_sync(0xffffffffu, near)) vet = false;
    }
    if (vet) {
      const float *pc = pred + (size_t)prw * ldp;
      for (int i = lane; i < nn; i += 32) {
        const double xp = w.xs[i];
        w.dx[i] = xp;
        // the output in the range of the training targets
        const double f = s0 * fmin(fmax((double)pc[i], -8.0), 8.0);
        w.xs[i] = (i < N) ? xp + f : xp * (1.0 + fmin(fmax(f, -0.5), 0.5));
      }
      __syncwarp();
    }
    // MIXED: a row-equilibrated FP32 factor of the Jacobian, reused across
    // iterations and across calls (the node's previous solve) while the chord
    // iteration contracts; `have` says the shared-memory factor is usable
    bool have = false, fresh = false, from_store = false, fresh_exact = false, no32 = false;
    bool fac32 = false;   // the factor at hand was built in FP32 (its first step may mislead)
    bool exact = false;   // retry: plain FP64 Newton, no factor reuse
    double sTf = 0.0;
    if (MIXED && cst.valid) no32 = (cst.valid[cell] & 2) != 0;   // FP32 factors failed this cell
    bool stored = false;   // a kept factor of this cell's node, built near its guess
    const double *src = nullptr;
    if (MIXED && cst.valid && (cst.valid[cell] & 1)) {
      // a stored factor is used only while the cell stays within 1e-4 (Y, and T
      // relative) of the state it was built at: a stale factor of a stiffer
      // Jacobian would shrink the chord step and fake convergence
      src = cst.f + (size_t)cell * cst.fs;
      const double *xf = src + nn * nn + 2 * nn + 2;
      bool near = true;   // compared without dividing by T
      for (int i = lane; i < nn; i += 32) {
        const double xi = w.xs[i];
        near = near && fabs(xi - xf[i]) <= ((i < N) ? 1e-4 : 1e-4 * xi);
      }
      if (__all_sync(0xffffffffu, near)) {
        stored = true;
        sTf = src[nn * nn + 2 * nn];
        fac32 = src[nn * nn + 2 * nn + 1] != 0.0;
      }
    }
    // copy the kept FP64 inverse into shared memory (chord steps use it)
    auto load_stored = [&]() {
      for (int e = lane; e < nn * nn; e += 32) {
        const int i = e / nn, j = e - i * nn;
        J[(size_t)i * ld + j] = src[e];
      }
      for (int i = lane; i < nn; i += 32) {
        w.piv[i] = src[nn * nn + i];
        w.res[i] = src[nn * nn + nn + i];
        w.sw[i] = cst.sw[(size_t)cell * cst.swld + i];
      }
      __syncwarp();
      have = true;
      from_store = true;
    };
    const bool certify = MIXED && stored && !fac32 && !vet && FRp && hspp;
    if (MIXED && stored && !certify) load_stored();
    {   // restart point: the plain guess x_p
      for (int i = lane; i < nn; i += 32) w.xg[i] = vet ? w.dx[i] : w.xs[i];
      __syncwarp();
    }
    // the solve started from an accepted learned guess: its root must lie near the
    // plain guess (within 100 times the scale s of the residual there), otherwise
    // the solve is repeated from x_p, whose root is the one the plain method finds
    bool guessed = false;
    int it0 = 1;              // first iteration of the loop below
    double dprev0 = INFINITY;  // size of the step taken before it (none)
    if (certify) {
      // A chord step certified without evaluating any rate: the residual of the
      // guess follows from its stored reaction term, r = b - Y_p + wdt F_p (and
      // h* - h_p), and the kept factor gives the step. A guess whose step is
      // below rtol / 10 is the solution: the cell keeps x_p, its species
      // enthalpies and theta, and only its reaction term (Y - b)/wdt is new.
      // The residual is formed in FP64 (it is a difference of nearly equal
      // values); the step only has to be compared with rtol / 10, so it is the
      // product of the FP32 copy of the kept inverse with the residual rounded to
      // FP32 (relative error ~1e-6, on the FP32 pipe), tested against 0.09 rtol.
      for (int i = lane; i < nn; i += 32) {
        const double r = (i < N) ? w.bs[i] - w.xs[i] + wdt * FRp[(size_t)i * cs + cell]
                                 : (hst - hp[cell]) * sTf;
        w.r64[i] = r;
        w.zf[i] = __double2float_rn(r);
      }
      __syncwarp();
      bool tiny = false;
      if (cst.z32 && !list) {   // (with a list the certification kernel has tested it)
        float z0 = 0.0f, z1 = 0.0f;
        for (int j = 0; j < nn; ++j) {
          const float rj = w.zf[j];
          if (lane < nn) z0 = fmaf(cst.z32[((size_t)j * nn + lane) * cs + cell], rj, z0);
          if (lane + 32 < nn) z1 = fmaf(cst.z32[((size_t)j * nn + lane + 32) * cs + cell], rj, z1);
        }
        const float thr = (float)(0.09 * rtol), thrT = thr * (float)w.xs[N];
        tiny = true;   // max(max|dY|, |dT|/T) <= 0.09 rtol, without dividing by T
        if (lane < nn) tiny = fabsf(z0) <= ((lane < N) ? thr : thrT);
        if (lane + 32 < nn) tiny = tiny && fabsf(z1) <= ((lane + 32 < N) ? thr : thrT);
      }
      if (__all_sync(0xffffffffu, tiny)) {
        for (int i = lane; i < N; i += 32) {
          const double y = w.xs[i];
          Yout[(size_t)i * cs + cell] = y;
          if (FR) FR[(size_t)i * cs + cell] = (y - w.bs[i]) * invw;
          if (hsp) hsp[(size_t)i * cs + cell] = hspp[(size_t)i * cs + cell];
        }
        if (lane == 0) {
          Tout[cell] = w.xs[N];
          if (theta) theta[cell] = thp[cell];
          if (iters) iters[cell] = 1;
        }
        __syncwarp();
        ++my_solves;
        ++my_iters;
        ++my_cert;
        my_max = max(my_max, 1);
        continue;
      }
      // Not certified, but a step of at most 1e-4 is the chord step the loop's
      // first iteration would take from x_p (there with the rates evaluated afresh
      // at x_p instead of the stored reaction term, which agree to the previous
      // solve's tolerance). Taken here (with the FP64 inverse), it is iteration 1
      // and costs no rate evaluation; fresh residuals from x_p + step on decide
      // convergence.
      load_stored();
      apply_kept(J, ld, nn, lane, w.r64, w.zd);
      bool fin = true;
      double dm = 0.0;
      for (int i = lane; i < nn; i += 32) {
        fin = fin && isfinite(w.zd[i]);
        if (i < N) dm = fmax(dm, fabs(w.zd[i]));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dm = fmax(dm, __shfl_xor_sync(0xffffffffu, dm, o));
      fin = __all_sync(0xffffffffu, fin);
      double d0 = 0.0;
      if (lane == 0) d0 = fmax(dm, fabs(w.zd[N]) / w.xs[N]);
      d0 = __shfl_sync(0xffffffffu, d0, 0);
      if (fin && d0 <= 1e-4 && maxit >= 2) {
        for (int i = lane; i < nn; i += 32) w.xs[i] += w.zd[i];
        __syncwarp();
        it0 = 2;
        dprev0 = d0;
        ++my_stored;
      }
    }
    double T = w.xs[N];
    double dprev = dprev0;
    int it, code = 0;
    // attempts: the solve itself; after a failure in mixed precision, plain FP64
    // Newton from x_p; and, before that, after a failed solve from an accepted
    // learned guess, the iteration the plain guess alone would have run (mixed:
    // from x_p with a fresh factor), so that a guess never leaves a cell worse
    // off than no guess
    int attempts = MIXED ? 2 : 1;
    for (int attempt = 0; attempt < attempts; ++attempt) {
    if (attempt >= 1) {
      if (code == 0) break;
      for (int i = lane; i < nn; i += 32) w.xs[i] = w.xg[i];
      __syncwarp();
      T = w.xs[N];
      code = 0;
      dprev = INFINITY;
      it0 = 1;
      have = fresh = from_store = fresh_exact = false;
      vet = false;
      if (!(MIXED && attempt == 1 && attempts == 3)) {
        exact = no32 = true;
        ++my_fb;
      }
    }
    for (it = it0; it <= maxit; ++it) {
      const bool jac = !MIXED || !have || exact;   // this iteration assembles the Jacobian
      // ---- thermo and concentrations (species over lanes). FP64 work is paid per
      // active lane on this part, so warp-uniform scalars are computed by lane 0
      // and broadcast.
      double lnT = 0.0, invT = 0.0;
      if (lane == 0) { lnT = log(T); invT = 1.0 / T; }
      lnT = __shfl_sync(0xffffffffu, lnT, 0);
      invT = __shfl_sync(0xffffffffu, invT, 0);
      // the mixture cp only scales the temperature row of a new Jacobian: chord
      // iterations (residual only, with the scale their factor was built with)
      // skip it
      double sh = 0.0, scp = 0.0;
      for (int i = lane; i < N; i += 32) {
        double hRT, gRT;
        species_hg(m, i, T, lnT, invT, hRT, gRT);
        const double y = w.xs[i];
        w.c[i] = m.rho * y * m.invW[i];
        w.g[i] = gRT;
        w.hRT[i] = hRT;
        const double hm = kRu * m.invW[i] * T * hRT;
        w.hm[i] = hm;
        sh = fma(y, hm, sh);
        if (jac) scp = fma(y, kRu * m.invW[i] * species_cpR(m, i, T), scp);
      }
      sh = warp_sum(sh);
      if (jac) scp = warp_sum(scp);
      __syncwarp();
      // ---- rates of progress, dq/dT and slot derivatives (reactions over lanes)
      for (int r = lane; r < R; r += 32) {
        const signed char *fs = m.fwd + kMaxSlots * r, *rs = m.rev + kMaxSlots * r;
        double cf[kMaxSlots], cr[kMaxSlots];
        double dg = 0.0, dh = 0.0;
#pragma unroll
        for (int p = 0; p < kMaxSlots; ++p) {
          const int sf = fs[p], sr = rs[p];
          cf[p] = 1.0;
          cr[p] = 1.0;
          if (sf >= 0) { dg -= w.g[sf]; cf[p] = w.c[sf]; }
          if (sr >= 0) { dg += w.g[sr]; cr[p] = w.c[sr]; }
          if (jac) {   // the reaction enthalpy only enters the Jacobian (dq/dT)
            if (sf >= 0) dh -= w.hRT[sf];
            if (sr >= 0) dh += w.hRT[sr];
          }
        }
        const double beta = m.beta[r], TA = m.TA[r], dn = m.dn[r];
        const double lnkf = m.lnA[r] + beta * lnT - TA * invT;
        const double lnKc = -dg + dn * (m.ln_p_over_R - lnT);
        const double kf = exp_tab(lnkf);
        const double kr = exp_tab(lnkf - lnKc);
        const double Ff = cf[0] * cf[1] * cf[2], Fr = cr[0] * cr[1] * cr[2];
        w.src[r] = kf * Ff - kr * Fr;
        if (jac) {
          const double dlnkf = (beta + TA * invT) * invT;
          const double dlnKc = (dh - dn) * invT;
          w.src[R + r] = kf * Ff * dlnkf - kr * Fr * (dlnkf - dlnKc);
          double *sd = w.src + 2 * R + 6 * r;
          sd[0] = kf * (cf[1] * cf[2]);
          sd[1] = kf * (cf[0] * cf[2]);
          sd[2] = kf * (cf[0] * cf[1]);
          sd[3] = -kr * (cr[1] * cr[2]);
          sd[4] = -kr * (cr[0] * cr[2]);
          sd[5] = -kr * (cr[0] * cr[1]);
        }
      }
      double sT = 0.0;
      if (jac) {
        if (lane == 0) sT = invT / scp;
        sT = __shfl_sync(0xffffffffu, sT, 0);
      }
      if (!jac) {
        // ---- chord iteration: FP64 residual only, wdot_i = sum_r W_i nu_ri q_r;
        // the temperature row keeps the scaling its stored factor was built with
        __syncwarp();
        for (int i = lane; i < N; i += 32) {
          double wd = 0.0;
          for (int p = m.sp_ptr[i]; p < m.sp_ptr[i + 1]; ++p) wd = fma(m.sp_coef[p], w.src[m.sp_rx[p]], wd);
          w.r64[i] = fma(wr, wd, w.bs[i] - w.xs[i]);
        }
        if (lane == 0) w.r64[N] = -(sh - hst) * sTf;
        __syncwarp();
      } else {
      ++my_jac;
      // ---- augmented matrix: identity species rows with b - Y, scaled T row
      for (int i = 0; i < N; ++i)
        for (int j = lane; j < na; j += 32)
          J[(size_t)i * ld + j] = (j == i) ? 1.0 : (j == nn ? w.bs[i] - w.xs[i] : 0.0);
      for (int j = lane; j < N; j += 32) J[(size_t)N * ld + j] = w.hm[j] * sT;
      if (lane == 0) {
        J[(size_t)N * ld + N] = scp * sT;
        J[(size_t)N * ld + nn] = -(sh - hst) * sT;
      }
      __syncwarp();
      // ---- Jacobian and residual contributions: J[t] -= wdt * sum w * src
      {
        int cur = -1;
        double acc = 0.0;
        for (int p = seg0; p < seg1; ++p) {
          const int pk = m.jc_pack[p];
          const int t = pk >> 16;
          if (t != cur) {
            if (cur >= 0) J[cur] = fma(-wdt, acc, J[cur]);
            cur = t;
            acc = 0.0;
          }
          acc = fma(m.jc_w[p], w.src[pk & 0xffff], acc);
        }
        if (cur >= 0) J[cur] = fma(-wdt, acc, J[cur]);
      }
      __syncwarp();
      if (MIXED) {
        // rows are equilibrated (scaled by 1/max|J_ij|) before rounding to FP32, which
        // keeps stiff rows (entries up to ~1e30) in range; the scaling does not change
        // the solution
        for (int i = lane; i < nn; i += 32) {
          double amax = 0.0;
          const double *Ji = J + (size_t)i * ld;
          for (int j = 0; j < nn; ++j) amax = fmax(amax, fabs(Ji[j]));
          w.res[i] = (amax > 0.0) ? 1.0 / amax : 1.0;
          w.r64[i] = Ji[nn];
        }
        __syncwarp();
      }
      }   // jac
      if (vet) {
        // Accept the learned guess only if the residual drops, measured in the
        // Jacobi-scaled max-norm max_i |r_i / J_ii| (species rows; the temperature
        // row as the relative temperature change) with the Jacobian at the guess
        // (a diagonal stand-in for the natural norm |J^{-1} r| of Newton's method,
        // which a plain residual norm would overweight along stiff directions;
        // MIXED: the row scales of its factor). The residual at x_p comes from the
        // stored reaction term of x_p. (A comparison of the two steps through the
        // factor at hand is no test when that factor was just built at a poor
        // guess: it accepted guesses that led to other roots.)
        vet = false;
        double rm = 0.0, rp = 0.0;
        for (int i = lane; i < nn; i += 32) {
          // the temperature row is already in units of dT/T; MIXED scales the
          // species rows by 1/max_j |J_ij| (the equilibration of its factor)
          double dinv, ri;
          if (MIXED) {
            dinv = (i < N) ? w.res[i] : 1.0;
            ri = w.r64[i];
          } else {
            dinv = (i < N) ? 1.0 / fabs(J[(size_t)i * ld + i]) : 1.0;
            ri = J[(size_t)i * ld + nn];
          }
          rm = fmax(rm, fabs(ri) * dinv);
          const double r0 = (i < N) ? w.bs[i] - w.dx[i] + wdt * FRp[(size_t)i * cs + cell]
                                    : (hst - hp[cell]) * (jac ? sT : sTf);
          rp = fmax(rp, fabs(r0) * dinv);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          rm = fmax(rm, __shfl_xor_sync(0xffffffffu, rm, o));
          rp = fmax(rp, __shfl_xor_sync(0xffffffffu, rp, o));
        }
        if (!(rm < rp)) {
          for (int i = lane; i < nn; i += 32) w.xs[i] = w.dx[i];
          __syncwarp();
          T = w.xs[N];
          ++my_rej;
          --it;   // evaluate again at x_p; the rejected evaluation is not an iteration
          continue;
        }
        ++my_sg;
        guessed = true;
        attempts = MIXED ? 3 : 2;
      }
      bool singular = false, fallback = false;
      if (MIXED) {
        // ---- mixed precision: chord (simplified Newton) steps driven by the FP64
        // residual, with a factor of a recent Jacobian kept in J (L below the
        // diagonal, U above, piv = 1/U_kk, row scales res, pivot rows sw). A new
        // factor is an FP32 LU of the row-equilibrated FP64 Jacobian where that is
        // well enough conditioned, else an FP64 LU (below, with fallback set).
        float *Jf = w.Jf;
        fresh = false;
        if (jac && no32) fallback = true;
        if (jac && !no32) {
          for (int i = 0; i < nn; ++i) {
            const double si = w.res[i];
            for (int j = lane; j < nn; j += 32)
              Jf[(size_t)i * ld + j] = __double2float_rn(J[(size_t)i * ld + j] * si);
          }
          __syncwarp();
          for (int k = 0; k < nn; ++k) {
            unsigned best = 0u;
            int bi = nn;
            for (int i = k + lane; i < nn; i += 32) {
              const unsigned v = (unsigned)__float_as_int(Jf[(size_t)i * ld + k]) & 0x7fffffffu;
              if (v > best) { best = v; bi = i; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              const unsigned ob = __shfl_xor_sync(0xffffffffu, best, o);
              const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
              if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (best == 0u || best >= 0x7f800000u) { fallback = true; break; }
            if (lane == 0) w.sw[k] = bi;
            if (bi != k) {
              for (int j = lane; j < nn; j += 32) {
                const float t = Jf[(size_t)k * ld + j];
                Jf[(size_t)k * ld + j] = Jf[(size_t)bi * ld + j];
                Jf[(size_t)bi * ld + j] = t;
              }
              __syncwarp();
            }
            const float pinv = 1.0f / Jf[(size_t)k * ld + k];
            if (lane == 0) w.pivf[k] = pinv;
            for (int i = k + 1 + lane; i < nn; i += 32) Jf[(size_t)i * ld + k] *= pinv;
            __syncwarp();
            const int rows = nn - 1 - k, cols = nn - 1 - k;
            const int total = rows * cols;
            if (total > 0) {
              int i = lane / cols, j = lane - i * cols;
              const int qs = 32 / cols, rsd = 32 - qs * cols;
              for (int e = lane; e < total; e += 32) {
                const size_t ri = (size_t)(k + 1 + i) * ld;
                Jf[ri + k + 1 + j] = fmaf(-Jf[ri + k], Jf[(size_t)k * ld + k + 1 + j], Jf[ri + k + 1 + j]);
                i += qs;
                j += rsd;
                if (j >= cols) { j -= cols; ++i; }
              }
            }
            __syncwarp();
          }
          if (!fallback) {
            // FP32 is only trusted where it can contract: with rows equilibrated,
            // the spread of the pivots max|U_kk| / min|U_kk| stands in for the
            // condition number; above 1e5 (eps32 x cond ~ 1e-2) the cell goes FP64
            float pmin = INFINITY, pmax = 0.0f;
            for (int k = lane; k < nn; k += 32) {
              const float a = fabsf(w.pivf[k]);   // 1 / |U_kk|
              pmin = fminf(pmin, a);
              pmax = fmaxf(pmax, a);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              pmin = fminf(pmin, __shfl_xor_sync(0xffffffffu, pmin, o));
              pmax = fmaxf(pmax, __shfl_xor_sync(0xffffffffu, pmax, o));
            }
            if (!(pmax <= 1e5f * pmin)) fallback = true;
          }
          if (fallback) {
            no32 = true;
          } else {
            // the FP32 factor, inverted in FP32 and widened with the row scales D
            // applied (Z = (D J)^{-1} D, the inverse of the unscaled Jacobian)
            invert_lu<float>(Jf, ld, nn, lane, w.pivf, w.zf, w.sw);
            for (int e = lane; e < nn * nn; e += 32) {
              const int i = e / nn, j = e - i * nn;
              J[(size_t)i * ld + j] = (double)Jf[(size_t)i * ld + j] * w.res[j];
            }
            for (int k = lane; k < nn; k += 32) w.piv[k] = (double)w.pivf[k];
            __syncwarp();
            have = fresh = true;
            fresh_exact = false;
            from_store = false;
            fac32 = true;
            sTf = sT;
          }
        }
        if (!fallback) apply_kept(J, ld, nn, lane, w.r64, w.dx);
      }
      if (!MIXED || fallback) {
        ++my_lu64;
        // ---- FP64 LU with partial pivoting
        for (int k = 0; k < nn; ++k) {
          unsigned long long best = 0ull;
          int bi = nn;
          for (int i = k + lane; i < nn; i += 32) {
            const unsigned long long v =
                (unsigned long long)__double_as_longlong(J[(size_t)i * ld + k]) & 0x7fffffffffffffffull;
            if (v > best) { best = v; bi = i; }
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
          }
          if (best == 0ull || best >= 0x7ff0000000000000ull) { singular = true; break; }
          if (MIXED && lane == 0) w.sw[k] = bi;
          if (bi != k) {
            for (int j = lane; j < na; j += 32) {
              const double t = J[(size_t)k * ld + j];
              J[(size_t)k * ld + j] = J[(size_t)bi * ld + j];
              J[(size_t)bi * ld + j] = t;
            }
            __syncwarp();
          }
          double pinv = 0.0;
          if (lane == 0) { pinv = 1.0 / J[(size_t)k * ld + k]; w.piv[k] = pinv; }
          pinv = __shfl_sync(0xffffffffu, pinv, 0);
          for (int i = k + 1 + lane; i < nn; i += 32) J[(size_t)i * ld + k] *= pinv;
          __syncwarp();
          const int rows = nn - 1 - k, cols = na - 1 - k;   // trailing block (k, nn) x (k, na)
          const int total = rows * cols;
          if (total > 0) {
            int i = lane / cols, j = lane - i * cols;
            const int qs = 32 / cols, rsd = 32 - qs * cols;
            for (int e = lane; e < total; e += 32) {
              const size_t ri = (size_t)(k + 1 + i) * ld;
              J[ri + k + 1 + j] = fma(-J[ri + k], J[(size_t)k * ld + k + 1 + j], J[ri + k + 1 + j]);
              i += qs;
              j += rsd;
              if (j >= cols) { j -= cols; ++i; }
            }
          }
          __syncwarp();
        }
        if (singular) { code = -2; break; }
        for (int k = nn - 1; k >= 0; --k) {
          double xk = 0.0;
          if (lane == 0) { xk = J[(size_t)k * ld + nn] * w.piv[k]; w.dx[k] = xk; }
          xk = __shfl_sync(0xffffffffu, xk, 0);
          for (int i = lane; i < k; i += 32)
            J[(size_t)i * ld + nn] = fma(-J[(size_t)i * ld + k], xk, J[(size_t)i * ld + nn]);
          __syncwarp();
        }
        if (MIXED) {   // an unscaled FP64 factor of the current Jacobian, kept as its inverse
          for (int i = lane; i < nn; i += 32) w.res[i] = 1.0;
          __syncwarp();
          invert_lu<double>(J, ld, nn, lane, w.piv, w.zd, w.sw);
          have = fresh = fresh_exact = true;
          from_store = false;
          fac32 = false;
          sTf = sT;
        }
      }
      if (MIXED && fresh && cst.f && !exact) {   // keep the new factor for this node's next solve
        double *dst = cst.f + (size_t)cell * cst.fs;
        for (int e = lane; e < nn * nn; e += 32) {
          const int i = e / nn, j = e - i * nn;
          const double v = J[(size_t)i * ld + j];
          dst[e] = v;
          if (cst.z32) cst.z32[((size_t)j * nn + i) * cs + cell] = __double2float_rn(v);
        }
        for (int i = lane; i < nn; i += 32) {
          dst[nn * nn + i] = w.piv[i];
          dst[nn * nn + nn + i] = w.res[i];
          dst[nn * nn + 2 * nn + 2 + i] = w.xs[i];
          cst.sw[(size_t)cell * cst.swld + i] = (unsigned char)w.sw[i];
          if (cst.xc) cst.xc[(size_t)i * cs + cell] = w.xs[i];
        }
        if (lane == 0) {
          dst[nn * nn + 2 * nn] = sT;
          dst[nn * nn + 2 * nn + 1] = fac32 ? 1.0 : 0.0;
          if (cst.sT) cst.sT[cell] = sT;
        }
      }
      // ---- update and convergence on d = max(max|dY|, |dT|/T)
      if (MIXED && exact) {
        // the restart of a failed mixed solve limits its steps to |dT| <= T/2 and
        // |dY_i| <= 1/2 (plain Newton from the previous iterate can overshoot at
        // steep fronts); converged steps are far inside the limits
        double big = 0.0;
        for (int i = lane; i < nn; i += 32)
          big = fmax(big, (i < N) ? 2.0 * fabs(w.dx[i]) : 2.0 * fabs(w.dx[i]) / w.xs[N]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) big = fmax(big, __shfl_xor_sync(0xffffffffu, big, o));
        if (big > 1.0) {
          const double lam = 1.0 / big;
          for (int i = lane; i < nn; i += 32) w.dx[i] *= lam;
          __syncwarp();
        }
      }
      double dmax = 0.0;
      bool fin = true;
      for (int i = lane; i < nn; i += 32) {
        const double v = w.xs[i] + w.dx[i];
        w.xs[i] = v;
        if (!isfinite(v)) fin = false;
        if (i < N) dmax = fmax(dmax, fabs(w.dx[i]));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      fin = __all_sync(0xffffffffu, fin);
      __syncwarp();
      T = w.xs[N];
      if (!fin || !(T > 0.0)) { code = -3; break; }
      // the temperature step relative to T before the step (1/T is at hand; the two
      // differ by the factor 1 + dT/T, which is 1 to the stopping tolerance)
      double d = 0.0;
      if (lane == 0) d = fmax(dmax, fabs(w.dx[N]) * invT);
      d = __shfl_sync(0xffffffffu, d, 0);
      if (!isfinite(d)) { code = -3; break; }
      if (!MIXED || exact || (fresh && fresh_exact)) {
        // exact Newton step: stop on the step size, or at the round-off floor of
        // very stiff cells (the step no longer halves below 1e-8)
        if (d <= rtol) break;
        if (d <= 1e-8 && d >= 0.5 * dprev) {
          ++my_floor;
          break;
        }
      } else if (fresh) {
        // a step with a new FP32 factor is judged only by the chord steps after it
      } else {
        // chord steps converge linearly: with the contraction th = d_k / d_{k-1} of
        // two steps on the same factor the remaining error is about d th / (1 - th);
        // a chord contracting by less than 10 gets a new factor. A first step on a
        // stored FP64-built factor below rtol / 10 is converged; one above
        // 1e-4 is undone and the factor rebuilt.
        if (it == 1) {
          if (!fac32 && d <= 0.1 * rtol) break;
          if (d > 1e-4) {
            for (int i = lane; i < nn; i += 32) w.xs[i] -= w.dx[i];
            __syncwarp();
            T = w.xs[N];
            have = false;
            d = INFINITY;
          }
        } else {
          // th = d / dprev < 0.1, and d th / (1 - th) = d^2 / (dprev - d) <= rtol,
          // both tested without dividing
          if (d < 0.1 * dprev) {
            if (d * d <= rtol * (dprev - d)) break;
          } else {
            have = false;
          }
        }
      }
      // chord steps only near the root: after a large step (d > 1e-4) the next
      // iteration builds a new factor, so far from convergence the iterates follow
      // Newton's own path (and the root it finds)
      if (MIXED && !exact && d > 1e-4) have = false;
      dprev = d;
    }
    if (code == 0 && it > maxit) code = -1;
    if (attempt == 0 && guessed && code == 0) {
      // the root reached from a learned guess must be the one the plain guess
      // leads to: near x_p (within 100 times the residual scale s there), and
      // without a mass fraction below the smallest of x_p (or 0) by more than
      // 1e-9 (a backward step of mass-action chemistry has one non-negative root)
      double far = 0.0, ymin = INFINITY, ypmin = 0.0;
      for (int i = lane; i < nn; i += 32) {
        far = fmax(far, (i < N) ? fabs(w.xs[i] - w.xg[i]) : fabs(w.xs[i] - w.xg[i]) / w.xg[i]);
        if (i < N) {
          ymin = fmin(ymin, w.xs[i]);
          ypmin = fmin(ypmin, w.xg[i]);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        far = fmax(far, __shfl_xor_sync(0xffffffffu, far, o));
        ymin = fmin(ymin, __shfl_xor_sync(0xffffffffu, ymin, o));
        ypmin = fmin(ypmin, __shfl_xor_sync(0xffffffffu, ypmin, o));
      }
      if (!(far <= 100.0 * s0 + 1e-10) || !(ymin >= ypmin - 1e-9))
        code = -4;   // another root: solve again from x_p
    }
    if (attempt == 0 && guessed && code) {
      ++my_rej;   // counted as a rejected guess
      --my_sg;
    }
    }   // attempt
    if (MIXED && code) {
      // both attempts failed: the cell keeps its finite starting point (the
      // failure is reported through the status word)
      for (int i = lane; i < nn; i += 32) w.xs[i] = w.xg[i];
      __syncwarp();
      T = w.xs[N];
    }
    // species enthalpies and theta at the solution; reaction term (Y - b)/wdt
    const double Tf = (code == -3 && !MIXED) ? 1000.0 : T;
    double th_f = 0.0;   // theta = (T/T_ref)^theta_exp = exp(theta_exp (ln T - ln T_ref))
    {
      double lnT = 0.0, invT = 0.0;
      if (lane == 0) {
        lnT = log(Tf);
        invT = 1.0 / Tf;
        th_f = exp_tab(m.theta_exp * (lnT - m.ln_Tref));
      }
      lnT = __shfl_sync(0xffffffffu, lnT, 0);
      invT = __shfl_sync(0xffffffffu, invT, 0);
      for (int i = lane; i < N; i += 32) {
        double hRT, gRT, cpR;
        species_thermo(m, i, Tf, lnT, invT, hRT, gRT, cpR);
        const double y = w.xs[i];
        Yout[(size_t)i * cs + cell] = y;
        if (FR) FR[(size_t)i * cs + cell] = (y - w.bs[i]) * invw;
        if (hsp) hsp[(size_t)i * cs + cell] = kRu * m.invW[i] * Tf * hRT;
      }
    }
    if (MIXED && cst.valid && lane == 0)
      cst.valid[cell] = ((have && code == 0 && !exact) ? 1 : 0) | (no32 ? 2 : 0) | (fac32 ? 4 : 0);
    if (lane == 0) {
      Tout[cell] = T;
      if (theta) theta[cell] = th_f;
      if (iters) iters[cell] = code ? code : it;
    }
    __syncwarp();
    my_solves++;
    if (code) {
      my_fail++;
      bits |= (code == -1) ? kBitNewton : (code == -2 ? kBitSingular : kBitNan);
    } else {
      my_iters += it;
      my_max = max(my_max, it);
    }
  }
  if (lane == 0 && my_solves) {
    atomicAdd(&st->newton_solves, my_solves);
    atomicAdd(&st->newton_iters, my_iters);
    if (my_fail) atomicAdd(&st->newton_fail, my_fail);
    atomicMax(&st->newton_max, my_max);
    if (bits) atomicOr(&st->status_bits, bits);
    if (my_sg) atomicAdd(&st->sg_used, my_sg);
    if (my_rej) atomicAdd(&st->sg_rejected, my_rej);
    if (my_fb) atomicAdd(&st->fp64_fallbacks, my_fb);
    if (my_jac) atomicAdd(&st->jacobians, my_jac);
    if (my_lu64) atomicAdd(&st->lu64, my_lu64);
    if (my_cert) atomicAdd(&st->certified, my_cert);
    if (my_stored) atomicAdd(&st->stored_steps, my_stored);
    if (my_floor) atomicAdd(&st->floor_stops, my_floor);
  }
}

// One solve: work items are a fixed grid-stride share per warp, or (A.work !=
// NULL) the next free item from a global counter, which balances the per-cell
// iteration counts.
template <bool MIXED>
__global__ void __launch_bounds__(128, 4) k_newton2(NewtonArgs A) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const size_t per_warp = newton_warp_doubles(A.m.N, A.m.R, A.ld, MIXED);
  int *work = A.work;
  auto next_item = [&](int cur) -> int {
    if (!work) return cur < 0 ? blockIdx.x * wpb + wib : cur + gridDim.x * wpb;
    int c = 0;
    if (lane == 0) c = atomicAdd(work, 1);
    return __shfl_sync(0xffffffffu, c, 0);
  };
  const int items = A.list ? *A.list_n : A.n;
  newton_items<MIXED>(A, smem + (size_t)wib * per_warp, next_item(-1), items, next_item);
}

// Several solves of one mechanism shape (independent flames at the same stage)
// in one persistent launch: their items are numbered one after another and each
// warp takes the next free number from one counter, so the per-cell iteration
// counts are balanced across the solves. A warp runs the items of a solve until
// the number it draws belongs to the next one.
template <bool MIXED>
__global__ void __launch_bounds__(128, 4) k_newton2_group(const NewtonArgs *__restrict__ jobs, int njobs,
                                                          int *__restrict__ work) {
  extern __shared__ double smem[];
  __shared__ int first_item[kMaxGroupJobs + 1];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int j = 0; j < njobs; ++j) {
      first_item[j] = acc;
      acc += jobs[j].list ? *jobs[j].list_n : jobs[j].n;
    }
    first_item[njobs] = acc;
  }
  __syncthreads();
  const int total = first_item[njobs];
  const size_t per_warp = newton_warp_doubles(jobs[0].m.N, jobs[0].m.R, jobs[0].ld, MIXED);
  double *wsm = smem + (size_t)wib * per_warp;
  auto draw = [&]() -> int {
    int c = 0;
    if (lane == 0) c = atomicAdd(work, 1);
    return __shfl_sync(0xffffffffu, c, 0);
  };
  int g = draw();
  while (g < total) {
    int f = 0;
    while (first_item[f + 1] <= g) ++f;   // the solve that item g belongs to
    const int lo = first_item[f], hi = first_item[f + 1];
    int after = total;   // the first drawn item past this solve
    auto next_item = [&](int) -> int {
      const int c = draw();
      if (c < hi) return c - lo;
      after = c;
      return hi - lo;
    };
    newton_items<MIXED>(jobs[f], wsm, g - lo, hi - lo, next_item);
    g = after;
  }
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

// warps per block: the requested count if its shared memory fits, else 4, 2 or 1
static size_t newton_smem(const DevMech &m, bool mixed, int &ld, int &wpb, int want = 0) {
  ld = newton_ld(m.N);
  const size_t per_warp = newton_warp_doubles(m.N, m.R, ld, mixed) * sizeof(double);
  const size_t cap = 200 * 1024;
  if (want < 1 || want > 4 || want * per_warp > cap) want = 0;
  wpb = want ? want : (4 * per_warp <= cap ? 4 : (2 * per_warp <= cap ? 2 : 1));
  return (size_t)wpb * per_warp;
}

int newton_max_wpb(const DevMech &m, bool mixed) {
  int ld, wpb;
  newton_smem(m, mixed, ld, wpb);
  return wpb;
}

static size_t rates_mma_smem(const DevMech &m) {
  return ((size_t)kMmaCells * mma_qld(m.R) + (size_t)4 * 5 * m.N) * sizeof(double);
}

// The shared-memory limit is an attribute of the kernel, not of a launch: every
// solver and every grouped launch in the process shares it, so it only ever grows
// to the largest need (a grouped launch already in a graph keeps its room).
static std::mutex g_smem_mu;
static size_t g_smem_have[7] = {0, 0, 0, 0, 0, 0, 0};

static void reserve_smem(int k, const void *fn, size_t need) {
  if (need > g_smem_have[k]) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    g_smem_have[k] = need;
  }
}

void prepare_chem_kernels(const DevMech &m) {
  std::lock_guard<std::mutex> lock(g_smem_mu);
  int ld, wpb;
  const size_t need[4] = {newton_smem(m, false, ld, wpb), newton_smem(m, true, ld, wpb),
                          (size_t)64 * 3 * m.N * sizeof(double), rates_mma_smem(m)};
  const void *fn[4] = {(const void *)k_newton2<false>, (const void *)k_newton2<true>,
                       (const void *)k_rates_t, (const void *)k_rates_mma};
  for (int k = 0; k < 4; ++k) reserve_smem(k, fn[k], need[k]);
  const size_t chord = chord_smem_bytes(m.N, 64);
  if (chord <= 200 * 1024) reserve_smem(6, (const void *)k_chord, chord);
}

void launch_temperature(const DevMech &m, int n, int cs, const double *Y, const double *h,
                        const double *Tguess, double *T, double *theta, double *hsp,
                        DevStats *st, cudaStream_t s) {
  if (n <= 0) return;
  k_temperature<<<(n + 255) / 256, 256, 0, s>>>(m, n, cs, Y, h, Tguess, T, theta, hsp, st);
}

void launch_enthalpy(const DevMech &m, int n, int cs, const double *Y, const double *T,
                     double *h, cudaStream_t s) {
  if (n <= 0) return;
  k_enthalpy<<<(n + 255) / 256, 256, 0, s>>>(m, n, cs, Y, T, h);
}

void launch_rates(const DevMech &m, int n, int cs, const double *Y, const double *T,
                  double *FR, cudaStream_t s, bool mma) {
  if (n <= 0) return;
  if (mma) {
    int grid = (n + kMmaCells - 1) / kMmaCells;
    grid = grid < sm_count() * 2 ? grid : sm_count() * 2;
    k_rates_mma<<<grid, 128, rates_mma_smem(m), s>>>(m, n, cs, Y, T, FR);
    return;
  }
  // one thread per cell (every FP64 lane busy: an FP64 warp instruction costs the
  // pipe the same whether 21 or 32 of its lanes work)
  const size_t sm = (size_t)64 * 3 * m.N * sizeof(double);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_rates_t, 64, sm);
  const int grid = std::max(1, std::min((n + 63) / 64, sm_count() * std::max(per_sm, 1)));
  k_rates_t<<<grid, 64, sm, s>>>(m, n, cs, Y, T, FR);
}

// Certification (k_certify, thread per cell, into `list`) and, where enabled and its
// shared-memory arrays fit, the thread-per-cell chord pass over the cells it left
// (k_chord, persistent, into `list2`). Returns the list the warp-per-cell Newton
// is to take.
static void launch_chord_pass(const DevMech &m, int n, int cs, double wdt, double rtol, int maxit,
                              const NewtonLaunch &cfg, const double *b, const double *hstar,
                              const double *Yg, const double *Tg, double *Y, double *T, double *FR,
                              double *hsp, double *theta, int *iters, DevStats *st, const double *sc,
                              double s_min, const int *prow, const double *FRp, const double *hp,
                              const ChordStore &cst, const double *hspp, const double *thp,
                              int **out_list, int **out_n, cudaStream_t s) {
  cudaMemsetAsync(cfg.list_n, 0, sizeof(int), s);
  k_certify<<<(n + 255) / 256, 256, 0, s>>>(m, n, cs, wdt, rtol, b, hstar, Yg, Tg, Y, T, FR, hsp, theta,
                                            iters, st, sc, s_min, prow, FRp, hp, cst, hspp, thp, cfg.list,
                                            cfg.list_n);
  *out_list = cfg.list;
  *out_n = cfg.list_n;
  const size_t smem = chord_smem_bytes(m.N, 64);
  if (cfg.chord_iters <= 0 || !cfg.list2 || !cfg.list2_n || smem > g_smem_have[6]) return;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_chord, 64, smem);
  const int grid = std::max(1, std::min((n + 63) / 64, sm_count() * std::max(per_sm, 1)));
  cudaMemsetAsync(cfg.list2_n, 0, sizeof(int), s);
  k_chord<<<grid, 64, smem, s>>>(m, n, cs, wdt, rtol, maxit, cfg.chord_iters, b, hstar, Yg, Tg, Y, T, FR,
                                 hsp, theta, iters, st, sc, s_min, prow, FRp, hp, cst, hspp, thp, cfg.list,
                                 cfg.list_n, cfg.list2, cfg.list2_n);
  *out_list = cfg.list2;
  *out_n = cfg.list2_n;
}

void launch_newton(const DevMech &m, int n, int cs, double wdt, double rtol, int maxit,
                   const double *b, const double *hstar, const double *Yg, const double *Tg,
                   double *Y, double *T, double *FR, double *hsp, double *theta, int *iters,
                   DevStats *st, cudaStream_t s, bool mixed, const float *pred, int ldp,
                   const double *sc, double s_min, const double *FRp, const double *hp,
                   const NewtonLaunch *cfg, const ChordStore *store, const int *prow,
                   const double *hspp, const double *thp) {
  if (n <= 0) return;
  int ld, wpb;
  const size_t sm = newton_smem(m, mixed, ld, wpb, cfg ? cfg->wpb : 0);
  int grid = (n + wpb - 1) / wpb;
  const int per_sm = (cfg && cfg->blocks_per_sm > 0) ? cfg->blocks_per_sm : (wpb == 4 ? 8 : 12);
  const int cap = sm_count() * per_sm;
  grid = grid < cap ? grid : cap;
  int *work = (cfg && cfg->dynamic) ? cfg->work : nullptr;
  if (work) cudaMemsetAsync(work, 0, sizeof(int), s);
  ChordStore cst{};
  if (mixed && store) cst = *store;
  // mixed precision with kept factors and the stored reaction terms of the
  // guesses: certification first (one thread per cell), then the warp-per-cell
  // Newton on the cells it left
  const bool split = mixed && cst.f && cst.valid && cst.z32 && cst.xc && cst.sT && FRp && hspp && hp &&
                     thp && cfg && cfg->list && cfg->list_n;
  const int *list = split ? cfg->list : nullptr, *list_n = split ? cfg->list_n : nullptr;
  if (split && !cfg->precertified) {
    int *l = nullptr, *ln = nullptr;
    launch_chord_pass(m, n, cs, wdt, rtol, maxit, *cfg, b, hstar, Yg, Tg, Y, T, FR, hsp, theta, iters, st,
                      pred ? sc : nullptr, s_min, prow, FRp, hp, cst, hspp, thp, &l, &ln, s);
    list = l;
    list_n = ln;
  }
  NewtonArgs A;
  A.m = m;
  A.n = n;
  A.cs = cs;
  A.wdt = wdt;
  A.rtol = rtol;
  A.maxit = maxit;
  A.ld = ld;
  A.b = b;
  A.hstar = hstar;
  A.Yg = Yg;
  A.Tg = Tg;
  A.Yout = Y;
  A.Tout = T;
  A.FR = FR;
  A.hsp = hsp;
  A.theta = theta;
  A.iters = iters;
  A.st = st;
  A.pred = pred;
  A.ldp = ldp;
  A.sc = sc;
  A.s_min = s_min;
  A.FRp = FRp;
  A.hp = hp;
  A.work = work;
  A.cst = cst;
  A.prow = prow;
  A.hspp = hspp;
  A.thp = thp;
  A.list = mixed ? list : nullptr;
  A.list_n = mixed ? list_n : nullptr;
  if (mixed)
    k_newton2<true><<<grid, wpb * 32, sm, s>>>(A);
  else
    k_newton2<false><<<grid, wpb * 32, sm, s>>>(A);
}

bool newton_kernel_args(const void *func, void **params, NewtonArgs *out, bool *mixed) {
  if (func == (const void *)k_newton2<true>) *mixed = true;
  else if (func == (const void *)k_newton2<false>) *mixed = false;
  else return false;
  *out = *(const NewtonArgs *)params[0];
  return true;
}

const void *newton_group_kernel(bool mixed) {
  return mixed ? (const void *)k_newton2_group<true> : (const void *)k_newton2_group<false>;
}

void newton_group_reserve_smem(bool mixed, size_t smem) {
  std::lock_guard<std::mutex> lock(g_smem_mu);
  reserve_smem(mixed ? 5 : 4, newton_group_kernel(mixed), smem);
}

int newton_group_grid(bool mixed, int wpb, size_t smem, int items) {
  const int blocks = (items + wpb - 1) / wpb;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, newton_group_kernel(mixed), wpb * 32, smem);
  if (per_sm <= 0) per_sm = 1;
  const int cap = sm_count() * per_sm;
  return blocks < 1 ? 1 : (blocks < cap ? blocks : cap);
}


bool launch_certify(const DevMech &m, int n, int cs, double wdt, double rtol, int maxit, const double *b,
                    const double *hstar, const double *Yg, const double *Tg, double *Y, double *T,
                    double *FR, double *hsp, double *theta, int *iters, DevStats *st,
                    const double *FRp, const double *hp, const ChordStore *store,
                    const double *hspp, const double *thp, NewtonLaunch *cfg, cudaStream_t s) {
  if (n <= 0 || !store) return false;
  const ChordStore &cst = *store;
  if (!(cst.f && cst.valid && cst.z32 && cst.xc && cst.sT && FRp && hspp && hp && thp && cfg &&
        cfg->list && cfg->list_n))
    return false;
  int *l = nullptr, *ln = nullptr;
  launch_chord_pass(m, n, cs, wdt, rtol, maxit, *cfg, b, hstar, Yg, Tg, Y, T, FR, hsp, theta, iters, st,
                    nullptr, 0.0, nullptr, FRp, hp, cst, hspp, thp, &l, &ln, s);
  cfg->list = l;      // the cells left for the learned guess and the warp-per-cell Newton
  cfg->list_n = ln;
  return true;
}

cudaError_t init_exp_table() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
  double tab[32];
  for (int j = 0; j < 32; ++j) tab[j] = (double)exp2l((long double)j / 32.0L);
  e = cudaMemcpyToSymbol(g_exp2_32, tab, sizeof(tab));
  if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
  return e;
}

cudaError_t launch_exp(const double *x, double *y, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t blocks = (n + 255) / 256;
  k_exp<<<(unsigned)(blocks < 65535 ? blocks : 65535), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

}  // namespace misdc
