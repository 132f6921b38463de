// Chemistry kernels: temperature diagnosis, production rates and the per-cell
// reaction Newton solve of step S5 (Sec. 3.3, eq.
// reaction_step_numerical_methodology), one warp per cell.
//
// Layout: every per-cell array is field-major, [field][cs] with a cell stride cs.
#include <math.h>

#include "misdc_internal.cuh"

namespace misdc {

namespace {

__device__ __forceinline__ void species_thermo(const DevMech &m, int i, double T, double lnT,
                                               double invT, double &hRT, double &gRT,
                                               double &cpR) {
  const double *a = m.hcoef + 6 * i;
  hRT = fma(a[5], invT, a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4]))));
  const double *s = m.scoef + 6 * i;
  double sR = fma(s[0], lnT, T * (s[1] + T * (s[2] + T * (s[3] + T * s[4])))) + s[5];
  gRT = hRT - sR;
  const double *c = m.cpcoef + 5 * i;
  cpR = c[0] + T * (c[1] + T * (c[2] + T * (c[3] + T * c[4])));
}

template <int RPL>
__device__ __forceinline__ double pick(const double (&a)[RPL], int q) {
  return (RPL == 1 || q == 0) ? a[0] : a[RPL - 1];
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
  mix_h_cp(m, Y, cs, c, lo, fl, d);
  mix_h_cp(m, Y, cs, c, hi, fh, d);
  double T;
  if (!(fl - h <= 0.0 && fh - h >= 0.0)) {
    atomicOr(&st->status_bits, kBitTdiag);
    T = NAN;
  } else {
    T = (Tg && Tg[c] > lo && Tg[c] < hi) ? Tg[c] : 1000.0;
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

__device__ __forceinline__ WarpChem carve(double *p, int N, int R) {
  WarpChem w;
  w.c = p; w.g = p + N; w.hRT = p + 2 * N; w.hm = p + 3 * N; w.cpm = p + 4 * N;
  w.q = p + 5 * N; w.kf = w.q + R; w.kr = w.kf + R; w.dqdT = w.kr + R;
  return w;
}

// thermo of every species at T, then every reaction's rate of progress (and
// what the Jacobian needs); concentrations w.c must be set.
__device__ void eval_chem(const DevMech &m, const WarpChem &w, int lane, double T, bool jac) {
  const double lnT = log(T), invT = 1.0 / T;
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
    const double kf = exp(lnkf);
    const double kr = exp(lnkf - lnKc);
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

// wdot_i = sum_r W_i nu_ri q_r for the species rows a lane owns
__device__ __forceinline__ double species_wdot(const DevMech &m, const WarpChem &w, int i) {
  double s = 0.0;
  for (int p = m.sp_ptr[i]; p < m.sp_ptr[i + 1]; ++p) s = fma(m.sp_coef[p], w.q[m.sp_rx[p]], s);
  return s;
}

__global__ void __launch_bounds__(128) k_rates(DevMech m, int n, int cs,
                                               const double *__restrict__ Y,
                                               const double *__restrict__ T,
                                               double *__restrict__ FR) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int N = m.N, R = m.R;
  WarpChem w = carve(smem + (size_t)wib * (5 * N + 4 * R), N, R);
  const double invrho = 1.0 / m.rho;
  for (int cell = blockIdx.x * wpb + wib; cell < n; cell += gridDim.x * wpb) {
    for (int i = lane; i < N; i += 32) w.c[i] = m.rho * Y[(size_t)i * cs + cell] * m.invW[i];
    __syncwarp();
    eval_chem(m, w, lane, T[cell], false);
    for (int i = lane; i < N; i += 32) FR[(size_t)i * cs + cell] = species_wdot(m, w, i) * invrho;
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Reaction Newton: one warp per cell, rows of the augmented (N+1)x(N+2)
// Jacobian in shared memory, lane i owns rows i, i+32, ...; partial pivoting
// by a warp argmax; dense LU by rank-1 row updates.
// Unknowns x = (Y_1..Y_N, T); residual r_i = Y_i - wdt wdot_i/rho - b_i,
// r_T = sum_i Y_i h_i(T) - h*.
// ---------------------------------------------------------------------------
template <int RPL>
__global__ void __launch_bounds__(128) k_newton(DevMech m, int n, int cs, double wdt, double rtol,
                                                int maxit, int ld, const double *__restrict__ b,
                                                const double *__restrict__ hstar,
                                                const double *Yg, const double *Tg,
                                                double *Yout, double *Tout,
                                                double *__restrict__ FR,
                                                double *__restrict__ hsp,
                                                double *__restrict__ theta,
                                                int *__restrict__ iters, DevStats *st) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int N = m.N, R = m.R, nn = N + 1;
  const size_t per_warp = (size_t)nn * ld + 5 * N + 4 * R;
  double *J = smem + (size_t)wib * per_warp;
  WarpChem w = carve(J + (size_t)nn * ld, N, R);
  const double invrho = 1.0 / m.rho, wr = wdt * invrho;
  const int qT = N >> 5, lT = N & 31;   // owner of the temperature row
  unsigned long long my_solves = 0, my_iters = 0, my_fail = 0;
  int my_max = 0;
  unsigned bits = 0;

  for (int cell = blockIdx.x * wpb + wib; cell < n; cell += gridDim.x * wpb) {
    double x[RPL], bb[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      int i = lane + 32 * q;
      x[q] = (i < N) ? Yg[(size_t)i * cs + cell] : (i == N ? Tg[cell] : 0.0);
      bb[q] = (i < N) ? b[(size_t)i * cs + cell] : 0.0;
    }
    const double hst = hstar[cell];
    double T = __shfl_sync(0xffffffffu, pick<RPL>(x, qT), lT);
    double dprev = INFINITY;
    int it, code = 0;
    for (it = 1; it <= maxit; ++it) {
      // concentrations, thermo and rates at the current iterate
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        int i = lane + 32 * q;
        if (i < N) w.c[i] = m.rho * x[q] * m.invW[i];
      }
      __syncwarp();
      eval_chem(m, w, lane, T, true);
      // species rows of the augmented Jacobian
      double sh = 0.0, scp = 0.0;
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        int i = lane + 32 * q;
        if (i < N) {
          double *row = J + (size_t)i * ld;
          for (int j = 0; j <= nn; ++j) row[j] = 0.0;
          row[i] = 1.0;
          double wd = 0.0, jT = 0.0;
          for (int p = m.sp_ptr[i]; p < m.sp_ptr[i + 1]; ++p) {
            const int r = m.sp_rx[p];
            const double co = m.sp_coef[p];
            wd = fma(co, w.q[r], wd);
            const double a = -wdt * co;
            const signed char *fs = m.fwd + kMaxSlots * r, *rs = m.rev + kMaxSlots * r;
#pragma unroll
            for (int s0 = 0; s0 < kMaxSlots; ++s0) {
              int sp = fs[s0];
              if (sp >= 0) {
                double prod = w.kf[r];
#pragma unroll
                for (int s1 = 0; s1 < kMaxSlots; ++s1)
                  if (s1 != s0 && fs[s1] >= 0) prod *= w.c[fs[s1]];
                row[sp] = fma(a * m.invW[sp], prod, row[sp]);
              }
              sp = rs[s0];
              if (sp >= 0) {
                double prod = w.kr[r];
#pragma unroll
                for (int s1 = 0; s1 < kMaxSlots; ++s1)
                  if (s1 != s0 && rs[s1] >= 0) prod *= w.c[rs[s1]];
                row[sp] = fma(-a * m.invW[sp], prod, row[sp]);
              }
            }
            jT = fma(co, w.dqdT[r], jT);
          }
          row[N] -= wr * jT;
          row[nn] = -(x[q] - wr * wd - bb[q]);
          sh = fma(x[q], w.hm[i], sh);
          scp = fma(x[q], w.cpm[i], scp);
        }
      }
      sh = warp_sum(sh);
      scp = warp_sum(scp);
      // temperature row: d/dY_j = h_j, d/dT = cp
      double *rowT = J + (size_t)N * ld;
      for (int j = lane; j < N; j += 32) rowT[j] = w.hm[j];
      if (lane == 0) { rowT[N] = scp; rowT[nn] = -(sh - hst); }
      __syncwarp();

      // LU with partial pivoting on the augmented matrix
      bool singular = false;
      for (int k = 0; k < nn; ++k) {
        double best = -1.0;
        int bi = nn;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          int i = lane + 32 * q;
          if (i >= k && i < nn) {
            double v = fabs(J[(size_t)i * ld + k]);
            if (v > best) { best = v; bi = i; }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          double ob = __shfl_xor_sync(0xffffffffu, best, o);
          int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (!(best > 0.0) || !isfinite(best)) { singular = true; break; }
        if (bi != k) {
          for (int j = lane; j <= nn; j += 32) {
            double t = J[(size_t)k * ld + j];
            J[(size_t)k * ld + j] = J[(size_t)bi * ld + j];
            J[(size_t)bi * ld + j] = t;
          }
        }
        __syncwarp();
        const double *rk = J + (size_t)k * ld;
        const double pinv = 1.0 / rk[k];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          int i = lane + 32 * q;
          if (i > k && i < nn) {
            double *ri = J + (size_t)i * ld;
            const double l = ri[k] * pinv;
            for (int j = k + 1; j <= nn; ++j) ri[j] = fma(-l, rk[j], ri[j]);
          }
        }
        __syncwarp();
      }
      if (singular) { code = -2; break; }
      double dx[RPL];
#pragma unroll
      for (int q = 0; q < RPL; ++q) dx[q] = 0.0;
      for (int k = nn - 1; k >= 0; --k) {
        const double xk = J[(size_t)k * ld + nn] / J[(size_t)k * ld + k];
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          int i = lane + 32 * q;
          if (i < k) J[(size_t)i * ld + nn] = fma(-J[(size_t)i * ld + k], xk, J[(size_t)i * ld + nn]);
          if (i == k) dx[q] = xk;
        }
        __syncwarp();
      }
      // update and convergence on d = max(max|dY|, |dT|/T): d <= rtol, or d <= 1e-8
      // no longer halving (the round-off floor of very stiff cells)
      bool fin = true;
      double dmax = 0.0;
      const double dT = __shfl_sync(0xffffffffu, pick<RPL>(dx, qT), lT);
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        int i = lane + 32 * q;
        if (i < nn) {
          x[q] += dx[q];
          if (!isfinite(x[q])) fin = false;
          if (i < N) dmax = fmax(dmax, fabs(dx[q]));
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      T = __shfl_sync(0xffffffffu, pick<RPL>(x, qT), lT);
      fin = __all_sync(0xffffffffu, fin);
      if (!fin || !(T > 0.0)) { code = -3; break; }
      const double d = fmax(dmax, fabs(dT) / T);
      if (!isfinite(d)) { code = -3; break; }
      if (d <= rtol || (d <= 1e-8 && d >= 0.5 * dprev)) break;
      dprev = d;
    }
    if (code == 0 && it > maxit) code = -1;
    // species enthalpies and theta at the solution; the reaction term of the new
    // state is the one the implicit equation assigns to it, (Y - b)/wdt
    const double Tf = (code == -3) ? 1000.0 : T;
    {
      const double lnT = log(Tf), invT = 1.0 / Tf;
      for (int i = lane; i < N; i += 32) {
        double hRT, gRT, cpR;
        species_thermo(m, i, Tf, lnT, invT, hRT, gRT, cpR);
        w.hm[i] = kRu * m.invW[i] * Tf * hRT;
      }
    }
    __syncwarp();
    const double invw = (wdt > 0.0) ? 1.0 / wdt : 0.0;
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      int i = lane + 32 * q;
      if (i < N) {
        Yout[(size_t)i * cs + cell] = x[q];
        if (FR) FR[(size_t)i * cs + cell] = (x[q] - bb[q]) * invw;
        if (hsp) hsp[(size_t)i * cs + cell] = w.hm[i];
      }
    }
    if (lane == 0) {
      Tout[cell] = T;
      if (theta) theta[cell] = pow(Tf / m.T_ref, m.theta_exp);
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

static size_t newton_smem(const DevMech &m, int &ld, int &wpb) {
  const int nn = m.N + 1;
  ld = nn + 1;
  if ((ld & 1) == 0) ld += 1;   // odd leading dimension spreads rows over banks
  const size_t per_warp = (size_t)nn * ld + 5 * m.N + 4 * m.R;
  wpb = (per_warp * 8 * 4 <= 200 * 1024) ? 4 : 2;
  return (size_t)wpb * per_warp * sizeof(double);
}

void prepare_chem_kernels(const DevMech &m) {
  int ld, wpb;
  const size_t sm = newton_smem(m, ld, wpb);
  cudaFuncSetAttribute(k_newton<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  cudaFuncSetAttribute(k_newton<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const size_t smr = (size_t)4 * (5 * m.N + 4 * m.R) * sizeof(double);
  cudaFuncSetAttribute(k_rates, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr);
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
                  double *FR, cudaStream_t s) {
  if (n <= 0) return;
  const int wpb = 4;
  size_t sm = (size_t)wpb * (5 * m.N + 4 * m.R) * sizeof(double);
  int grid = (n + wpb - 1) / wpb;
  grid = grid < sm_count() * 16 ? grid : sm_count() * 16;
  k_rates<<<grid, wpb * 32, sm, s>>>(m, n, cs, Y, T, FR);
}

void launch_newton(const DevMech &m, int n, int cs, double wdt, double rtol, int maxit,
                   const double *b, const double *hstar, const double *Yg, const double *Tg,
                   double *Y, double *T, double *FR, double *hsp, double *theta, int *iters,
                   DevStats *st, cudaStream_t s) {
  if (n <= 0) return;
  const int nn = m.N + 1;
  int ld, wpb;
  const size_t sm = newton_smem(m, ld, wpb);
  int grid = (n + wpb - 1) / wpb;
  const int cap = sm_count() * (wpb == 4 ? 8 : 12);
  grid = grid < cap ? grid : cap;
  if (nn <= 32) {
    k_newton<1><<<grid, wpb * 32, sm, s>>>(m, n, cs, wdt, rtol, maxit, ld, b, hstar, Yg, Tg, Y, T,
                                           FR, hsp, theta, iters, st);
  } else {
    k_newton<2><<<grid, wpb * 32, sm, s>>>(m, n, cs, wdt, rtol, maxit, ld, b, hstar, Yg, Tg, Y, T,
                                           FR, hsp, theta, iters, st);
  }
}

}  // namespace misdc
