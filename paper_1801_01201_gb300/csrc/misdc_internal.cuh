// Internal declarations shared by the CUDA translation units of libmisdc.
// Not part of the C ABI (see include/misdc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/misdc.h"

namespace misdc {

constexpr double kRu = 8.314462618;        // J/(mol K)
constexpr double kTlo = 50.0, kThi = 6000.0;   // temperature range of the one-range polynomials
constexpr int kMaxSlots = 3;               // molecules per reaction side
constexpr int kMaxSpecies = 63;
constexpr int kMaxNodes = 9;
constexpr int kMaxCheb = 512;   // cap on Chebyshev sweeps per diffusion solve

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
};

// Mechanism tables in device memory (built by the engine from misdc_mech_desc).
struct DevMech {
  int N, R;
  double rho, T_ref, theta_exp, alpha0, ln_p_over_R;
  const double *invW;      // [N] 1/W
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
};

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
                  double *FR, cudaStream_t s);
// Reaction Newton (S5). b [N][cs], hstar [cs], guess Yg [N][cs], Tg [cs];
// outputs Y, T, FR (wdot/rho at the solution), hsp [N][cs] and theta at the solution.
void launch_newton(const DevMech &m, int n, int cs, double wdt, double rtol, int maxit,
                   const double *b, const double *hstar, const double *Yg, const double *Tg,
                   double *Y, double *T, double *FR, double *hsp, double *theta, int *iters,
                   DevStats *st, cudaStream_t s, bool mixed = false);

// ---- grid kernels (misdc_grid.cu) ----
struct LinComb {
  int n_out, n_in;
  double *out[8];
  const double *in[16];
  double w[8][16];
};
void launch_lincomb(const LinComb &lc, size_t n, cudaStream_t s);
void launch_operators(const DevMech &m, const DevGrid &g, int i0, const double *phi,
                      const double *hsp, const double *theta_face, const double *vel,
                      double *FE, double *FD, cudaStream_t s);
// theta at cells -> theta at the low face of every cell (harmonic mean)
void launch_theta_faces(const DevGrid &g, const double *theta, double *thf, cudaStream_t s);
void prepare_chem_kernels(const DevMech &m);
// D-step solve of every field but i0: (I - c_f L_theta) x = rhs, Chebyshev-accelerated
// Jacobi (the multigrid smoother), optional V-cycles, reconstruction and closure.
struct DiffWork {
  double *thf;       // [dim][cs] face coefficients
  double *invdiag;   // [N+1][cs]
  double *xa, *xb, *xc;   // [N+1][cs] iterates
  double *res;       // [N+1][cs] residual (multigrid)
  unsigned long long *rho_bits;   // measured Gershgorin bound (bit pattern)
  int *kdev;                      // planned Chebyshev sweep count
  double *omega;                  // [kMaxCheb] Chebyshev weights
  // multigrid levels (level 0 = this grid, compact [solved field][cells] storage)
  int levels, cycles;
  DevGrid lg[8];
  double *lthf[8], *linvdiag[8], *lb[8], *lx[8], *lr[8], *ly[8];
};
void diffusion_solve(const DevMech &m, const DevGrid &g, int i0, double wdt, const double *theta,
                     const double *rhs, double *out, DiffWork &w, int sweeps, double rho_bound,
                     double lin_rtol, DevStats *st, cudaStream_t s);
int chebyshev_sweeps(double rho_bound, double reduction);

}  // namespace misdc
