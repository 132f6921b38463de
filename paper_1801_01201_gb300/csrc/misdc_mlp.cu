// Learned initial guess of the reaction Newton: a small MLP
// (n_in -> 256 -> 256 -> 256 -> n_out, GELU, BF16 weights and activations,
// FP32 accumulation) with forward, backward and AdamW kernels.
//
// The contractions run on the 5th-generation tensor cores: one CTA of four
// warps computes a 128 x N tile (N <= 256) with tcgen05.mma (kind::f16, BF16
// operands, FP32 accumulator in tensor memory). Operands are staged in shared
// memory in the canonical K-major layout without swizzle (core matrices of
// 8 rows x 16 bytes stored contiguously); MMA completion is tracked by an
// mbarrier and the accumulator is read back with tcgen05.ld for a fused
// epilogue (bias, GELU, GELU derivative, split-K accumulation).
//
// Features of a cell (n_in = 2N + 3), built from the guess x_p = (Y_p, T_p)
// of the reaction step, its reaction term F_p, its enthalpy h_p, and the
// step's b, h*, wdt:
//   r_i = b_i - Y_p,i + wdt F_p,i       (minus the Newton residual at x_p)
//   r_T = (h* - h_p) / (cp(x_p) T_p)
//   s   = max(max_i |r_i|, |r_T|)
//   f   = [Y_p, (T_p - 1150)/850, log10(wdt) + 6, r / s, r_T / s]
// Target (n_out = N + 1): [(Y* - Y_p)/s, (T* - T_p)/(T_p s)], clipped to
// [-8, 8]. The guess handed to Newton is Y_p + s p_Y, T_p (1 + s p_T).
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <random>
#include <vector>

#include "misdc_internal.cuh"

namespace misdc {
namespace mlp {

constexpr int kTileM = 128;   // rows per CTA = TMEM lanes
constexpr int kTileK = 64;    // K per shared-memory stage (4 MMAs of K = 16)
constexpr int kMaxN = 256;    // accumulator columns
constexpr int kThreads = 128;
constexpr long long kWaitCycles = 2000000000ll;   // about one second at 2 GHz
constexpr float kTargetClip = 8.0f;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, K-major, no swizzle: start address,
// lbo = byte distance between core matrices adjacent along K, sbo = between
// core matrices adjacent along M (N); bit 46 is the descriptor version.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait for phase `parity` of the mbarrier for at most kWaitCycles; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > kWaitCycles) return false;
  }
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 TMEM lanes x 16 consecutive 32-bit columns: thread t of the warp gets
// lane (base lane + t), columns [col, col + 16)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// Stage a tile_rows x 64 block of a BF16 operand (element (r, k) at p[r*sm + k*sk],
// rows >= nrows or k >= K read as zero) into core-matrix order: element (r, k)
// goes to ((r/8)*8 + k/8)*64 + (r%8)*8 + k%8.
__device__ __forceinline__ void stage(__nv_bfloat16 *dst, const Operand &op, int tile_rows, int r0,
                                      int k0, int K, bool vec) {
  const int tid = threadIdx.x;
  if (vec) {
    // 16-byte chunks (8 consecutive k); chunk e = ((r/8)*8 + kc)*8 + r%8 is also
    // its position in shared memory, so the stores are linear
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (int e = tid; e < tile_rows * 8; e += kThreads) {
      const int r7 = e & 7, kc = (e >> 3) & 7, rg = e >> 6;
      const int r = rg * 8 + r7, gr = r0 + r, gk = k0 + kc * 8;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (gr < op.rows && gk < K)
        v = *reinterpret_cast<const uint4 *>(op.p + (size_t)gr * op.sm + gk);
      d4[e] = v;
    }
  } else {
    // strided along K (transposed operand): consecutive threads take consecutive rows
    for (int e = tid; e < tile_rows * kTileK; e += kThreads) {
      const int r = e % tile_rows, k = e / tile_rows;
      const int gr = r0 + r, gk = k0 + k;
      __nv_bfloat16 v = __float2bfloat16(0.0f);
      if (gr < op.rows && gk < K) v = op.p[(size_t)gr * op.sm + (size_t)gk * op.sk];
      dst[((r >> 3) * 8 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7)] = v;
    }
  }
}

// C[M x N] (+)= A[M x K] B[K x N] with B given as Bt (N rows, K along the row).
// Grid: (ceil(M / 128), splits); CTA y handles K in [y k_split, (y+1) k_split).
// N is a multiple of 16 in [16, 256]. Dynamic shared memory: kGemmSmemLaunch.
__global__ void __launch_bounds__(kThreads) k_umma_gemm(Operand A, Operand Bt, int M, int N, int K,
                                                        int k_split, int vecA, int vecB, Epi ep,
                                                        int *err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(smraw);
  __nv_bfloat16 *sB = reinterpret_cast<__nv_bfloat16 *>(smraw + kTileM * kTileK * 2);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smraw + (kTileM + kMaxN) * kTileK * 2);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTileM;
  const int kb = blockIdx.y * k_split, ke = min(K, kb + k_split);
  const uint32_t ncols = (N <= 32) ? 32u : (N <= 64 ? 64u : (N <= 128 ? 128u : 256u));

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) mbar_init(bar, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const uint32_t idesc = instr_desc(kTileM, N);
  bool ok = true;
  int issued = 0;

  for (int k0 = kb; k0 < ke; k0 += kTileK) {
    stage(sA, A, kTileM, m0, k0, ke, vecA != 0);
    stage(sB, Bt, N, 0, k0, ke, vecB != 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
      for (int kk = 0; kk < kTileK / 16; ++kk) {
        // K = 16 spans two core matrices along K (lbo = 128 B); 8-row groups are
        // 8 core matrices apart (sbo = 1024 B)
        const uint64_t da = smem_desc(a0 + kk * 256, 128, 1024);
        const uint64_t db = smem_desc(b0 + kk * 256, 128, 1024);
        umma_bf16(tmem, da, db, idesc, (issued > 0 || kk > 0) ? 1u : 0u);
      }
      umma_commit(bar);
    }
    __syncwarp();
    if (!mbar_wait(bar, (uint32_t)(issued & 1))) ok = false;   // stage consumed
    ++issued;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (!__syncthreads_and(ok)) { ok = false; break; }
  }

  // epilogue: warp w owns TMEM lanes 32w..32w+31 = tile rows
  const int row = m0 + warp * 32 + lane;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  if (ok && issued > 0) {
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tmem_ld16(trow + (uint32_t)c0, v);
      if (row < M) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int col = c0 + i;
          if (col >= ep.n_store) continue;
          const size_t o = (size_t)row * ep.ldo + col;
          float x = v[i];
          switch (ep.mode) {
            case kEpiStore:
              if (ep.bias) x += ep.bias[col];
              ep.out_f32[o] = x;
              break;
            case kEpiBiasGelu:
              x += ep.bias[col];
              if (ep.out_f32) ep.out_f32[o] = x;
              ep.out_bf16[o] = __float2bfloat16(gelu(x));
              break;
            case kEpiGeluGrad: {
              const float g = x * gelu_grad(ep.zsaved[o]);
              if (ep.out_f32) ep.out_f32[o] = g;
              ep.out_bf16[o] = __float2bfloat16(g);
              break;
            }
            default:
              atomicAdd(ep.out_f32 + o, x);
          }
        }
      }
    }
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

// ---------------------------------------------------------------------------
// elementwise kernels
// ---------------------------------------------------------------------------

// Features (see the file header) of cells [0, n) and their scale s [n]. Dense
// mode (counter == NULL): row c of X [n][ldx] (columns >= n_in zero). Record
// mode: cells with s > s_min take the next free row of X [cap][ldx] through
// *counter and store it in rowmap[c] (-1: not recorded). Thread per cell.
__global__ void k_features(DevMech m, int n, int cs, double wdt, const double *__restrict__ b,
                           const double *__restrict__ hstar, const double *__restrict__ Yp,
                           const double *__restrict__ Tp, const double *__restrict__ FRp,
                           const double *__restrict__ hp, int ldx, __nv_bfloat16 *__restrict__ X,
                           double *__restrict__ scale, double s_min,
                           unsigned long long *__restrict__ counter, long long cap,
                           int *__restrict__ rowmap, const int *__restrict__ list,
                           const int *__restrict__ list_n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (list ? *list_n : n)) return;
  const int c = list ? list[k] : k;
  const int N = m.N;
  const double T = Tp[c];
  double cp = 0.0, rmax = 0.0;
  bool finite = isfinite(T) && T > 0.0;
  for (int i = 0; i < N; ++i) {
    const double *a = m.cpcoef + 5 * i;
    const double cpR = a[0] + T * (a[1] + T * (a[2] + T * (a[3] + T * a[4])));
    const double y = Yp[(size_t)i * cs + c];
    cp = fma(y, kRu * m.invW[i] * cpR, cp);
    const double r = b[(size_t)i * cs + c] - y + wdt * FRp[(size_t)i * cs + c];
    finite = finite && isfinite(y) && isfinite(r);   // (fmax below would drop a NaN)
    rmax = fmax(rmax, fabs(r));
  }
  const double rT = (hstar[c] - hp[c]) / (cp * T);
  const double s = fmax(rmax, fabs(rT));
  const double inv = (s > 0.0) ? 1.0 / s : 0.0;
  scale[c] = s;
  long long row = c;
  if (counter) {
    row = -1;
    // a cell whose state is not finite (a failed solve upstream) gives no row
    if (s > s_min && isfinite(s) && finite) {
      row = (long long)atomicAdd(counter, 1ull);
      if (row >= cap) row = -1;
    }
    rowmap[c] = (int)row;
    if (row < 0) return;
  }
  __nv_bfloat16 *x = X + (size_t)row * ldx;
  for (int i = 0; i < N; ++i) {
    const double y = Yp[(size_t)i * cs + c];
    x[i] = __double2bfloat16(y);
    x[N + 2 + i] =
        __double2bfloat16((b[(size_t)i * cs + c] - y + wdt * FRp[(size_t)i * cs + c]) * inv);
  }
  x[N] = __double2bfloat16((T - 1150.0) / 850.0);
  x[N + 1] = __double2bfloat16(log10(wdt) + 6.0);
  x[2 * N + 2] = __double2bfloat16(rT * inv);
  for (int j = 2 * N + 3; j < ldx; ++j) x[j] = __float2bfloat16(0.0f);
}

// Training targets of cells [0, n) after their solve, into row rowmap[c] of
// tgt [.][ldt] (f32; cells with rowmap[c] < 0 are skipped).
__global__ void k_targets(int N, int n, int cs, const double *__restrict__ Yp,
                          const double *__restrict__ Tp, const double *__restrict__ Ys,
                          const double *__restrict__ Ts, const double *__restrict__ scale,
                          const int *__restrict__ rowmap, int ldt, float *__restrict__ tgt) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int row = rowmap[c];
  if (row < 0) return;
  const double s = scale[c];
  const double inv = (s > 0.0) ? 1.0 / s : 0.0;
  float *t = tgt + (size_t)row * ldt;
  bool finite = isfinite(Ts[c]) && Ts[c] > 0.0;
  for (int i = 0; i < N; ++i) finite = finite && isfinite(Ys[(size_t)i * cs + c]);
  if (!finite) {   // the solve failed: a zero step, not a NaN
    for (int j = 0; j < ldt; ++j) t[j] = 0.0f;
    return;
  }
  for (int i = 0; i < N; ++i) {
    const double d = (Ys[(size_t)i * cs + c] - Yp[(size_t)i * cs + c]) * inv;
    t[i] = (float)fmin(fmax(d, -(double)kTargetClip), (double)kTargetClip);
  }
  const double dT = (Ts[c] - Tp[c]) / Tp[c] * inv;
  t[N] = (float)fmin(fmax(dT, -(double)kTargetClip), (double)kTargetClip);
  for (int j = N + 1; j < ldt; ++j) t[j] = 0.0f;
}

// Mean-squared loss over the first n_out columns and its gradient:
// dO = 2 (O - Y) / (B n_out) as f32 and bf16; the loss is added to *loss.
__global__ void k_mse(int B, int n_out, int ld, const float *__restrict__ O,
                      const float *__restrict__ Yt, float *__restrict__ dO,
                      __nv_bfloat16 *__restrict__ dOb, float *__restrict__ loss) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (e < (size_t)B * ld) {
    const int col = (int)(e % ld);
    float g = 0.0f;
    if (col < n_out) {
      const float d = O[e] - Yt[e];
      l = d * d;
      g = 2.0f * d / ((float)B * (float)n_out);
    }
    dO[e] = g;
    dOb[e] = __float2bfloat16(g);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && l != 0.0f) atomicAdd(loss, l / ((float)B * (float)n_out));
}

// out[j] += sum_r in[r][j] for j < n; block (32, 8)
__global__ void k_colsum(int rows, int n, int ld, const float *__restrict__ in,
                         float *__restrict__ out) {
  __shared__ float part[8][33];
  const int j = blockIdx.x * 32 + threadIdx.x;
  float s = 0.0f;
  if (j < n)
    for (int r = threadIdx.y; r < rows; r += 8) s += in[(size_t)r * ld + j];
  part[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.y == 0 && j < n) {
    float t = 0.0f;
    for (int k = 0; k < 8; ++k) t += part[k][threadIdx.x];
    out[j] += t;
  }
}

// AdamW (Adam with decoupled weight decay) on the flat FP32 parameter vector;
// the first n_decay entries (the weights) decay, the rest (biases) do not.
// Refreshes the BF16 copy.
__global__ void k_adamw(size_t n, size_t n_decay, float *__restrict__ P, const float *__restrict__ G,
                        float *__restrict__ Mm, float *__restrict__ Vm,
                        __nv_bfloat16 *__restrict__ Pb, float lr, float beta1, float beta2,
                        float eps, float wd, float bc1, float bc2) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = G[i];
  const float mi = beta1 * Mm[i] + (1.0f - beta1) * g;
  const float vi = beta2 * Vm[i] + (1.0f - beta2) * g * g;
  Mm[i] = mi;
  Vm[i] = vi;
  float p = P[i];
  if (i < n_decay) p -= lr * wd * p;
  p -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  P[i] = p;
  Pb[i] = __float2bfloat16(p);
}

__global__ void k_to_bf16(size_t n, const float *__restrict__ in, __nv_bfloat16 *__restrict__ out) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16(in[i]);
}

// splitmix64 output function (Steele, Lea & Flood, 2014) as a counter-based generator
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Minibatch gather: batch row b is dataset row mix64(seed + b) mod rows.
__global__ void k_gather(int B, long long rows, unsigned long long seed, int ldx, int ldt,
                         const __nv_bfloat16 *__restrict__ DX, const float *__restrict__ DT,
                         __nv_bfloat16 *__restrict__ X, float *__restrict__ Yt) {
  const int bi = blockIdx.x;
  if (bi >= B) return;
  const long long r =
      (long long)(mix64(seed + (unsigned long long)bi) % (unsigned long long)rows);
  for (int j = threadIdx.x; j < ldx; j += blockDim.x) X[(size_t)bi * ldx + j] = DX[(size_t)r * ldx + j];
  for (int j = threadIdx.x; j < ldt; j += blockDim.x) Yt[(size_t)bi * ldt + j] = DT[(size_t)r * ldt + j];
}

// ---------------------------------------------------------------------------
// Fused inference: features (or given BF16 rows) -> four layers -> outputs, one
// CTA per 128 rows. Activations never leave the SM: each layer's FP32
// accumulator lives in tensor memory, its GELU epilogue writes the BF16 result
// back into shared memory as the next layer's A operand. Weights stream through
// a two-stage shared-memory ring in K chunks of 64, the copy of chunk k+1
// overlapping the MMAs of chunk k.
// ---------------------------------------------------------------------------
constexpr int kFThreads = 256;               // 8 warps: 2 per TMEM lane quadrant
constexpr int kFKmax = 256;                  // widest layer input
constexpr int kFSmemA = kTileM * kFKmax * 2; // 64 KB, A operand, core-matrix layout
constexpr int kFSmemB = kMaxN * kTileK * 2;  // 32 KB per weight stage
constexpr int kFSmem = kFSmemA + 2 * kFSmemB + 64;

struct FusedArgs {
  // features from the state (FEAT) ...
  DevMech m;
  int cs;
  double wdt;
  const double *b, *hstar, *Yp, *Tp, *FRp, *hp;
  double *scale;
  // ... or BF16 rows X [n][ldx]
  const __nv_bfloat16 *X;
  const unsigned long long *count;   // optional: rows actually present (device), <= n
  int n, ldx, k1;          // rows, feature row length, layer-1 K (ldx rounded up to 64)
  const __nv_bfloat16 *W[4];
  const float *bias[4];
  int ldo;                 // output width (layer-4 N, multiple of 16)
  float *out;              // [n][ldo]
  int *err;
};

// element (r, k) of the 128 x 256 A buffer: ((r/8)*32 + k/8)*64 + (r%8)*8 + k%8
__device__ __forceinline__ int a_index(int r, int k) {
  return (((r >> 3) << 5) + (k >> 3)) * 64 + ((r & 7) << 3) + (k & 7);
}

template <bool FEAT>
__global__ void __launch_bounds__(kFThreads, 1) k_mlp_fused(FusedArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  __nv_bfloat16 *sA = reinterpret_cast<__nv_bfloat16 *>(smraw);
  __nv_bfloat16 *sB0 = reinterpret_cast<__nv_bfloat16 *>(smraw + kFSmemA);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smraw + kFSmemA + 2 * kFSmemB);   // [2]
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  int nrows = a.n;
  if (a.count) {   // compacted rows: only the tiles below the device row count
    const unsigned long long nr = *a.count;
    if (nr < (unsigned long long)nrows) nrows = (int)nr;
  }
  const int ntiles = (nrows + kTileM - 1) / kTileM;
  if ((int)blockIdx.x >= ntiles) return;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  uint32_t phase[2] = {0u, 0u};
  bool ok = true;
  // persistent CTAs: one 128-row tile after another
  for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
  const int r0 = tile * kTileM;
  // ---- layer-1 input rows into the A buffer
  if (FEAT) {
    if (tid < kTileM) {
      const int r = tid, c = r0 + r;
      const int N = a.m.N;
      if (c < nrows) {
        const int cs = a.cs;
        const double T = a.Tp[c];
        double cp = 0.0, rmax = 0.0;
        for (int i = 0; i < N; ++i) {
          const double *q = a.m.cpcoef + 5 * i;
          const double cpR = q[0] + T * (q[1] + T * (q[2] + T * (q[3] + T * q[4])));
          const double y = a.Yp[(size_t)i * cs + c];
          cp = fma(y, kRu * a.m.invW[i] * cpR, cp);
          rmax = fmax(rmax, fabs(a.b[(size_t)i * cs + c] - y + a.wdt * a.FRp[(size_t)i * cs + c]));
        }
        const double rT = (a.hstar[c] - a.hp[c]) / (cp * T);
        const double sc = fmax(rmax, fabs(rT));
        const double inv = (sc > 0.0) ? 1.0 / sc : 0.0;
        a.scale[c] = sc;
        // features straight into the A buffer (columns beyond n_in stay zero)
        for (int i = 0; i < N; ++i) {
          const double y = a.Yp[(size_t)i * cs + c];
          sA[a_index(r, i)] = __double2bfloat16(y);
          sA[a_index(r, N + 2 + i)] =
              __double2bfloat16((a.b[(size_t)i * cs + c] - y + a.wdt * a.FRp[(size_t)i * cs + c]) * inv);
        }
        sA[a_index(r, N)] = __double2bfloat16((T - 1150.0) / 850.0);
        sA[a_index(r, N + 1)] = __double2bfloat16(log10(a.wdt) + 6.0);
        sA[a_index(r, 2 * N + 2)] = __double2bfloat16(rT * inv);
        for (int j = 2 * N + 3; j < a.k1; ++j) sA[a_index(r, j)] = __float2bfloat16(0.0f);
      } else {
        for (int j = 0; j < a.k1; ++j) sA[a_index(r, j)] = __float2bfloat16(0.0f);
      }
    }
  } else {
    for (int e = tid; e < kTileM * a.k1; e += kFThreads) {
      const int r = e / a.k1, k = e - r * a.k1, c = r0 + r;
      __nv_bfloat16 v = __float2bfloat16(0.0f);
      if (c < nrows && k < a.ldx) v = a.X[(size_t)c * a.ldx + k];
      sA[a_index(r, k)] = v;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");

  for (int L = 0; L < 4; ++L) {
    const int K = (L == 0) ? a.k1 : kFKmax;
    const int N = (L == 3) ? a.ldo : kMaxN;
    const int ldw = (L == 0) ? a.ldx : kFKmax;   // weight row length (K of the stored matrix)
    const int kvalid = (L == 0) ? a.ldx : kFKmax;
    const __nv_bfloat16 *W = a.W[L];
    const uint32_t idesc = instr_desc(kTileM, N);
    const int nch = K / kTileK;
    for (int kc = 0; kc < nch; ++kc) {
      const int st = kc & 1;
      __nv_bfloat16 *sB = sB0 + st * (kFSmemB / 2);
      if (kc >= 2) {   // the MMAs of chunk kc-2 read this stage
        if (!mbar_wait(bar + st, phase[st])) ok = false;
        phase[st] ^= 1u;
      }
      // weight chunk: rows n < N, K columns [64 kc, 64 kc + 64), 16-byte pieces
      for (int e = tid; e < N * 8; e += kFThreads) {
        const int r7 = e & 7, q = (e >> 3) & 7, rg = e >> 6;
        const int nrow = rg * 8 + r7, k = kc * kTileK + q * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (k < kvalid) v = *reinterpret_cast<const uint4 *>(W + (size_t)nrow * ldw + k);
        reinterpret_cast<uint4 *>(sB)[e] = v;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = smem_u32(sA) + kc * 1024, b0 = smem_u32(sB);
#pragma unroll
        for (int kk = 0; kk < kTileK / 16; ++kk) {
          const uint64_t da = smem_desc(a0 + kk * 256, 128, 4096);
          const uint64_t db = smem_desc(b0 + kk * 256, 128, 1024);
          umma_bf16(tmem, da, db, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
        }
        umma_commit(bar + st);
      }
      __syncwarp();
    }
    // wait for the outstanding commits in order: all MMAs of the layer are done
    for (int kc = (nch >= 2 ? nch - 2 : 0); kc < nch; ++kc) {
      const int st = kc & 1;
      if (!mbar_wait(bar + st, phase[st])) ok = false;
      phase[st] ^= 1u;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    ok = __syncthreads_and(ok);
    if (!ok) break;
    // epilogue: warp w reads lanes 32 (w % 4) .. + 31; the N/16 column chunks are
    // split between the two warps of a lane quadrant (the first takes the odd one)
    const int quad = warp & 3, half = warp >> 2;
    const int row = quad * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
    const int nck = N / 16, first = (nck + 1) / 2;
    const int cbeg = half ? first * 16 : 0, cend = half ? N : first * 16;
    const float *bias = a.bias[L];
    for (int c0 = cbeg; c0 < cend; c0 += 16) {
      float v[16];
      tmem_ld16(trow + (uint32_t)c0, v);
      if (L < 3) {
#pragma unroll
        for (int i = 0; i < 16; ++i) sA[a_index(row, c0 + i)] = __float2bfloat16(gelu(v[i] + bias[c0 + i]));
      } else if (r0 + row < nrows) {
        float *o = a.out + (size_t)(r0 + row) * a.ldo;
#pragma unroll
        for (int i = 0; i < 16; ++i) o[c0 + i] = v[i] + bias[c0 + i];
      }
    }
    // the next layer's MMAs read sA and overwrite tensor memory
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
  }
  }   // tile
  if (!ok && tid == 0) atomicExch(a.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

}  // namespace mlp

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
using namespace mlp;

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

void mlp_prepare() {
  // 100 KB of shared memory keeps at most two CTAs (2 x 256 TMEM columns) per SM,
  // so tcgen05.alloc never waits for another CTA's columns; the fused kernel
  // (160 KB) runs one CTA per SM
  cudaFuncSetAttribute(k_umma_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmemLaunch);
  cudaFuncSetAttribute(k_mlp_fused<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFSmem);
  cudaFuncSetAttribute(k_mlp_fused<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFSmem);
}

void mlp_fused_forward(const Surrogate &g, const DevMech *m, int cs, double wdt, const double *b,
                       const double *hstar, const double *Yp, const double *Tp, const double *FRp,
                       const double *hp, double *scale, const __nv_bfloat16 *X, int n, float *out,
                       cudaStream_t s, const unsigned long long *count) {
  if (n <= 0) return;
  FusedArgs a;
  memset(&a, 0, sizeof(a));
  if (m) a.m = *m;
  a.cs = cs;
  a.wdt = wdt;
  a.b = b; a.hstar = hstar; a.Yp = Yp; a.Tp = Tp; a.FRp = FRp; a.hp = hp; a.scale = scale;
  a.X = X;
  a.count = count;
  a.n = n;
  a.ldx = g.ldx;
  a.k1 = (g.ldx + kTileK - 1) / kTileK * kTileK;
  for (int L = 0; L < 4; ++L) {
    a.W[L] = g.Pb + g.off[L];
    a.bias[L] = g.P + g.off[4 + L];
  }
  a.ldo = g.ldo;
  a.out = out;
  a.err = g.err;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int tiles = (n + kTileM - 1) / kTileM;
  const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);   // one 160 KB CTA per SM
  if (m)
    k_mlp_fused<true><<<grid, kFThreads, kFSmem, s>>>(a);
  else
    k_mlp_fused<false><<<grid, kFThreads, kFSmem, s>>>(a);
}

void mlp_gemm(const Operand &A, const Operand &Bt, int M, int N, int K, int splits, const Epi &ep,
              int *err, cudaStream_t s) {
  if (M <= 0 || K <= 0 || N <= 0 || N > kMaxN) return;
  const int Np = (N + 15) / 16 * 16;
  splits = splits < 1 ? 1 : splits;
  int k_split = (K + splits - 1) / splits;
  k_split = (k_split + kTileK - 1) / kTileK * kTileK;
  const int gy = (K + k_split - 1) / k_split;
  const int vecA = (A.sk == 1 && A.sm % 8 == 0 && K % 8 == 0 && aligned16(A.p)) ? 1 : 0;
  const int vecB = (Bt.sk == 1 && Bt.sm % 8 == 0 && K % 8 == 0 && aligned16(Bt.p)) ? 1 : 0;
  dim3 grid((M + kTileM - 1) / kTileM, gy);
  k_umma_gemm<<<grid, kThreads, kGemmSmemLaunch, s>>>(A, Bt, M, Np, K, k_split, vecA, vecB, ep,
                                                      err);
}

void mlp_features(const DevMech &m, int n, int cs, double wdt, const double *b,
                  const double *hstar, const double *Yp, const double *Tp, const double *FRp,
                  const double *hp, int ldx, __nv_bfloat16 *X, double *scale, double s_min,
                  unsigned long long *counter, long long cap, int *rowmap, cudaStream_t s,
                  const int *list, const int *list_n) {
  if (n <= 0) return;
  k_features<<<(n + 127) / 128, 128, 0, s>>>(m, n, cs, wdt, b, hstar, Yp, Tp, FRp, hp, ldx, X,
                                             scale, s_min, counter, cap, rowmap, list, list_n);
}

void mlp_targets(int N, int n, int cs, const double *Yp, const double *Tp, const double *Ys,
                 const double *Ts, const double *scale, const int *rowmap, int ldt, float *tgt,
                 cudaStream_t s) {
  if (n <= 0) return;
  k_targets<<<(n + 127) / 128, 128, 0, s>>>(N, n, cs, Yp, Tp, Ys, Ts, scale, rowmap, ldt, tgt);
}

void mlp_mse(int B, int n_out, int ld, const float *O, const float *Yt, float *dO,
             __nv_bfloat16 *dOb, float *loss, cudaStream_t s) {
  const size_t n = (size_t)B * ld;
  if (!n) return;
  k_mse<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(B, n_out, ld, O, Yt, dO, dOb, loss);
}

void mlp_colsum(int rows, int n, int ld, const float *in, float *out, cudaStream_t s) {
  if (n <= 0) return;
  k_colsum<<<(n + 31) / 32, dim3(32, 8), 0, s>>>(rows, n, ld, in, out);
}

void mlp_adamw(size_t n, size_t n_decay, float *P, const float *G, float *Mm, float *Vm,
               __nv_bfloat16 *Pb, float lr, float beta1, float beta2, float eps, float wd,
               float bc1, float bc2, cudaStream_t s) {
  if (!n) return;
  k_adamw<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, n_decay, P, G, Mm, Vm, Pb, lr, beta1,
                                                      beta2, eps, wd, bc1, bc2);
}

void mlp_to_bf16(size_t n, const float *in, __nv_bfloat16 *out, cudaStream_t s) {
  if (!n) return;
  k_to_bf16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, in, out);
}

void mlp_gather(int B, long long rows, unsigned long long seed, int ldx, int ldt,
                const __nv_bfloat16 *DX, const float *DT, __nv_bfloat16 *X, float *Yt,
                cudaStream_t s) {
  if (B <= 0 || rows <= 0) return;
  k_gather<<<B, 64, 0, s>>>(B, rows, seed, ldx, ldt, DX, DT, X, Yt);
}

// ---------------------------------------------------------------------------
// Surrogate: parameters, buffers and the forward / backward / AdamW passes
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t Surrogate::alloc(T **p, size_t n) {
  cudaError_t e = cudaMalloc((void **)p, (n ? n : 1) * sizeof(T));
  if (e == cudaSuccess) allocs.push_back(*p);
  return e;
}

Surrogate::~Surrogate() {
  for (void *p : allocs) cudaFree(p);
}

#define SG_CK(call)                          \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return e_;        \
  } while (0)

cudaError_t Surrogate::setup(int n_species) {
  N = n_species;
  n_in = 2 * N + 3;
  ldx = (n_in + 7) / 8 * 8;
  n_out = N + 1;
  ldo = (n_out + 15) / 16 * 16;
  off[0] = 0;
  off[1] = off[0] + (size_t)H * ldx;
  off[2] = off[1] + (size_t)H * H;
  off[3] = off[2] + (size_t)H * H;
  n_weights = off[3] + (size_t)ldo * H;
  off[4] = n_weights;
  off[5] = off[4] + H;
  off[6] = off[5] + H;
  off[7] = off[6] + H;
  n_params = off[7] + ldo;
  SG_CK(alloc(&P, n_params));
  SG_CK(alloc(&G, n_params));
  SG_CK(alloc(&Mm, n_params));
  SG_CK(alloc(&Vm, n_params));
  SG_CK(alloc(&Pb, n_params));
  SG_CK(alloc(&err, 1));
  SG_CK(cudaMemset(err, 0, sizeof(int)));
  SG_CK(cudaMemset(P, 0, n_params * sizeof(float)));
  SG_CK(cudaMemset(Pb, 0, n_params * sizeof(__nv_bfloat16)));
  return cudaSuccess;
}

// Uniform initialisation with variance 1/fan_in for the hidden layers and a
// 0.1 smaller output layer, so that an untrained network predicts a small
// correction; zero biases.
void Surrogate::init_params(unsigned long long seed, std::vector<float> &h) const {
  h.assign(n_params, 0.0f);
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  auto fill = [&](size_t o, int rows, int cols, int ld, int fan_in, double gain) {
    const double a = gain * sqrt(3.0 / fan_in);
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) h[o + (size_t)r * ld + c] = (float)(a * u(rng));
  };
  fill(off[0], H, n_in, ldx, n_in, 1.0);
  fill(off[1], H, H, H, H, 1.0);
  fill(off[2], H, H, H, H, 1.0);
  fill(off[3], n_out, H, H, H, 0.1);
}

cudaError_t Surrogate::upload(const float *host, cudaStream_t s) {
  SG_CK(cudaMemcpyAsync(P, host, n_params * sizeof(float), cudaMemcpyHostToDevice, s));
  SG_CK(cudaMemsetAsync(Mm, 0, n_params * sizeof(float), s));
  SG_CK(cudaMemsetAsync(Vm, 0, n_params * sizeof(float), s));
  mlp_to_bf16(n_params, P, Pb, s);
  adam_t = 0;
  ready = true;
  return cudaGetLastError();
}

cudaError_t Surrogate::ensure_inference(int cells) {
  if (cells <= cap_inf) return cudaSuccess;
  cap_inf = cells;
  SG_CK(alloc(&Xi, (size_t)cells * ldx));
  SG_CK(alloc(&Ha, (size_t)cells * H));
  SG_CK(alloc(&Hb, (size_t)cells * H));
  SG_CK(alloc(&Oi, (size_t)cells * ldo));
  SG_CK(alloc(&scale, (size_t)cells));
  SG_CK(alloc(&rowmap, (size_t)cells));
  if (!inf_count) SG_CK(alloc(&inf_count, 1));
  return cudaSuccess;
}

cudaError_t Surrogate::ensure_training(int batch, int steps) {
  if (steps > loss_cap) {
    loss_cap = steps;
    SG_CK(alloc(&loss, (size_t)steps));
  }
  if (batch <= cap_tr) return cudaSuccess;
  cap_tr = batch;
  const size_t B = batch;
  SG_CK(alloc(&Xt, B * ldx));
  SG_CK(alloc(&H1, B * H));
  SG_CK(alloc(&H2, B * H));
  SG_CK(alloc(&H3, B * H));
  SG_CK(alloc(&dOb, B * ldo));
  SG_CK(alloc(&dZa, B * H));
  SG_CK(alloc(&dZb, B * H));
  SG_CK(alloc(&Z1, B * H));
  SG_CK(alloc(&Z2, B * H));
  SG_CK(alloc(&Z3, B * H));
  SG_CK(alloc(&Ot, B * ldo));
  SG_CK(alloc(&dO, B * ldo));
  SG_CK(alloc(&dZf, B * H));
  SG_CK(alloc(&Yt, B * ldo));
  return cudaSuccess;
}

cudaError_t Surrogate::ensure_dataset(long long cap) {
  if (!ds_count) {
    SG_CK(alloc(&ds_count, 1));
    SG_CK(cudaMemset(ds_count, 0, sizeof(unsigned long long)));
  }
  if (cap <= ds_cap) return cudaSuccess;
  // a larger dataset starts empty
  SG_CK(alloc(&DX, (size_t)cap * ldx));
  SG_CK(alloc(&DT, (size_t)cap * ldo));
  SG_CK(cudaMemset(ds_count, 0, sizeof(unsigned long long)));
  ds_cap = cap;
  return cudaSuccess;
}

void Surrogate::forward(const __nv_bfloat16 *X, int n, float *O, bool train, cudaStream_t s) {
  const __nv_bfloat16 *W1 = Pb + off[0], *W2 = Pb + off[1], *W3 = Pb + off[2], *W4 = Pb + off[3];
  __nv_bfloat16 *h1 = train ? H1 : Ha, *h2 = train ? H2 : Hb, *h3 = train ? H3 : Ha;
  Epi e{kEpiBiasGelu, H, H, P + off[4], train ? Z1 : nullptr, h1, nullptr};
  mlp_gemm(Operand{X, ldx, 1, n}, Operand{W1, ldx, 1, H}, n, H, ldx, 1, e, err, s);
  e.bias = P + off[5];
  e.out_f32 = train ? Z2 : nullptr;
  e.out_bf16 = h2;
  mlp_gemm(Operand{h1, H, 1, n}, Operand{W2, H, 1, H}, n, H, H, 1, e, err, s);
  e.bias = P + off[6];
  e.out_f32 = train ? Z3 : nullptr;
  e.out_bf16 = h3;
  mlp_gemm(Operand{h2, H, 1, n}, Operand{W3, H, 1, H}, n, H, H, 1, e, err, s);
  const Epi e4{kEpiStore, ldo, ldo, P + off[7], O, nullptr, nullptr};
  mlp_gemm(Operand{h3, H, 1, n}, Operand{W4, H, 1, ldo}, n, ldo, H, 1, e4, err, s);
}

void Surrogate::backward(const __nv_bfloat16 *X, int B, float *loss_slot, cudaStream_t s) {
  const __nv_bfloat16 *W2 = Pb + off[1], *W3 = Pb + off[2], *W4 = Pb + off[3];
  const int splits = B / 256 < 1 ? 1 : (B / 256 > 32 ? 32 : B / 256);
  mlp_mse(B, n_out, ldo, Ot, Yt, dO, dOb, loss_slot, s);
  cudaMemsetAsync(G, 0, n_params * sizeof(float), s);
  // output layer: dW4 = dO^T H3, db4 = colsum dO
  mlp_gemm(Operand{dOb, 1, ldo, n_out}, Operand{H3, 1, H, H}, n_out, H, B, splits,
           Epi{kEpiAtomic, H, H, nullptr, G + off[3], nullptr, nullptr}, err, s);
  mlp_colsum(B, n_out, ldo, dO, G + off[7], s);
  // dZ3 = (dO W4) gelu'(Z3)
  mlp_gemm(Operand{dOb, ldo, 1, B}, Operand{W4, 1, H, H}, B, H, ldo, 1,
           Epi{kEpiGeluGrad, H, H, nullptr, dZf, dZa, Z3}, err, s);
  mlp_gemm(Operand{dZa, 1, H, H}, Operand{H2, 1, H, H}, H, H, B, splits,
           Epi{kEpiAtomic, H, H, nullptr, G + off[2], nullptr, nullptr}, err, s);
  mlp_colsum(B, H, H, dZf, G + off[6], s);
  // dZ2 = (dZ3 W3) gelu'(Z2)
  mlp_gemm(Operand{dZa, H, 1, B}, Operand{W3, 1, H, H}, B, H, H, 1,
           Epi{kEpiGeluGrad, H, H, nullptr, dZf, dZb, Z2}, err, s);
  mlp_gemm(Operand{dZb, 1, H, H}, Operand{H1, 1, H, H}, H, H, B, splits,
           Epi{kEpiAtomic, H, H, nullptr, G + off[1], nullptr, nullptr}, err, s);
  mlp_colsum(B, H, H, dZf, G + off[5], s);
  // dZ1 = (dZ2 W2) gelu'(Z1)
  mlp_gemm(Operand{dZb, H, 1, B}, Operand{W2, 1, H, H}, B, H, H, 1,
           Epi{kEpiGeluGrad, H, H, nullptr, dZf, dZa, Z1}, err, s);
  mlp_gemm(Operand{dZa, 1, H, H}, Operand{X, 1, ldx, ldx}, H, ldx, B, splits,
           Epi{kEpiAtomic, ldx, ldx, nullptr, G + off[0], nullptr, nullptr}, err, s);
  mlp_colsum(B, H, H, dZf, G + off[4], s);
}

void Surrogate::adamw(float lr, float wd, cudaStream_t s) {
  ++adam_t;
  const double b1 = 0.9, b2 = 0.999;
  const float bc1 = (float)(1.0 - pow(b1, (double)adam_t));
  const float bc2 = (float)(1.0 - pow(b2, (double)adam_t));
  mlp_adamw(n_params, n_weights, P, G, Mm, Vm, Pb, lr, (float)b1, (float)b2, 1e-8f, wd, bc1, bc2, s);
}

}  // namespace misdc
