// Learned warm start of the equilibrium solve (Sec. 5, "Computing Equilibrium
// States": x(p) is recomputed by Newton's method after every design update;
// this module predicts its starting point from the design).
//
//   design map    p = Phi theta, Phi[e][k] = exp(-|X_e - c_k|^2 / (2 w^2))
//   basis         mean u_bar and leading left singular vectors U of the
//                 centred displacement snapshots, by a randomised SVD (range
//                 finder with one power iteration, Halko, Martinsson & Tropp
//                 2011): tall GEMMs on the GPU, only R x R eigenproblems on
//                 the host (R = n_modes + 32)
//   network       3-layer MLP with exact GELU, BF16 operands / FP32
//                 accumulation, FP32 master weights, AdamW on the GPU
//   warm start    x0 = X + u_bar + U (scale * MLP(theta * in_scale))
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <type_traits>
#include <vector>

#include <cuda.h>

#include "../../include/sgn_learn.h"
#include "common.cuh"
#include "tc_update.cuh"

namespace {

using bf16 = __nv_bfloat16;
using sgn::Ctx;
constexpr int TPB = 256;
inline unsigned nblk(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + TPB - 1) / TPB); }

// SplitMix64 (Steele, Lea & Flood 2014): counter-based 64-bit generator
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__host__ __device__ inline double u01(uint64_t r) { return ((double)(r >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

template <typename ACC, typename T>
__device__ __forceinline__ ACC as_acc(T v) {
  if constexpr (std::is_same_v<T, bf16>) return (ACC)__bfloat162float(v);
  else return (ACC)v;
}

// ------------------------------------------------ BF16 GEMM on tcgen05
// C(m, n) = alpha sum_k A(m, k) B(k, n) + beta C(m, n) for the MLP layers:
// both operands are first packed (converted to BF16, zero-padded) into
// K-major tiles, A as [Mp][Kp] and B as [Np][Kp] (Mp a multiple of 128, Np
// of 64, Kp of 64), then one CTA per 128 x 64 output tile streams 64-wide K
// stages by TMA (128B swizzle) and accumulates in TMEM with
// tcgen05.mma.kind::f16 (BF16 inputs, FP32 accumulation), 4 MMAs of K = 16
// per stage.  Warp 0 lane 0 issues the copies, warp 1 lane 0 the MMAs, all
// four warps read TMEM (32 lanes = 32 rows each) for the epilogue.  Every
// wait is bounded and records DEV_TIMEOUT on expiry.
constexpr int GM = 128, GN = 64, GK = 64, GSTAGES = 3;
constexpr int GA_BYTES = GM * GK * 2, GB_BYTES = GN * GK * 2, GSTAGE_BYTES = GA_BYTES + GB_BYTES;
constexpr int GSMEM = GSTAGES * GSTAGE_BYTES + 1024;

// instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = GN
constexpr uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GN >> 3) << 17) | ((uint32_t)(GM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__global__ void __launch_bounds__(128, 1) k_gemm_bf16_tc(const __grid_constant__ CUtensorMap ma,
                                                          const __grid_constant__ CUtensorMap mb, int M, int N,
                                                          int kchunks, float alpha, float beta, float *__restrict__ C,
                                                          int64_t scm, int64_t scn, int *status) {
  using namespace sgn::tc;
  extern __shared__ __align__(1024) unsigned char g_smem_raw[];
  __shared__ uint64_t full_bar[GSTAGES], empty_bar[GSTAGES], done_bar;
  __shared__ uint32_t tmem_base;
  unsigned char *sm = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(g_smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
  if (threadIdx.x == 0) {
    for (int s = 0; s < GSTAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
    mbar_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(GN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (warp == 0 && lane == 0) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&ma) : "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&mb) : "memory");
    int issued = 0;
    for (int kc = 0; kc < kchunks; ++kc) {
      const int s = kc % GSTAGES;
      if (kc >= GSTAGES && !mbar_wait(&empty_bar[s], ((kc / GSTAGES) - 1) & 1, status, sgn::DEV_TIMEOUT)) break;
      unsigned char *st = sm + s * GSTAGE_BYTES;
      mbar_expect_tx(&full_bar[s], GSTAGE_BYTES);
      tma_load_2d(st, &ma, &full_bar[s], kc * GK, m0);
      tma_load_2d(st + GA_BYTES, &mb, &full_bar[s], kc * GK, n0);
      issued = kc + 1;
    }
    // the copies still in flight complete before the CTA can exit (bounded)
    for (int q = (issued > GSTAGES ? issued - GSTAGES : 0); q < issued; ++q)
      mbar_wait(&full_bar[q % GSTAGES], (q / GSTAGES) & 1, status, sgn::DEV_TIMEOUT);
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16();
    for (int kc = 0; kc < kchunks; ++kc) {
      const int s = kc % GSTAGES;
      if (!mbar_wait(&full_bar[s], (kc / GSTAGES) & 1, status, sgn::DEV_TIMEOUT)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t base = smem_u32(sm + s * GSTAGE_BYTES);
#pragma unroll
      for (int k = 0; k < GK / 16; ++k) {
        const uint64_t ad = umma_desc_sw128(base + k * 32);
        const uint64_t bd = umma_desc_sw128(base + GA_BYTES + k * 32);
        umma_bf16(tmem, ad, bd, idesc, (kc | k) != 0);
      }
      umma_commit(&empty_bar[s]);
    }
    umma_commit(&done_bar);  // also after an early exit, so the epilogue does not wait out its bound
  }
  __syncwarp();
  const bool ok = __all_sync(0xffffffffu, mbar_wait(&done_bar, 0, status, sgn::DEV_TIMEOUT));
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int m = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int cb = 0; cb < GN; cb += 32) {
      uint32_t v[32];
      tmem_ld_32x32b_x32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
      if (m < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int n = n0 + cb + j;
          if (n < N) {
            float *c = C + (int64_t)m * scm + (int64_t)n * scn;
            const float r = alpha * __uint_as_float(v[j]);
            *c = beta != 0.f ? r + beta * *c : r;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GN) : "memory");
}

// dst[r][c] (rowsP x colsP, BF16) = src(r, c) = src[r srs + c scs] inside
// rows x cols, zero outside
template <typename TS>
__global__ void k_pack_bf16(int rows, int cols, const TS *__restrict__ src, int64_t srs, int64_t scs,
                            bf16 *__restrict__ dst, int rowsP, int colsP) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)rowsP * colsP) return;
  const int r = (int)(i / colsP), cc = (int)(i % colsP);
  float v = 0.f;
  if (r < rows && cc < cols) v = as_acc<float>(src[(int64_t)r * srs + (int64_t)cc * scs]);
  dst[i] = __float2bfloat16_rn(v);
}

// ------------------------------------------------------------------- GEMMs
// C(m, n) = alpha sum_k A(m, k) B(k, n) + beta C(m, n), arbitrary strides:
// A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn], C(m, n) = C[m scm + n scn].
// 64 x 64 output tile per CTA, 256 threads with 4 x 4 outputs each, K staged
// by 16 through shared memory; operand loads run along whichever index has
// unit stride.  With split-K (gridDim.z > 1) CTA z reduces its K range into
// ws[z][M][N] and k_splitk_sum finishes C.
template <typename TA, typename TB, typename TC, typename ACC>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, int kchunk, ACC alpha, const TA *__restrict__ A,
                                              int64_t sam, int64_t sak, const TB *__restrict__ B, int64_t sbk,
                                              int64_t sbn, ACC beta, TC *__restrict__ C, int64_t scm, int64_t scn,
                                              ACC *__restrict__ ws) {
  __shared__ ACC As[16][65], Bs[16][65];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const bool a_k_fast = (sak == 1), b_k_fast = (sbk == 1);
  ACC acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = ACC(0);
  for (int k0 = kb; k0 < ke; k0 += 16) {
    ACC av[4], bv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = tid + u * 256;  // 1024 = 16 (k) x 64 (row / column)
      int kk = a_k_fast ? (idx & 15) : (idx >> 6);
      int r = a_k_fast ? (idx >> 4) : (idx & 63);
      const int m = m0 + r;
      int k = k0 + kk;
      av[u] = (m < M && k < ke) ? as_acc<ACC>(A[(int64_t)m * sam + (int64_t)k * sak]) : ACC(0);
      kk = b_k_fast ? (idx & 15) : (idx >> 6);
      r = b_k_fast ? (idx >> 4) : (idx & 63);
      const int n = n0 + r;
      k = k0 + kk;
      bv[u] = (n < N && k < ke) ? as_acc<ACC>(B[(int64_t)k * sbk + (int64_t)n * sbn]) : ACC(0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = tid + u * 256;
      if (a_k_fast) As[idx & 15][idx >> 4] = av[u];
      else As[idx >> 6][idx & 63] = av[u];
      if (b_k_fast) Bs[idx & 15][idx >> 4] = bv[u];
      else Bs[idx >> 6][idx & 63] = bv[u];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      ACC a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + ty + 16 * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int n = n0 + tx + 16 * j;
      if (n >= N) continue;
      if (ws) {
        ws[((int64_t)blockIdx.z * M + m) * N + n] = acc[i][j];
      } else {
        TC *c = C + (int64_t)m * scm + (int64_t)n * scn;
        ACC v = alpha * acc[i][j];
        if (beta != ACC(0)) v += beta * (ACC)(*c);
        *c = (TC)v;
      }
    }
  }
}

template <typename TC, typename ACC>
__global__ void k_splitk_sum(int M, int N, int splits, ACC alpha, const ACC *__restrict__ ws, ACC beta,
                             TC *__restrict__ C, int64_t scm, int64_t scn) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)M * N) return;
  ACC s = ACC(0);
  for (int z = 0; z < splits; ++z) s += ws[(int64_t)z * M * N + i];
  const int m = (int)(i / N), n = (int)(i % N);
  TC *c = C + (int64_t)m * scm + (int64_t)n * scn;
  ACC v = alpha * s;
  if (beta != ACC(0)) v += beta * (ACC)(*c);
  *c = (TC)v;
}

template <typename TA, typename TB, typename TC, typename ACC>
void gemm(Ctx &c, int M, int N, int K, ACC alpha, const TA *A, int64_t sam, int64_t sak, const TB *B, int64_t sbk,
          int64_t sbn, ACC beta, TC *C, int64_t scm, int64_t scn, ACC *ws = nullptr, int64_t ws_elems = 0) {
  if (M <= 0 || N <= 0) return;
  const int64_t tiles = (int64_t)((M + 63) / 64) * ((N + 63) / 64);
  int splits = 1;
  if (ws && K > 4096 && tiles < 2 * (int64_t)c.num_sms) {
    const int64_t want = (2 * (int64_t)c.num_sms + tiles - 1) / tiles;
    splits = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)K / 2048, want, 64, ws_elems / ((int64_t)M * N)}));
  }
  int kchunk = K;
  if (splits > 1) {
    kchunk = (((K + splits - 1) / splits + 15) / 16) * 16;
    splits = (K + kchunk - 1) / kchunk;
  }
  dim3 g((N + 63) / 64, (M + 63) / 64, splits);
  k_gemm<TA, TB, TC, ACC><<<g, 256, 0, c.stream>>>(M, N, K, kchunk, alpha, A, sam, sak, B, sbk, sbn, beta, C, scm,
                                                  scn, splits > 1 ? ws : nullptr);
  c.count();
  if (splits > 1) {
    k_splitk_sum<TC, ACC><<<nblk((int64_t)M * N), TPB, 0, c.stream>>>(M, N, splits, alpha, ws, beta, C, scm, scn);
    c.count();
  }
}

// ------------------------------------------------------------ small kernels
__global__ void k_phi(int ne, int nr, int dim, const double *__restrict__ cent, const double *__restrict__ ctr,
                      double inv2w2, double *__restrict__ phi) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)ne * nr) return;
  const int e = (int)(i / nr), k = (int)(i % nr);
  double d2 = 0.0;
  for (int a = 0; a < dim; ++a) {
    const double t = cent[(int64_t)e * dim + a] - ctr[(int64_t)k * dim + a];
    d2 += t * t;
  }
  phi[i] = exp(-d2 * inv2w2);
}

// mean[i] = (1 / ns) sum_j A[i + j n]
__global__ void k_rowmean(int64_t n, int ns, const double *__restrict__ A, double *__restrict__ mean) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int j = 0; j < ns; ++j) s += A[i + (int64_t)j * n];
  mean[i] = s / ns;
}

// standard normal draws, Box-Muller on two SplitMix64 outputs per entry
__global__ void k_gauss(int64_t n, uint64_t seed, double *__restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t s = splitmix64(seed);
  const double u1 = u01(splitmix64(s ^ (2 * (uint64_t)i))), u2 = u01(splitmix64(s ^ (2 * (uint64_t)i + 1)));
  out[i] = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// s[j] = sum_i A[i + j rows]
__global__ void k_colsum(int rows, int cols, const double *__restrict__ A, double *__restrict__ s) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  double t = 0.0;
  for (int i = 0; i < rows; ++i) t += A[i + (int64_t)j * rows];
  s[j] = t;
}

// C[m scm + n scn] -= u[m] v[n] (u == nullptr: u = 1)
__global__ void k_rank1_sub(int M, int N, const double *__restrict__ u, const double *__restrict__ v,
                            double *__restrict__ C, int64_t scm, int64_t scn) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)M * N) return;
  const int m = (int)(i % M), n = (int)(i / M);
  C[m * scm + n * scn] -= (u ? u[m] : 1.0) * v[n];
}

// weights ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)), biases (fan_in 0) zero
__global__ void k_init_params(int64_t n, const int32_t *__restrict__ fan_in, uint64_t seed, float *__restrict__ p32,
                              bf16 *__restrict__ p16, float *__restrict__ m, float *__restrict__ v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int fi = fan_in[i];
  float w = 0.f;
  if (fi > 0) w = (float)((2.0 * u01(splitmix64(seed + (uint64_t)i)) - 1.0) / sqrt((double)fi));
  p32[i] = w;
  p16[i] = __float2bfloat16(w);
  m[i] = 0.f;
  v[i] = 0.f;
}

__global__ void k_to_bf16(int64_t n, const float *__restrict__ a, bf16 *__restrict__ b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16(a[i]);
}

// out = 1 / rms(a) (1 when a is all zero); one CTA
__global__ void k_inv_rms(int64_t n, const double *__restrict__ a, float *__restrict__ out) {
  __shared__ double sh[TPB];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += TPB) s += a[i] * a[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double rms = sqrt(sh[0] / (double)(n > 0 ? n : 1));
    out[0] = rms > 0.0 ? (float)(1.0 / rms) : 1.f;
  }
}

// per-column rms of a row-major [rows][cols] matrix (1 for an all-zero column)
__global__ void k_col_rms(int rows, int cols, const double *__restrict__ a, float *__restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  double s = 0.0;
  for (int i = 0; i < rows; ++i) s += a[(int64_t)i * cols + j] * a[(int64_t)i * cols + j];
  const double rms = sqrt(s / (rows > 0 ? rows : 1));
  out[j] = rms > 0.0 ? (float)rms : 1.f;
}

// training matrices: X[s][k] = theta[s][k] in_scale, T[s][m] = coef[s][m] / scale[m]
__global__ void k_prep_xt(int ns, int nr, int nm, const double *__restrict__ theta, const double *__restrict__ coef,
                          const float *__restrict__ in_scale, const float *__restrict__ scale, float *__restrict__ X,
                          float *__restrict__ T) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < (int64_t)ns * nr) X[i] = (float)(theta[i] * (double)in_scale[0]);
  if (i < (int64_t)ns * nm) T[i] = (float)(coef[i] / (double)scale[i % nm]);
}

// the permutation of 0..n-1 that sorts the keys SplitMix64(seed, epoch, i):
// every entry finds its rank by counting smaller keys (n is a few hundred)
__global__ void k_epoch_perm(int n, uint64_t seed, uint64_t epoch, int32_t *__restrict__ perm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t base = splitmix64(seed ^ splitmix64(epoch + 0x51EDull));
  const uint64_t ki = splitmix64(base + (uint64_t)i);
  int rank = 0;
  for (int j = 0; j < n; ++j) {
    const uint64_t kj = splitmix64(base + (uint64_t)j);
    rank += (kj < ki) || (kj == ki && j < i);
  }
  perm[rank] = i;
}

__global__ void k_gather_batch(int B, int nr, int nm, const int32_t *__restrict__ idx, const float *__restrict__ X,
                               const float *__restrict__ T, bf16 *__restrict__ Xb, float *__restrict__ Tb) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < (int64_t)B * nr) {
    const int b = (int)(i / nr), j = (int)(i % nr);
    Xb[i] = __float2bfloat16(X[(int64_t)idx[b] * nr + j]);
  }
  if (i < (int64_t)B * nm) {
    const int b = (int)(i / nm), j = (int)(i % nm);
    Tb[i] = T[(int64_t)idx[b] * nm + j];
  }
}

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
}

// Z (row-major, n columns) += bias; H = gelu(Z) in BF16
__global__ void k_bias_gelu(int64_t total, int n, float *__restrict__ Z, const float *__restrict__ bias,
                            bf16 *__restrict__ H) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= total) return;
  const float z = Z[i] + bias[i % n];
  Z[i] = z;
  H[i] = __float2bfloat16(gelu_f(z));
}

__global__ void k_bias_add(int64_t total, int n, float *__restrict__ Y, const float *__restrict__ bias) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < total) Y[i] += bias[i % n];
}

// dY = (Y - T) / B and per-CTA partial sums of (Y - T)^2
__global__ void k_mse(int64_t total, float invB, const float *__restrict__ Y, const float *__restrict__ T,
                      float *__restrict__ dY, float *__restrict__ part) {
  __shared__ float sh[TPB];
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float r = 0.f;
  if (i < total) {
    r = Y[i] - T[i];
    dY[i] = r * invB;
  }
  sh[threadIdx.x] = r * r;
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_gelu_bwd(int64_t total, const float *__restrict__ dH, const float *__restrict__ Z,
                           float *__restrict__ dZ) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < total) dZ[i] = dH[i] * gelu_grad_f(Z[i]);
}

// db[o] = sum_b dZ[b][o]
__global__ void k_bias_grad(int B, int n, const float *__restrict__ dZ, float *__restrict__ db) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dZ[(int64_t)b * n + o];
  db[o] = s;
}

// AdamW with decoupled weight decay; c1 = 1 - b1^t, c2 = 1 - b2^t
__global__ void k_adamw(int64_t n, float lr, float wd, float b1, float b2, float eps, float c1, float c2,
                        const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                        float *__restrict__ p, bf16 *__restrict__ p16) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
  p[i] = pi;
  p16[i] = __float2bfloat16(pi);
}

// network input of one design: Xb[0][k] = bf16(theta[k] in_scale)
__global__ void k_prep_theta(int nr, const double *__restrict__ theta, const float *__restrict__ in_scale,
                             bf16 *__restrict__ Xb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nr) Xb[k] = __float2bfloat16((float)(theta[k] * (double)in_scale[0]));
}

__global__ void k_scale_coef(int nm, const float *__restrict__ y, const float *__restrict__ scale,
                             double *__restrict__ c) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < nm) c[m] = (double)y[m] * (double)scale[m];
}

// out = X + a + b
__global__ void k_add3(int64_t n, const double *__restrict__ X, const double *__restrict__ a,
                       const double *__restrict__ b, double *__restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = X[i] + a[i] + b[i];
}

// --------------------------------------------------- host dense linear algebra
// (R x R problems of the randomised SVD; R = n_modes + 32)

// Cholesky G = R^T R, R upper triangular, in place (row-major n x n);
// false if G is not numerically positive definite
bool cholesky_upper(std::vector<double> &G, int n) {
  for (int j = 0; j < n; ++j) {
    double s = G[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= G[(size_t)k * n + j] * G[(size_t)k * n + j];
    if (!(s > 0.0)) return false;
    const double r = std::sqrt(s);
    G[(size_t)j * n + j] = r;
    for (int i = j + 1; i < n; ++i) {
      double t = G[(size_t)j * n + i];
      for (int k = 0; k < j; ++k) t -= G[(size_t)k * n + j] * G[(size_t)k * n + i];
      G[(size_t)j * n + i] = t / r;
    }
    for (int i = 0; i < j; ++i) G[(size_t)j * n + i] = 0.0;
  }
  return true;
}

// R^{-1} of an upper-triangular R (row-major), by back substitution
std::vector<double> upper_inverse(const std::vector<double> &R, int n) {
  std::vector<double> X((size_t)n * n, 0.0);
  for (int c = 0; c < n; ++c)
    for (int i = c; i >= 0; --i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = i + 1; k <= c; ++k) s -= R[(size_t)i * n + k] * X[(size_t)k * n + c];
      X[(size_t)i * n + c] = s / R[(size_t)i * n + i];
    }
  return X;
}

// cyclic Jacobi eigensolver (Golub & Van Loan, Sec. 8.5) of a symmetric
// n x n matrix (row-major): eigenvalues w descending, eigenvectors as the
// columns of V (row-major)
void jacobi_eig(std::vector<double> A, int n, std::vector<double> &w, std::vector<double> &V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double a = A[(size_t)i * n + j];
        tot += a * a;
        if (i != j) off += a * a;
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J^T A
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // V <- V J
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return A[(size_t)a * n + a] > A[(size_t)b * n + b]; });
  w.resize(n);
  std::vector<double> V2((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = A[(size_t)ord[j] * n + ord[j]];
    for (int i = 0; i < n; ++i) V2[(size_t)i * n + j] = V[(size_t)i * n + ord[j]];
  }
  V.swap(V2);
}

}  // namespace

struct sgn_learn_ctx {
  sgn_ctx *h = nullptr;
  int n_rbf = 0, n_modes = 0, hidden = 0, max_snap = 0, batch = 0, R = 0;
  int dim = 0, n_nodes = 0, n_elem = 0;
  int64_t n_dof = 0;
  double width = 0.0;
  std::vector<double> centers, centroids;
  std::vector<int32_t> h_fan;
  int64_t n_params = 0, off[6] = {0, 0, 0, 0, 0, 0};
  int64_t ws_elems = 0;
  bool bound = false, have_basis = false, have_scales = false;
  int64_t adam_t = 0;
  std::vector<double> sigma;
  // device (carved from the caller's buffer)
  double *ctr = nullptr, *cent = nullptr, *phi = nullptr, *Xd = nullptr, *mean = nullptr, *basis = nullptr;
  double *Y = nullptr, *Y2 = nullptr, *Om = nullptr, *Zs = nullptr, *small = nullptr;
  double *vec = nullptr, *ws = nullptr, *coef = nullptr, *cvec = nullptr, *disp = nullptr, *xa = nullptr;
  double *pbuf = nullptr;
  float *Xall = nullptr, *Tall = nullptr, *coef_scale = nullptr, *in_scale = nullptr;
  float *p32 = nullptr, *g32 = nullptr, *am = nullptr, *av = nullptr;
  bf16 *p16 = nullptr;
  int32_t *fan_in = nullptr, *idx = nullptr;
  bf16 *Xb = nullptr, *H1 = nullptr, *H2 = nullptr;
  float *Tb = nullptr, *Z1 = nullptr, *Z2 = nullptr, *Yb = nullptr, *dY = nullptr, *dH = nullptr, *dZ = nullptr;
  float *part = nullptr;
  bf16 *gA = nullptr, *gB = nullptr;  // packed K-major operands of the tensor-core GEMMs
  int64_t g_elems = 0;                // elements of each
};

namespace {

struct Carve {
  char *base;
  size_t off = 0;
  template <typename T>
  T *take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += std::max<size_t>(n, 1) * sizeof(T);
    return p;
  }
};

size_t carve_learn(sgn_learn_ctx &L, char *base) {
  Carve c{base};
  const size_t nd = (size_t)L.n_dof, ne = (size_t)L.n_elem, R = (size_t)L.R, ms = (size_t)L.max_snap;
  const size_t nm = (size_t)L.n_modes, nr = (size_t)L.n_rbf, B = (size_t)L.batch, H = (size_t)L.hidden;
  L.ctr = c.take<double>(nr * L.dim);
  L.cent = c.take<double>(ne * L.dim);
  L.phi = c.take<double>(ne * nr);
  L.Xd = c.take<double>(nd);
  L.mean = c.take<double>(nd);
  L.basis = c.take<double>(nd * nm);
  L.Y = c.take<double>(nd * R);
  L.Y2 = c.take<double>(nd * R);
  L.Om = c.take<double>(ms * R);
  L.Zs = c.take<double>(ms * R);
  L.small = c.take<double>(R * R);
  L.vec = c.take<double>(std::max({R, ms, nm}));
  L.ws = c.take<double>((size_t)L.ws_elems);
  L.coef = c.take<double>(ms * nm);
  L.cvec = c.take<double>(nm);
  L.disp = c.take<double>(nd);
  L.xa = c.take<double>(nd);
  L.pbuf = c.take<double>(ne);
  L.Xall = c.take<float>(ms * nr);
  L.Tall = c.take<float>(ms * nm);
  L.coef_scale = c.take<float>(nm);
  L.in_scale = c.take<float>(1);
  L.p32 = c.take<float>((size_t)L.n_params);
  L.g32 = c.take<float>((size_t)L.n_params);
  L.am = c.take<float>((size_t)L.n_params);
  L.av = c.take<float>((size_t)L.n_params);
  L.p16 = c.take<bf16>((size_t)L.n_params);
  L.fan_in = c.take<int32_t>((size_t)L.n_params);
  L.idx = c.take<int32_t>(ms);
  {
    const size_t D = std::max({B, nm, H, nr});
    L.g_elems = (int64_t)(((D + 127) / 128) * 128 * ((D + 63) / 64) * 64);
    L.gA = c.take<bf16>((size_t)L.g_elems);
    L.gB = c.take<bf16>((size_t)L.g_elems);
  }
  L.Xb = c.take<bf16>(B * nr);
  L.Tb = c.take<float>(B * nm);
  L.Z1 = c.take<float>(B * H);
  L.H1 = c.take<bf16>(B * H);
  L.Z2 = c.take<float>(B * H);
  L.H2 = c.take<bf16>(B * H);
  L.Yb = c.take<float>(B * nm);
  L.dY = c.take<float>(B * nm);
  L.dH = c.take<float>(B * H);
  L.dZ = c.take<float>(B * H);
  L.part = c.take<float>(nblk((int64_t)(B * nm)));
  return c.off + 256;
}

sgn_status fail(sgn_learn_ctx &L, const char *what) {
  cudaError_t e = cudaGetLastError();
  L.h->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return SGN_ECUDA;
}
sgn_status check(sgn_learn_ctx &L, const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) return SGN_OK;
  L.h->last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return SGN_ECUDA;
}

// ---- randomised SVD pieces; A is the snapshot matrix, column-major n_dof x ns
// Yout (column-major n_dof x r) = (A - mean 1^T) W for W column-major ns x r
void apply_Ac(sgn_learn_ctx &L, const double *A, int ns, const double *W, int r, double *Yout) {
  Ctx &c = *L.h;
  const int64_t nd = L.n_dof;
  gemm<double, double, double, double>(c, (int)nd, r, ns, 1.0, A, 1, nd, W, 1, ns, 0.0, Yout, 1, nd);
  k_colsum<<<nblk(r), TPB, 0, c.stream>>>(ns, r, W, L.vec);
  k_rank1_sub<<<nblk(nd * r), TPB, 0, c.stream>>>((int)nd, r, L.mean, L.vec, Yout, 1, nd);
  c.count(2);
}

// Zout (column-major ns x r) = (A - mean 1^T)^T Q for Q column-major n_dof x r
void apply_AcT(sgn_learn_ctx &L, const double *A, int ns, const double *Q, int r, double *Zout) {
  Ctx &c = *L.h;
  const int64_t nd = L.n_dof;
  gemm<double, double, double, double>(c, ns, r, (int)nd, 1.0, A, nd, 1, Q, 1, nd, 0.0, Zout, 1, ns, L.ws,
                                       L.ws_elems);
  gemm<double, double, double, double>(c, 1, r, (int)nd, 1.0, L.mean, 0, 1, Q, 1, nd, 0.0, L.vec, 0, 1, L.ws,
                                       L.ws_elems);
  k_rank1_sub<<<nblk((int64_t)ns * r), TPB, 0, c.stream>>>(ns, r, nullptr, L.vec, Zout, 1, ns);
  c.count();
}

// G (r x r, host) = M^T M for M column-major rows x r
bool gram(sgn_learn_ctx &L, const double *M, int64_t rows, int r, std::vector<double> &G) {
  Ctx &c = *L.h;
  gemm<double, double, double, double>(c, r, r, (int)rows, 1.0, M, rows, 1, M, 1, rows, 0.0, L.small, r, 1, L.ws,
                                       L.ws_elems);
  G.resize((size_t)r * r);
  if (cudaMemcpyAsync(G.data(), L.small, G.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream) !=
      cudaSuccess)
    return false;
  return cudaStreamSynchronize(c.stream) == cudaSuccess;
}

// Orthonormal basis of range(M) for M column-major rows x r, left in M
// (scratch: rows x r).  Pass 1: eigen-decomposition G = M^T M = V diag(l) V^T,
// Q = M V_k l_k^{-1/2} over the k eigenvalues above 1e-14 l_max (directions
// of relative size below 1e-7 are beyond what one FP64 pass can
// orthogonalise and are dropped); pass 2: Cholesky-QR of Q restores
// orthogonality to working precision.  Returns k (0 for M = 0, -1 on failure).
int orthonormalise(sgn_learn_ctx &L, double *M, int64_t rows, int r, double *scratch) {
  Ctx &c = *L.h;
  std::vector<double> G, w, V;
  if (!gram(L, M, rows, r, G)) return -1;
  jacobi_eig(G, r, w, V);
  if (!(w[0] > 0.0)) return 0;
  int k = 0;
  while (k < r && w[k] > 1e-14 * w[0]) ++k;
  std::vector<double> T((size_t)r * k);
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < k; ++j) T[(size_t)i * k + j] = V[(size_t)i * r + j] / std::sqrt(w[j]);
  if (cudaMemcpyAsync(L.small, T.data(), T.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream) !=
      cudaSuccess)
    return -1;
  gemm<double, double, double, double>(c, (int)rows, k, r, 1.0, M, 1, rows, L.small, k, 1, 0.0, scratch, 1, rows);
  if (!gram(L, scratch, rows, k, G)) return -1;
  if (!cholesky_upper(G, k)) return -1;
  std::vector<double> Ri = upper_inverse(G, k);
  if (cudaMemcpyAsync(L.small, Ri.data(), Ri.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream) !=
      cudaSuccess)
    return -1;
  gemm<double, double, double, double>(c, (int)rows, k, k, 1.0, scratch, 1, rows, L.small, k, 1, 0.0, M, 1, rows);
  return k;
}

// ---- MLP
// forward of the B rows in Xb; Yb receives the (normalised) outputs
typedef CUresult (*EncodeTiledFnL)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// TMA map of a packed [rows][kp] BF16 operand, box 64 (K) x box_rows, 128B swizzle
bool encode_bf16(CUtensorMap *m, void *addr, int kp, int rows, int box_rows) {
  static EncodeTiledFnL enc = nullptr;
  if (!enc) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return false;
    enc = (EncodeTiledFnL)fn;
  }
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)GK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, addr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C(m, n) = alpha sum_k A(m, k) B(k, n) + beta C(m, n) on the tensor cores
// (same operand convention as gemm above; A and B converted to BF16)
template <typename TA, typename TB>
void gemm_tc(sgn_learn_ctx &L, int M, int N, int K, float alpha, const TA *A, int64_t sam, int64_t sak, const TB *B,
             int64_t sbk, int64_t sbn, float beta, float *C, int64_t scm, int64_t scn) {
  Ctx &c = *L.h;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm_bf16_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, GSMEM);
    attr = true;
  }
  const int Mp = ((M + GM - 1) / GM) * GM, Np = ((N + GN - 1) / GN) * GN, Kp = ((K + GK - 1) / GK) * GK;
  if ((int64_t)Mp * Kp > L.g_elems || (int64_t)Np * Kp > L.g_elems) {
    c.last_error = "tensor-core GEMM operands exceed their packing buffers";
    return;
  }
  k_pack_bf16<TA><<<nblk((int64_t)Mp * Kp), TPB, 0, c.stream>>>(M, K, A, sam, sak, L.gA, Mp, Kp);
  k_pack_bf16<TB><<<nblk((int64_t)Np * Kp), TPB, 0, c.stream>>>(N, K, B, sbn, sbk, L.gB, Np, Kp);
  CUtensorMap ma, mb;
  if (!encode_bf16(&ma, L.gA, Kp, Mp, GM) || !encode_bf16(&mb, L.gB, Kp, Np, GN)) {
    c.last_error = "cuTensorMapEncodeTiled failed for a GEMM operand";
    return;
  }
  k_gemm_bf16_tc<<<dim3(Np / GN, Mp / GM), 128, GSMEM, c.stream>>>(ma, mb, M, N, Kp / GK, alpha, beta, C, scm, scn,
                                                                    c.status);
  c.count(3);
}

void mlp_forward(sgn_learn_ctx &L, int B) {
  Ctx &c = *L.h;
  const int H = L.hidden, nr = L.n_rbf, nm = L.n_modes;
  const bf16 *W1 = L.p16 + L.off[0], *W2 = L.p16 + L.off[2], *W3 = L.p16 + L.off[4];
  const int64_t bh = (int64_t)B * H, bm = (int64_t)B * nm;
  // Z1[b][o] = sum_i X[b][i] W1[o][i]
  gemm_tc<bf16, bf16>(L, B, H, nr, 1.f, L.Xb, nr, 1, W1, 1, nr, 0.f, L.Z1, H, 1);
  k_bias_gelu<<<nblk(bh), TPB, 0, c.stream>>>(bh, H, L.Z1, L.p32 + L.off[1], L.H1);
  gemm_tc<bf16, bf16>(L, B, H, H, 1.f, L.H1, H, 1, W2, 1, H, 0.f, L.Z2, H, 1);
  k_bias_gelu<<<nblk(bh), TPB, 0, c.stream>>>(bh, H, L.Z2, L.p32 + L.off[3], L.H2);
  gemm_tc<bf16, bf16>(L, B, nm, H, 1.f, L.H2, H, 1, W3, 1, H, 0.f, L.Yb, nm, 1);
  k_bias_add<<<nblk(bm), TPB, 0, c.stream>>>(bm, nm, L.Yb, L.p32 + L.off[5]);
  c.count(3);
}

// forward, loss L = 1/(2B) sum ||Y - T||^2 (partial sums in L.part) and its
// parameter gradients into g32, for the batch in (Xb, Tb)
void mlp_backward(sgn_learn_ctx &L, int B) {
  Ctx &c = *L.h;
  const int H = L.hidden, nr = L.n_rbf, nm = L.n_modes;
  mlp_forward(L, B);
  const int64_t bm = (int64_t)B * nm, bh = (int64_t)B * H;
  k_mse<<<nblk(bm), TPB, 0, c.stream>>>(bm, 1.f / B, L.Yb, L.Tb, L.dY, L.part);
  const bf16 *W2 = L.p16 + L.off[2], *W3 = L.p16 + L.off[4];
  float *g = L.g32;
  // output layer: dW3 = dY^T H2, db3 = column sums of dY, dH2 = dY W3
  gemm_tc<float, bf16>(L, nm, H, B, 1.f, L.dY, 1, nm, L.H2, H, 1, 0.f, g + L.off[4], H, 1);
  k_bias_grad<<<nblk(nm), TPB, 0, c.stream>>>(B, nm, L.dY, g + L.off[5]);
  gemm_tc<float, bf16>(L, B, H, nm, 1.f, L.dY, nm, 1, W3, H, 1, 0.f, L.dH, H, 1);
  k_gelu_bwd<<<nblk(bh), TPB, 0, c.stream>>>(bh, L.dH, L.Z2, L.dZ);
  // hidden layer 2
  gemm_tc<float, bf16>(L, H, H, B, 1.f, L.dZ, 1, H, L.H1, H, 1, 0.f, g + L.off[2], H, 1);
  k_bias_grad<<<nblk(H), TPB, 0, c.stream>>>(B, H, L.dZ, g + L.off[3]);
  gemm_tc<float, bf16>(L, B, H, H, 1.f, L.dZ, H, 1, W2, H, 1, 0.f, L.dH, H, 1);
  k_gelu_bwd<<<nblk(bh), TPB, 0, c.stream>>>(bh, L.dH, L.Z1, L.dZ);
  // hidden layer 1
  gemm_tc<float, bf16>(L, H, nr, B, 1.f, L.dZ, 1, H, L.Xb, nr, 1, 0.f, g + L.off[0], nr, 1);
  k_bias_grad<<<nblk(H), TPB, 0, c.stream>>>(B, H, L.dZ, g + L.off[1]);
  c.count(6);
}

void adamw(sgn_learn_ctx &L, float lr, float wd) {
  Ctx &c = *L.h;
  ++L.adam_t;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 - std::pow(b1, (double)L.adam_t));
  const float c2 = (float)(1.0 - std::pow(b2, (double)L.adam_t));
  k_adamw<<<nblk(L.n_params), TPB, 0, c.stream>>>(L.n_params, lr, wd, (float)b1, (float)b2, 1e-8f, c1, c2, L.g32,
                                                  L.am, L.av, L.p32, L.p16);
  c.count();
}

// x (node-major) = X + u_bar + U (scale * MLP(theta * in_scale))
void predict_into(sgn_learn_ctx &L, const double *theta_d, double *x) {
  Ctx &c = *L.h;
  const int64_t nd = L.n_dof;
  k_prep_theta<<<nblk(L.n_rbf), TPB, 0, c.stream>>>(L.n_rbf, theta_d, L.in_scale, L.Xb);
  c.count();
  mlp_forward(L, 1);
  k_scale_coef<<<nblk(L.n_modes), TPB, 0, c.stream>>>(L.n_modes, L.Yb, L.coef_scale, L.cvec);
  c.count();
  gemm<double, double, double, double>(c, (int)nd, 1, L.n_modes, 1.0, L.basis, 1, nd, L.cvec, 1, 1, 0.0, L.disp, 1,
                                       1);
  k_add3<<<nblk(nd), TPB, 0, c.stream>>>(nd, L.Xd, L.mean, L.disp, x);
  c.count();
}

// ||f_int(x) - f_ext|| / ||f_ext|| at (x, p); +inf if x inverts an element
double start_residual(sgn_learn_ctx &L, const double *x, const double *p, const double *fext) {
  Ctx &c = *L.h;
  const int64_t nx = (int64_t)c.S.n_free * c.S.dim;
  const int nbk = sgn::energy_blocks(c);
  sgn::launch_energy_partials(c, x, p, c.partial, nbk);
  std::vector<double> hp(nbk);
  cudaMemcpyAsync(hp.data(), c.partial, nbk * sizeof(double), cudaMemcpyDeviceToHost, c.stream);
  cudaStreamSynchronize(c.stream);
  double e = 0.0;
  for (double v : hp) e += v;
  if (!std::isfinite(e)) return INFINITY;
  double *fr = c.eq, *cr = c.eq + nx;
  sgn::launch_from_nodes(c, fext, fr);
  const double fn = std::sqrt(sgn::device_sumsq3(c, fr, nx, nullptr, 0, nullptr, 0));
  sgn::launch_elem_state(c, x, p);
  sgn::launch_internal_force(c, cr);
  sgn::launch_axpy(c, cr, fr, -1.0, nx);
  const double cn = std::sqrt(sgn::device_sumsq3(c, cr, nx, nullptr, 0, nullptr, 0));
  return cn / (fn > 0 ? fn : 1.0);
}

}  // namespace

extern "C" {

sgn_status sgn_learn_create(sgn_t h, const sgn_learn_opts *o, sgn_learn_t *out) {
  if (!h || !o || !out || !o->centers_h || o->n_rbf <= 0 || o->n_modes <= 0 || o->hidden <= 0 || o->max_snap <= 1 ||
      o->batch <= 0 || o->batch > o->max_snap || !(o->width > 0.0))
    return SGN_EINVAL;
  if (!h->bound) return SGN_ESTATE;
  const auto &S = h->S;
  const int64_t nd = (int64_t)S.n_nodes * S.dim;
  if (nd > INT32_MAX || o->n_modes > o->max_snap || o->n_modes > nd) return SGN_EINVAL;
  sgn_learn_ctx *L = new (std::nothrow) sgn_learn_ctx();
  if (!L) return SGN_ENOMEM;
  L->h = h;
  L->dim = S.dim;
  L->n_nodes = S.n_nodes;
  L->n_elem = S.n_elem;
  L->n_dof = nd;
  L->n_rbf = o->n_rbf;
  L->n_modes = o->n_modes;
  L->hidden = o->hidden;
  L->max_snap = o->max_snap;
  L->batch = o->batch;
  L->width = o->width;
  L->R = (int)std::min<int64_t>({(int64_t)o->n_modes + 32, (int64_t)o->max_snap, nd});
  L->ws_elems = 64 * (int64_t)std::max(L->R, o->n_modes) * std::max(L->R, o->max_snap);
  L->centers.assign(o->centers_h, o->centers_h + (size_t)o->n_rbf * S.dim);
  L->centroids.assign((size_t)S.n_elem * S.dim, 0.0);
  const int nv = S.dim + 1;
  for (int e = 0; e < S.n_elem; ++e)
    for (int a = 0; a < nv; ++a) {
      const int v = S.elem_node[(size_t)a * S.n_elem + e];
      for (int i = 0; i < S.dim; ++i) L->centroids[(size_t)e * S.dim + i] += S.X[(size_t)v * S.dim + i] / nv;
    }
  const int64_t H = o->hidden, nr = o->n_rbf, nm = o->n_modes;
  L->off[0] = 0;                   // W1 [H][nr]
  L->off[1] = L->off[0] + H * nr;  // b1 [H]
  L->off[2] = L->off[1] + H;       // W2 [H][H]
  L->off[3] = L->off[2] + H * H;   // b2 [H]
  L->off[4] = L->off[3] + H;       // W3 [nm][H]
  L->off[5] = L->off[4] + nm * H;  // b3 [nm]
  L->n_params = L->off[5] + nm;
  L->h_fan.assign((size_t)L->n_params, 0);
  std::fill(L->h_fan.begin() + L->off[0], L->h_fan.begin() + L->off[1], (int32_t)nr);
  std::fill(L->h_fan.begin() + L->off[2], L->h_fan.begin() + L->off[3], (int32_t)H);
  std::fill(L->h_fan.begin() + L->off[4], L->h_fan.begin() + L->off[5], (int32_t)H);
  *out = L;
  return SGN_OK;
}

sgn_status sgn_learn_device_bytes(sgn_learn_t L, size_t *bytes) {
  if (!L || !bytes) return SGN_EINVAL;
  *bytes = carve_learn(*L, nullptr);
  return SGN_OK;
}

sgn_status sgn_learn_bind(sgn_learn_t L, void *dev, size_t bytes) {
  if (!L || !dev || ((uintptr_t)dev & 255)) return SGN_EINVAL;
  if (bytes < carve_learn(*L, nullptr)) return SGN_ENOMEM;
  carve_learn(*L, (char *)dev);
  Ctx &c = *L->h;
  const auto &S = c.S;
  if (cudaMemcpyAsync(L->ctr, L->centers.data(), L->centers.size() * 8, cudaMemcpyHostToDevice, c.stream) ||
      cudaMemcpyAsync(L->cent, L->centroids.data(), L->centroids.size() * 8, cudaMemcpyHostToDevice, c.stream) ||
      cudaMemcpyAsync(L->Xd, S.X.data(), S.X.size() * 8, cudaMemcpyHostToDevice, c.stream) ||
      cudaMemcpyAsync(L->fan_in, L->h_fan.data(), L->h_fan.size() * 4, cudaMemcpyHostToDevice, c.stream) ||
      cudaMemsetAsync(L->mean, 0, (size_t)L->n_dof * 8, c.stream) ||
      cudaMemsetAsync(L->basis, 0, (size_t)L->n_dof * L->n_modes * 8, c.stream))
    return fail(*L, "sgn_learn_bind upload");
  k_phi<<<nblk((int64_t)L->n_elem * L->n_rbf), TPB, 0, c.stream>>>(L->n_elem, L->n_rbf, L->dim, L->cent, L->ctr,
                                                                   1.0 / (2.0 * L->width * L->width), L->phi);
  k_init_params<<<nblk(L->n_params), TPB, 0, c.stream>>>(L->n_params, L->fan_in, 0x5EEDull, L->p32, L->p16, L->am,
                                                         L->av);
  c.count(2);
  const float one = 1.f;
  std::vector<float> ones((size_t)L->n_modes, 1.f);
  if (cudaMemcpyAsync(L->in_scale, &one, sizeof(float), cudaMemcpyHostToDevice, c.stream) ||
      cudaMemcpyAsync(L->coef_scale, ones.data(), ones.size() * sizeof(float), cudaMemcpyHostToDevice, c.stream) ||
      cudaStreamSynchronize(c.stream))
    return fail(*L, "sgn_learn_bind");
  sgn_status s = check(*L, "sgn_learn_bind");
  if (s != SGN_OK) return s;
  L->adam_t = 0;
  L->bound = true;
  return SGN_OK;
}

void sgn_learn_destroy(sgn_learn_t L) { delete L; }

int64_t sgn_learn_param_count(sgn_learn_t L) { return L ? L->n_params : -1; }

sgn_status sgn_rbf_params(sgn_learn_t L, const double *theta_d, double *p_d) {
  if (!L || !theta_d || !p_d) return SGN_EINVAL;
  if (!L->bound) return SGN_ESTATE;
  // p[e] = sum_k Phi[e][k] theta[k]
  gemm<double, double, double, double>(*L->h, L->n_elem, 1, L->n_rbf, 1.0, L->phi, L->n_rbf, 1, theta_d, 1, 1, 0.0,
                                       p_d, 1, 1);
  return check(*L, "sgn_rbf_params");
}

sgn_status sgn_learn_basis(sgn_learn_t L, const double *A, int32_t ns, uint64_t seed, double *sigma_h) {
  if (!L || !A || ns < 2 || ns > L->max_snap) return SGN_EINVAL;
  if (!L->bound) return SGN_ESTATE;
  Ctx &c = *L->h;
  const int64_t nd = L->n_dof;
  const int nm = L->n_modes;
  const int R = std::min(L->R, (int)ns);
  L->have_basis = false;
  L->have_scales = false;
  // the centred snapshot matrix A_c = A - mean 1^T is never formed
  k_rowmean<<<nblk(nd), TPB, 0, c.stream>>>(nd, ns, A, L->mean);
  k_gauss<<<nblk((int64_t)ns * R), TPB, 0, c.stream>>>((int64_t)ns * R, seed, L->Om);
  c.count(2);
  // range finder with one power iteration, re-orthonormalised after every
  // product so that no step sees the squared spectrum:
  // Q = orth(A_c orth(A_c^T orth(A_c Omega)))
  apply_Ac(*L, A, ns, L->Om, R, L->Y);
  int r = orthonormalise(*L, L->Y, nd, R, L->Y2);
  if (r > 0) {
    apply_AcT(*L, A, ns, L->Y, r, L->Zs);
    r = orthonormalise(*L, L->Zs, ns, r, L->Om);  // Omega is no longer needed
  }
  if (r > 0) {
    apply_Ac(*L, A, ns, L->Zs, r, L->Y);
    r = orthonormalise(*L, L->Y, nd, r, L->Y2);
  }
  if (r < 0) {
    c.last_error = "sgn_learn_basis: orthonormalisation failed";
    return SGN_ENONFINITE;
  }
  std::vector<double> w;
  if (cudaMemsetAsync(L->basis, 0, (size_t)nd * nm * 8, c.stream)) return fail(*L, "sgn_learn_basis");
  if (r > 0) {
    // B = Q^T A_c (r x ns); S = B B^T = V diag(sigma^2) V^T; U = Q V
    apply_AcT(*L, A, ns, L->Y, r, L->Zs);  // Zs = B^T, column-major ns x r
    gemm<double, double, double, double>(c, r, r, ns, 1.0, L->Zs, ns, 1, L->Zs, 1, ns, 0.0, L->small, r, 1, L->ws,
                                         L->ws_elems);
    std::vector<double> S((size_t)r * r), V;
    if (cudaMemcpyAsync(S.data(), L->small, S.size() * 8, cudaMemcpyDeviceToHost, c.stream) ||
        cudaStreamSynchronize(c.stream))
      return fail(*L, "sgn_learn_basis");
    jacobi_eig(S, r, w, V);
    // U = Q V[:, :k], k = min(r, n_modes); columns past k stay zero
    const int k = std::min(r, nm);
    std::vector<double> Vk((size_t)r * k);
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < k; ++j) Vk[(size_t)i * k + j] = V[(size_t)i * r + j];
    if (cudaMemcpyAsync(L->small, Vk.data(), Vk.size() * 8, cudaMemcpyHostToDevice, c.stream))
      return fail(*L, "sgn_learn_basis");
    gemm<double, double, double, double>(c, (int)nd, k, r, 1.0, L->Y, 1, nd, L->small, k, 1, 0.0, L->basis, 1, nd);
  }
  L->sigma.assign((size_t)nm, 0.0);
  for (int j = 0; j < std::min(r, nm); ++j) L->sigma[j] = std::sqrt(std::max(w[j], 0.0));
  if (sigma_h) std::copy(L->sigma.begin(), L->sigma.end(), sigma_h);
  if (cudaStreamSynchronize(c.stream)) return fail(*L, "sgn_learn_basis");
  sgn_status s = check(*L, "sgn_learn_basis");
  if (s != SGN_OK) return s;
  L->have_basis = true;
  return SGN_OK;
}

sgn_status sgn_learn_train(sgn_learn_t L, const double *thetas_d, const double *A, int32_t ns, int32_t steps,
                           float lr, float wd, uint64_t seed, float *final_loss_h) {
  if (!L || !thetas_d || !A || ns < 1 || ns > L->max_snap || steps < 0 || !(lr >= 0.f) || !(wd >= 0.f))
    return SGN_EINVAL;
  if (!L->bound || !L->have_basis) return SGN_ESTATE;
  Ctx &c = *L->h;
  const int64_t nd = L->n_dof;
  const int nm = L->n_modes, nr = L->n_rbf;
  // targets: coef[s][m] = U[:, m]^T (A[:, s] - mean), normalised per mode by its rms
  gemm<double, double, double, double>(c, ns, nm, (int)nd, 1.0, A, nd, 1, L->basis, 1, nd, 0.0, L->coef, nm, 1,
                                       L->ws, L->ws_elems);
  gemm<double, double, double, double>(c, 1, nm, (int)nd, 1.0, L->mean, 0, 1, L->basis, 1, nd, 0.0, L->vec, 0, 1,
                                       L->ws, L->ws_elems);
  k_rank1_sub<<<nblk((int64_t)ns * nm), TPB, 0, c.stream>>>(ns, nm, nullptr, L->vec, L->coef, nm, 1);
  k_col_rms<<<nblk(nm), TPB, 0, c.stream>>>(ns, nm, L->coef, L->coef_scale);
  k_inv_rms<<<1, TPB, 0, c.stream>>>((int64_t)ns * nr, thetas_d, L->in_scale);
  k_prep_xt<<<nblk((int64_t)ns * std::max(nr, nm)), TPB, 0, c.stream>>>(ns, nr, nm, thetas_d, L->coef, L->in_scale,
                                                                         L->coef_scale, L->Xall, L->Tall);
  c.count(4);
  L->have_scales = true;
  const int Bt = std::min(L->batch, (int)ns);
  const int nbat = ns / Bt;
  for (int st = 0; st < steps; ++st) {
    const int j = st % nbat;
    if (j == 0) {
      k_epoch_perm<<<nblk(ns), TPB, 0, c.stream>>>(ns, seed, (uint64_t)(st / nbat), L->idx);
      c.count();
    }
    k_gather_batch<<<nblk((int64_t)Bt * std::max(nr, nm)), TPB, 0, c.stream>>>(Bt, nr, nm, L->idx + (int64_t)j * Bt,
                                                                               L->Xall, L->Tall, L->Xb, L->Tb);
    c.count();
    mlp_backward(*L, Bt);
    adamw(*L, lr, wd);
  }
  if (final_loss_h) {
    if (steps == 0) {
      *final_loss_h = NAN;
    } else {
      const int nb = (int)nblk((int64_t)Bt * nm);
      std::vector<float> part((size_t)nb);
      if (cudaMemcpyAsync(part.data(), L->part, nb * sizeof(float), cudaMemcpyDeviceToHost, c.stream) ||
          cudaStreamSynchronize(c.stream))
        return fail(*L, "sgn_learn_train");
      double s = 0.0;
      for (float v : part) s += v;
      *final_loss_h = (float)(s / ((double)Bt * nm));
    }
  }
  if (cudaStreamSynchronize(c.stream)) return fail(*L, "sgn_learn_train");
  return check(*L, "sgn_learn_train");
}

sgn_status sgn_learn_predict(sgn_learn_t L, const double *theta_d, double *x0_d) {
  if (!L || !theta_d || !x0_d) return SGN_EINVAL;
  if (!L->bound || !L->have_basis || !L->have_scales) return SGN_ESTATE;
  predict_into(*L, theta_d, x0_d);
  return check(*L, "sgn_learn_predict");
}

sgn_status sgn_equilibrium_warm(sgn_learn_t L, const double *theta_d, const double *fext_d, const double *x_prev_d,
                                double *x_d, const sgn_newton_opts *opts, sgn_newton_report *rep,
                                int32_t *used_warm_start) {
  if (!L || !theta_d || !fext_d || !x_d) return SGN_EINVAL;
  if (!L->bound || !L->have_basis || !L->have_scales) return SGN_ESTATE;
  Ctx &c = *L->h;
  const int64_t nd = L->n_dof;
  sgn_status s = sgn_rbf_params(L, theta_d, L->pbuf);
  if (s != SGN_OK) return s;
  predict_into(*L, theta_d, L->xa);
  const double r_warm = start_residual(*L, L->xa, L->pbuf, fext_d);
  const double *other = x_prev_d ? x_prev_d : L->Xd;
  const double r_other = start_residual(*L, other, L->pbuf, fext_d);
  const bool warm = r_warm <= r_other;
  const double *start = warm ? L->xa : other;
  if (start != x_d && cudaMemcpyAsync(x_d, start, (size_t)nd * sizeof(double), cudaMemcpyDeviceToDevice, c.stream))
    return fail(*L, "sgn_equilibrium_warm");
  if (used_warm_start) *used_warm_start = warm ? 1 : 0;
  s = check(*L, "sgn_equilibrium_warm");
  if (s != SGN_OK) return s;
  return sgn_equilibrium(L->h, L->pbuf, fext_d, x_d, opts, rep);
}

sgn_status sgn_learn_params(sgn_learn_t L, float *params_h, int32_t set) {
  if (!L || !params_h) return SGN_EINVAL;
  if (!L->bound) return SGN_ESTATE;
  Ctx &c = *L->h;
  const size_t bytes = (size_t)L->n_params * sizeof(float);
  if (set) {
    if (cudaMemcpyAsync(L->p32, params_h, bytes, cudaMemcpyHostToDevice, c.stream) ||
        cudaMemsetAsync(L->am, 0, bytes, c.stream) || cudaMemsetAsync(L->av, 0, bytes, c.stream))
      return fail(*L, "sgn_learn_params");
    k_to_bf16<<<nblk(L->n_params), TPB, 0, c.stream>>>(L->n_params, L->p32, L->p16);
    c.count();
    L->adam_t = 0;
  } else if (cudaMemcpyAsync(params_h, L->p32, bytes, cudaMemcpyDeviceToHost, c.stream)) {
    return fail(*L, "sgn_learn_params");
  }
  if (cudaStreamSynchronize(c.stream)) return fail(*L, "sgn_learn_params");
  return check(*L, "sgn_learn_params");
}

sgn_status sgn_learn_grads(sgn_learn_t L, const float *x_h, const float *t_h, int32_t n, float *loss_h,
                           float *grads_h) {
  if (!L || !x_h || !t_h || n < 1 || n > L->batch) return SGN_EINVAL;
  if (!L->bound) return SGN_ESTATE;
  Ctx &c = *L->h;
  const int nr = L->n_rbf, nm = L->n_modes;
  std::vector<int32_t> iota((size_t)n);
  std::iota(iota.begin(), iota.end(), 0);
  if (cudaMemcpyAsync(L->Xall, x_h, (size_t)n * nr * sizeof(float), cudaMemcpyHostToDevice, c.stream) ||
      cudaMemcpyAsync(L->Tall, t_h, (size_t)n * nm * sizeof(float), cudaMemcpyHostToDevice, c.stream) ||
      cudaMemcpyAsync(L->idx, iota.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream))
    return fail(*L, "sgn_learn_grads");
  k_gather_batch<<<nblk((int64_t)n * std::max(nr, nm)), TPB, 0, c.stream>>>(n, nr, nm, L->idx, L->Xall, L->Tall,
                                                                            L->Xb, L->Tb);
  c.count();
  mlp_backward(*L, n);
  const int nb = (int)nblk((int64_t)n * nm);
  std::vector<float> part((size_t)nb);
  if (cudaMemcpyAsync(part.data(), L->part, nb * sizeof(float), cudaMemcpyDeviceToHost, c.stream) ||
      (grads_h &&
       cudaMemcpyAsync(grads_h, L->g32, (size_t)L->n_params * sizeof(float), cudaMemcpyDeviceToHost, c.stream)) ||
      cudaStreamSynchronize(c.stream))
    return fail(*L, "sgn_learn_grads");
  double s = 0.0;
  for (float v : part) s += v;
  if (loss_h) *loss_h = (float)(0.5 * s / n);
  return check(*L, "sgn_learn_grads");
}

sgn_status sgn_learn_apply(sgn_learn_t L, const float *grads_h, float lr, float wd) {
  if (!L || !grads_h || !(lr >= 0.f) || !(wd >= 0.f)) return SGN_EINVAL;
  if (!L->bound) return SGN_ESTATE;
  Ctx &c = *L->h;
  if (cudaMemcpyAsync(L->g32, grads_h, (size_t)L->n_params * sizeof(float), cudaMemcpyHostToDevice, c.stream))
    return fail(*L, "sgn_learn_apply");
  adamw(*L, lr, wd);
  if (cudaStreamSynchronize(c.stream)) return fail(*L, "sgn_learn_apply");
  return check(*L, "sgn_learn_apply");
}

sgn_status sgn_learn_basis_get(sgn_learn_t L, double *mean_h, double *basis_h) {
  if (!L) return SGN_EINVAL;
  if (!L->bound || !L->have_basis) return SGN_ESTATE;
  Ctx &c = *L->h;
  if ((mean_h && cudaMemcpyAsync(mean_h, L->mean, (size_t)L->n_dof * 8, cudaMemcpyDeviceToHost, c.stream)) ||
      (basis_h &&
       cudaMemcpyAsync(basis_h, L->basis, (size_t)L->n_dof * L->n_modes * 8, cudaMemcpyDeviceToHost, c.stream)) ||
      cudaStreamSynchronize(c.stream))
    return fail(*L, "sgn_learn_basis_get");
  return check(*L, "sgn_learn_basis_get");
}

}  // extern "C"
