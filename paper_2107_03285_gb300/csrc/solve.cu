// Forward, diagonal and backward substitutions with a multifrontal factor
// (front.cu), and the inverses of the factor's 128-wide diagonal blocks they
// use.
#include <cmath>
#include <cstdio>
#include <functional>

#include "common.cuh"
#include "front_view.cuh"

namespace sgn {

namespace {

// ------------------------------------------------------------------ solves
__global__ void k_fwd_gather(DevSym d, SV sv, int64_t item_base, int64_t n, const double *__restrict__ b) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n) return;
  const int dpn = sv.dpn;
  const int64_t item = item_base + idx / dpn;
  const int kd = (int)(idx % dpn);
  const int s = d.item_sn[item], P = d.item_P[item];
  const int nown = d.sn_nown[s];
  double v = P < nown ? b[(int64_t)(d.sn_first[s] + P) * dpn + kd] : 0.0;
  const int coff = d.sn_child_off[s], nch = d.sn_nchild[s];
  for (int j = 0; j < nch; ++j) {
    int c = d.children[coff + j];
    int q = d.cmap[d.cmap_off[coff + j] + P];
    if (q >= 0) v += sv.rhs[sv.rhs_off[c] + (int64_t)d.sn_nown[c] * dpn + (int64_t)q * dpn + kd];
  }
  sv.rhs[sv.rhs_off[s] + (int64_t)P * dpn + kd] = v;
}


// Arithmetic of the substitutions is done in the factor's precision (AT = T):
// with FP32 fronts every solve is the correction solve of mixed-precision
// iterative refinement, whose residual and update are formed in FP64 outside.

// Inverse X = L_bb^{-1} of every SB x SB unit-lower diagonal block of the
// factor, stored as a dense row-major w x w block (unit diagonal, zeros
// above) in the store's inverse array.  One CTA per block, thread c
// computes column c of X by forward substitution (no cross-thread
// dependency).  Run once per level after its factorization, so that every
// later solve replaces the sequential triangular solve of a block by a
// matrix-vector product read with vector loads.
template <typename T>
__global__ void __launch_bounds__(SB) k_diag_inverse(DevSym d, SV sv, const int32_t *__restrict__ fronts) {
  extern __shared__ unsigned char inv_raw[];
  T(*A)[SB + 1] = reinterpret_cast<T(*)[SB + 1]>(inv_raw);  // A[t][i] = L(t, i) (i < t), A[c][t] = X(t, c) (t > c)
  const int s = fronts[blockIdx.y];
  const int dpn = sv.dpn;
  const int ns = d.sn_nown[s] * dpn;
  const int k = blockIdx.x * SB;
  if (k >= ns) return;
  const int f = front_order(d, s, dpn);
  const int w = min(SB, ns - k);
  T *F = (T *)sv.F + sv.front_off[s];
  const int c = threadIdx.x;
  for (int i = 0; i < w; ++i)
    if (c > i && c < w) A[c][i] = F[(int64_t)(k + c) + (int64_t)(k + i) * f];
  __syncthreads();
  if (c < w) {
    for (int t = c + 1; t < w; ++t) {
      T acc = A[t][c];
      for (int i = c + 1; i < t; ++i) acc += A[t][i] * A[c][i];
      A[c][t] = -acc;
    }
  }
  __syncthreads();
  T *X = (T *)sv.Xinv + sv.xinv_off[s] + (int64_t)blockIdx.x * SB * SB;
  for (int j = 0; j < w; ++j)  // row j, the threads along its columns c
    if (c < w) X[(int64_t)j * w + c] = c < j ? A[c][j] : (c == j ? T(1) : T(0));
}

// loads X = L_bb^{-1} of the block at k (block index k / SB) as U[j][i] =
// X(j, i): the dense row-major block is read as 16-byte vectors, 8 per thread
// in flight (one round trip for a 128 x 128 FP32 block and 512 threads)
template <typename T, typename AT>
__device__ __forceinline__ void load_block_inverse(const SV &sv, int s, int k, int w, AT (*U)[SB + 1]) {
  const T *X = (const T *)sv.Xinv + sv.xinv_off[s] + (int64_t)(k / SB) * SB * SB;
  constexpr int VE = 16 / sizeof(T);  // elements per vector
  constexpr int NV = 8;               // vectors in flight per thread
  const int nv = (w * w + VE - 1) / VE;
  for (int base = threadIdx.x; base < nv; base += NV * blockDim.x) {
    T v[NV][VE];
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      const int q = base + u * blockDim.x;
      if (q < nv) {
        if constexpr (sizeof(T) == 4) {
          const float4 t = reinterpret_cast<const float4 *>(X)[q];
          v[u][0] = t.x; v[u][1] = t.y; v[u][2] = t.z; v[u][3] = t.w;
        } else {
          const double2 t = reinterpret_cast<const double2 *>(X)[q];
          v[u][0] = t.x; v[u][1] = t.y;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < NV; ++u) {
      const int q = base + u * blockDim.x;
      if (q >= nv) continue;
#pragma unroll
      for (int e = 0; e < VE; ++e) {
        const int idx = q * VE + e;
        if (idx < w * w) U[idx / w][idx % w] = (AT)v[u][e];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Dataflow substitutions.  The forward (backward) substitution of a level is
// one launch with one CTA per item of the level's schedule: a 128-row band of
// a front (forward) or a 128-column block (backward).  A CTA takes its item by
// ticket, so every item it depends on belongs to a CTA that started before
// it; it streams its part of the factor while waiting, bounded, for the
// values of the blocks it depends on, and publishes its own block's values
// for the CTAs after it.  The sequential chain of 128-wide blocks thus costs
// one publish-and-observe latency per block instead of a kernel launch.

constexpr int SBT = 4 * SB;                          // threads of a substitution CTA
constexpr long long SOLVE_WAIT_CYCLES = 1ll << 31;  // ~1 s at 2 GHz

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ bool timed_out(const int *status) {
  return (*(volatile const int *)status & DEV_TIMEOUT) != 0;
}

// compensated (Kahan) running sum in the substitution's precision
template <typename AT>
__device__ __forceinline__ void kahan_add(AT &sum, AT &comp, AT x) {
  const AT y = x - comp;
  const AT t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

template <typename AT>
struct SolveShared {
  AT xs[2][SB];       // values of the block being consumed (double-buffered)
  AT dp[4][SB];       // per-quarter (per-column) compensated sums
  AT ap[4][SB];       // per-quarter partial block products
  AT rb[SB];          // right-hand side of the own block
  AT yb[SB];          // the own block's values
  int item, abort;
};

// publishes the w values of the block at pivot position p under tag (thread
// t < w holds value t); every thread calls it
template <typename T>
__device__ __forceinline__ void publish_block(const SV &sv, int64_t p, int w, unsigned tag, T val) {
  const int t = threadIdx.x;
  if constexpr (sizeof(T) == 4) {
    if (t < w) st_relaxed_u64(sv.pub + p + t, ((unsigned long long)tag << 32) | __float_as_uint(val));
  } else {
    if (t < w) reinterpret_cast<double *>(sv.pub)[p + t] = val;
    __syncthreads();
    if (t == 0) {
      __threadfence();
      st_release_u32(sv.pflag + p, tag);
    }
  }
}

// waits for the block at pivot position p published under tag and copies its
// w values to dst[0, w) (zeros up to SB); every thread calls it, and it ends
// with a barrier.  False (DEV_TIMEOUT recorded) when the wait bound expires
// or another CTA already gave up.
// FP32 form of the wait: the w words at a[0, w), each a value's bits with
// its tag, into dst[0, w) (zeros up to SB); thread t polls word t.  No
// barrier.
__device__ __forceinline__ void wait_words(const unsigned long long *a, int w, unsigned tag, float *dst,
                                           int *status, int *abort) {
  const int t = threadIdx.x;
  if (t < w) {
    unsigned long long v = ld_relaxed_u64(a + t);
    if ((unsigned)(v >> 32) != tag) {
      const long long t0 = clock64();
      for (int n = 1; (unsigned)((v = ld_relaxed_u64(a + t)) >> 32) != tag; ++n) {
        if ((n & 255) == 0 && (timed_out(status) || clock64() - t0 > SOLVE_WAIT_CYCLES)) {
          atomicOr(status, DEV_TIMEOUT);
          *abort = 1;
          break;
        }
      }
    }
    dst[t] = __uint_as_float((unsigned)v);
  } else if (t < SB) {
    dst[t] = 0.f;
  }
}

template <typename T>
__device__ __forceinline__ bool wait_block(const SV &sv, int64_t p, int w, unsigned tag, T *dst, int *status,
                                           int *abort) {
  const int t = threadIdx.x;
  if constexpr (sizeof(T) == 4) {
    wait_words(sv.pub + p, w, tag, dst, status, abort);
  } else {
    if (t == 0 && ld_acquire_u32(sv.pflag + p) != tag) {
      const long long t0 = clock64();
      for (int n = 1; ld_acquire_u32(sv.pflag + p) != tag; ++n) {
        if ((n & 255) == 0 && (timed_out(status) || clock64() - t0 > SOLVE_WAIT_CYCLES)) {
          atomicOr(status, DEV_TIMEOUT);
          *abort = 1;
          break;
        }
      }
    }
    __syncthreads();
    if (t < w) dst[t] = __ldcg(reinterpret_cast<const double *>(sv.pub) + p + t);
    else if (t < SB) dst[t] = 0.0;
  }
  __syncthreads();
  return *abort == 0;
}

// item ticket and completion: the last CTA of a launch resets the counters
// for the next launch of the same store
template <typename AT>
__device__ __forceinline__ bool solve_item_begin(unsigned *ctl, int *status, SolveShared<AT> &sm) {
  if (threadIdx.x == 0) {
    sm.item = (int)atomicAdd(&ctl[1], 1u);
    sm.abort = 0;
    if (sm.item >= (int)gridDim.x) {  // counters not reset by the previous launch
      atomicOr(status, DEV_TIMEOUT);
      sm.abort = 1;
    } else if (timed_out(status)) {
      sm.abort = 1;
    }
  }
  __syncthreads();
  return sm.abort == 0;
}

__device__ __forceinline__ void solve_item_end(unsigned *ctl) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctl[2], 1u) == gridDim.x - 1) {
      atomicExch(&ctl[1], 0u);
      atomicExch(&ctl[2], 0u);
    }
  }
}

// a new solve: new tags (2e forward, 2e + 1 backward), counters cleared
__global__ void k_solve_begin(unsigned *ctl) {
  ctl[0] += 1u;
  ctl[1] = 0u;
  ctl[2] = 0u;
}

// Forward item: rows [r0, r0 + nr) of front s.  Thread (row, quarter qq)
// accumulates sum_j L(row, block j) y_j over its 32 columns of every own
// block j the band depends on.  A struct band subtracts the sums from its
// right-hand side (read by the parent's gather); own band b forms r_b =
// P rhs_b - sums, y_b = X_b r_b with X_b = L_bb^{-1}, publishes y_b and writes
// z_b = D_b^{-1} y_b.
template <typename T>
__device__ __forceinline__ void fwd_item(const DevSym &d, const SV &sv, const int32_t *__restrict__ lvl_fronts,
                                         SolveItem itm, int nb, unsigned tag, int *status, T (*U)[SB + 1],
                                         SolveShared<T> &sm) {
  using AT = T;
  const int s = lvl_fronts[itm.q];
  const int dpn = sv.dpn;
  const int ns = d.sn_nown[s] * dpn;
  const int f = front_order(d, s, dpn);
  const int nbo = (ns + SB - 1) / SB;
  const bool own = itm.key < nbo;
  const int r0 = own ? itm.key * SB : ns + (itm.key - nbo) * SB;
  const int nr = min(SB, (own ? ns : f) - r0);  // an own band ends at the last own row
  const int ndep = own ? itm.key : nbo;
  const T *F = (const T *)sv.F + sv.front_off[s];
  const int64_t po = sv.piv_off[s];
  const int tid = threadIdx.x, row = tid & (SB - 1), qq = tid >> 7;
  if (own) load_block_inverse<T, AT>(sv, s, r0, nr, U);
  AT sum = AT(0), comp = AT(0);
  for (int j = 0; j < ndep; ++j) {
    const int kc = j * SB, wc = min(SB, ns - kc);
    const T *Fc = F + (int64_t)(kc + 32 * qq) * f + r0 + row;
    T v[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) v[u] = (row < nr && 32 * qq + u < wc) ? Fc[(int64_t)u * f] : T(0);
    AT *y = sm.xs[j & 1];
    if (!wait_block<T>(sv, po + kc, wc, tag, y, status, &sm.abort)) return;
    AT a = AT(0);
#pragma unroll
    for (int u = 0; u < 32; ++u) a += (AT)v[u] * y[32 * qq + u];
    kahan_add(sum, comp, a);
  }
  // partial sums are joined in the factor's precision; FP64 (slow on this
  // part) only for the one subtraction per row from the FP64 right-hand side
  sm.dp[qq][row] = sum - comp;
  __syncthreads();
  if (!own) {
    if (tid < nr) {
      double *rhs = sv.rhs + sv.rhs_off[s];
      rhs[r0 + tid] -= (double)((sm.dp[0][tid] + sm.dp[1][tid]) + (sm.dp[2][tid] + sm.dp[3][tid]));
    }
    return;
  }
  const int w = nr;
  if (tid < SB) {
    AT r = AT(0);
    if (tid < w) {
      // the factor's rows are in final pivoted order; the pivots permute
      // positions inside their panel of nb columns
      const int pos = r0 + tid, pstart = (pos / nb) * nb;
      const double b = sv.rhs[sv.rhs_off[s] + pstart + sv.piv_perm[po + pos]];
      r = (AT)(b - (double)((sm.dp[0][tid] + sm.dp[1][tid]) + (sm.dp[2][tid] + sm.dp[3][tid])));
    }
    sm.rb[tid] = r;
  }
  __syncthreads();
  {
    AT a = AT(0);
    const int i1 = min(32 * qq + 32, row);
    for (int i = 32 * qq; i < i1; ++i) a += U[row][i] * sm.rb[i];
    sm.ap[qq][row] = a;
  }
  __syncthreads();
  AT y = AT(0);
  if (tid < w) {
    y = sm.rb[tid] + ((sm.ap[0][tid] + sm.ap[1][tid]) + (sm.ap[2][tid] + sm.ap[3][tid]));
    sm.yb[tid] = y;
  }
  publish_block<T>(sv, po + r0, w, tag, y);
  __syncthreads();
  if (tid < w) {
    const int64_t p = po + r0 + tid;
    const int ty = sv.piv_type[p];
    if (ty == 0) {
      sv.yz[p] = (double)y / sv.D0[p];
    } else if (ty == 1) {
      const double d11 = sv.D0[p], d21 = sv.D1[p], d22 = sv.D0[p + 1];
      const double det = d11 * d22 - d21 * d21;
      const double y1 = (double)y, y2 = (double)sm.yb[tid + 1];
      sv.yz[p] = (d22 * y1 - d21 * y2) / det;
      sv.yz[p + 1] = (d11 * y2 - d21 * y1) / det;
    }
  }
  if (nbo > 1) return;
  // a single-block front has no struct-band items: this CTA updates its
  // struct rows' right-hand side with y_b from shared memory, 128 rows a pass
  if (tid >= w && tid < SB) sm.yb[tid] = AT(0);
  __syncthreads();
  double *rhs = sv.rhs + sv.rhs_off[s];
  for (int rs = ns; rs < f; rs += SB) {
    const int nrs = min(SB, f - rs);
    const T *Fc = F + (int64_t)(32 * qq) * f + rs + row;
    T v[32];
#pragma unroll
    for (int u = 0; u < 32; ++u) v[u] = (row < nrs && 32 * qq + u < w) ? Fc[(int64_t)u * f] : T(0);
    AT a = AT(0);
#pragma unroll
    for (int u = 0; u < 32; ++u) a += (AT)v[u] * sm.yb[32 * qq + u];
    sm.ap[qq][row] = a;
    __syncthreads();
    if (tid < nrs) rhs[rs + tid] -= (double)((sm.ap[0][tid] + sm.ap[1][tid]) + (sm.ap[2][tid] + sm.ap[3][tid]));
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(SBT, sizeof(T) == 4 ? 2 : 1)
    k_fwd_level(DevSym d, SV sv, const int32_t *__restrict__ lvl_fronts, const SolveItem *__restrict__ items, int nb,
                unsigned *ctl, int *status) {
  extern __shared__ unsigned char blk_raw[];
  __shared__ SolveShared<T> sm;
  if (solve_item_begin(ctl, status, sm)) {
    const unsigned tag = 2u * *(volatile unsigned *)ctl;
    fwd_item<T>(d, sv, lvl_fronts, items[sm.item], nb, tag, status, reinterpret_cast<T(*)[SB + 1]>(blk_raw), sm);
  }
  solve_item_end(ctl);
}

// Backward item: own block b = [k, k + w) of front s.  Warp wq owns columns
// k + 8 wq .. + 8 with its lanes along the rows (coalesced) and accumulates
// L(rows, column)^T x over the struct rows (x there is the ancestors'
// solution) and over every later own block; v_b = z_b minus those sums gives
// x_b = X_b^T v_b, which is published for the earlier blocks and written,
// un-pivoted, into the solution.
template <typename T>
__device__ __forceinline__ void bwd_item(const DevSym &d, const SV &sv, const int32_t *__restrict__ lvl_fronts,
                                         SolveItem itm, int nb, unsigned tag, int *status, double *__restrict__ sol,
                                         T (*U)[SB + 1], SolveShared<T> &sm, T *xall, int xcap) {
  using AT = T;
  const int s = lvl_fronts[itm.q];
  const int dpn = sv.dpn;
  const int ns = d.sn_nown[s] * dpn;
  const int f = front_order(d, s, dpn);
  const int nbo = (ns + SB - 1) / SB;
  const int b = nbo - 1 - itm.key;
  const int k = b * SB, w = min(SB, ns - k);
  const T *F = (const T *)sv.F + sv.front_off[s];
  const int64_t po = sv.piv_off[s];
  const int tid = threadIdx.x, row = tid & (SB - 1), qq = tid >> 7;
  const int warp = tid >> 5, lane = tid & 31, c0 = 8 * warp;
  load_block_inverse<T, AT>(sv, s, k, w, U);
  AT sum[8], comp[8];
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) sum[cc] = comp[cc] = AT(0);
  int ph = 0;  // alternates the value buffers across both loops
  // struct rows: the solution there (the ancestors') is final
  const int nown = d.sn_nown[s];
  const int32_t *sr = d.struct_ranks + d.sn_struct_off[s];
  const int nparts = sizeof(T) == 4 ? bwd_parts(f - ns) : 0;
  // the product's parts, published by their own CTAs (listed first)
  for (int h = 0; h < nparts; ++h, ++ph) {
    AT *x = sm.xs[ph & 1];
    wait_words(sv.bpart + sv.part_off[s] + (int64_t)h * ns + k, w, tag, reinterpret_cast<float *>(x), status,
               &sm.abort);
    __syncthreads();
    if (sm.abort) return;
    if (lane == 0) {
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) kahan_add(sum[cc], comp[cc], x[c0 + cc]);
    }
  }
  if (nparts == 0 && f - ns <= xcap) {
    // all of it gathered into shared memory once, then 128 rows a pass
    // without a barrier (the warps overlap)
    for (int idx = tid; idx < f - ns; idx += blockDim.x)
      xall[idx] = (AT)sol[(int64_t)sr[(ns + idx) / dpn - nown] * dpn + (ns + idx) % dpn];
    __syncthreads();
    for (int rs = ns; rs < f; rs += SB) {
      const int nrs = min(SB, f - rs);
      const T *Fc = F + (int64_t)(k + c0) * f + rs + lane;
      T q[8][4];
#pragma unroll
      for (int cc = 0; cc < 8; ++cc)
#pragma unroll
        for (int m = 0; m < 4; ++m)
          q[cc][m] = (c0 + cc < w && lane + 32 * m < nrs) ? Fc[(int64_t)cc * f + 32 * m] : T(0);
      AT xv[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) xv[m] = lane + 32 * m < nrs ? xall[rs - ns + lane + 32 * m] : AT(0);
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        AT a = AT(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) a += (AT)q[cc][m] * xv[m];
        kahan_add(sum[cc], comp[cc], a);
      }
    }
  }
  // otherwise gathered 128 rows a pass; the struct-rank index of the next
  // pass is read one pass ahead
  const bool by_pass = nparts == 0 && f - ns > xcap;
  int sidx = (by_pass && tid < SB && ns + tid < f) ? sr[(ns + tid) / dpn - nown] : 0;
  for (int rs = ns; by_pass && rs < f; rs += SB, ++ph) {
    const int nrs = min(SB, f - rs);
    const T *Fc = F + (int64_t)(k + c0) * f + rs + lane;
    T q[8][4];
#pragma unroll
    for (int cc = 0; cc < 8; ++cc)
#pragma unroll
      for (int m = 0; m < 4; ++m)
        q[cc][m] = (c0 + cc < w && lane + 32 * m < nrs) ? Fc[(int64_t)cc * f + 32 * m] : T(0);
    AT *x = sm.xs[ph & 1];
    if (tid < SB) {
      const int ii = rs + tid;
      const int cur = sidx;
      if (ii + SB < f) sidx = sr[(ii + SB) / dpn - nown];
      x[tid] = tid < nrs ? (AT)sol[(int64_t)cur * dpn + ii % dpn] : AT(0);
    }
    __syncthreads();
    AT xv[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) xv[m] = x[lane + 32 * m];
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      AT a = AT(0);
#pragma unroll
      for (int m = 0; m < 4; ++m) a += (AT)q[cc][m] * xv[m];
      kahan_add(sum[cc], comp[cc], a);
    }
  }
  // later own blocks, as their values are published
  for (int j = nbo - 1; j > b; --j, ++ph) {
    const int kr = j * SB, wr = min(SB, ns - kr);
    const T *Fc = F + (int64_t)(k + c0) * f + kr + lane;
    T q[8][4];
#pragma unroll
    for (int cc = 0; cc < 8; ++cc)
#pragma unroll
      for (int m = 0; m < 4; ++m)
        q[cc][m] = (c0 + cc < w && lane + 32 * m < wr) ? Fc[(int64_t)cc * f + 32 * m] : T(0);
    AT *x = sm.xs[ph & 1];
    if (!wait_block<T>(sv, po + kr, wr, tag, x, status, &sm.abort)) return;
    AT xv[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) xv[m] = x[lane + 32 * m];
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      AT a = AT(0);
#pragma unroll
      for (int m = 0; m < 4; ++m) a += (AT)q[cc][m] * xv[m];
      kahan_add(sum[cc], comp[cc], a);
    }
  }
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    AT t = sum[cc] - comp[cc];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sm.dp[0][c0 + cc] = t;
  }
  __syncthreads();
  if (tid < SB) sm.rb[tid] = tid < w ? (AT)(sv.yz[po + k + tid] - (double)sm.dp[0][tid]) : AT(0);
  __syncthreads();
  {
    AT a = AT(0);
    const int j1 = min(32 * qq + 32, w);
    for (int jj = max(32 * qq, row + 1); jj < j1; ++jj) a += U[jj][row] * sm.rb[jj];
    sm.ap[qq][row] = a;
  }
  __syncthreads();
  AT x = AT(0);
  if (tid < w) x = sm.rb[tid] + ((sm.ap[0][tid] + sm.ap[1][tid]) + (sm.ap[2][tid] + sm.ap[3][tid]));
  publish_block<T>(sv, po + k, w, tag, x);
  if (tid < w) {
    // piv_perm is local to the pivot panel (width nb) holding position k + tid
    const int pos = k + tid, pstart = (pos / nb) * nb;
    sol[(int64_t)d.sn_first[s] * dpn + pstart + sv.piv_perm[po + pos]] = (double)x;
  }
}

// one part of a backward block's ancestor-row product (FP32 fronts, key < 0):
// rows [r0, r0 + rn) of the front's struct rows times their solution values,
// for the block's w columns, gathered into shared memory xcap rows at a time;
// published at bpart[part_off[s] + h ns + k + t] for the block's CTA
template <typename T>
__device__ __noinline__ void bwd_part(const DevSym &d, const SV &sv, const int32_t *__restrict__ lvl_fronts,
                                      SolveItem itm, unsigned tag, const double *__restrict__ sol,
                                      SolveShared<T> &sm, T *xall, int xcap) {
  using AT = T;
  const int s = lvl_fronts[itm.q];
  const int dpn = sv.dpn;
  const int ns = d.sn_nown[s] * dpn;
  const int f = front_order(d, s, dpn);
  const int j = -1 - itm.key, b = j / BWD_PARTS_MAX, h = j % BWD_PARTS_MAX;
  const int k = b * SB, w = min(SB, ns - k);
  const int rp = bwd_part_rows(f - ns);
  const int r0 = h * rp, rn = min(rp, f - ns - r0);
  const T *F = (const T *)sv.F + sv.front_off[s];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, c0 = 8 * warp;
  const int nown = d.sn_nown[s];
  const int32_t *sr = d.struct_ranks + d.sn_struct_off[s];
  AT sum[8], comp[8];
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) sum[cc] = comp[cc] = AT(0);
  for (int g0 = 0; xcap > 0 && g0 < rn; g0 += xcap) {
    const int gn = min(xcap, rn - g0);
    if (g0 > 0) __syncthreads();  // the previous chunk's reads are done
    for (int idx = tid; idx < gn; idx += blockDim.x) {
      const int ii = ns + r0 + g0 + idx;
      xall[idx] = (AT)sol[(int64_t)sr[ii / dpn - nown] * dpn + ii % dpn];
    }
    __syncthreads();
    for (int rs = ns + r0 + g0; rs < ns + r0 + g0 + gn; rs += SB) {
      const int nrs = min(SB, ns + r0 + g0 + gn - rs);
      const T *Fc = F + (int64_t)(k + c0) * f + rs + lane;
      T q[8][4];
#pragma unroll
      for (int cc = 0; cc < 8; ++cc)
#pragma unroll
        for (int m = 0; m < 4; ++m)
          q[cc][m] = (c0 + cc < w && lane + 32 * m < nrs) ? Fc[(int64_t)cc * f + 32 * m] : T(0);
      AT xv[4];
#pragma unroll
      for (int m = 0; m < 4; ++m)
        xv[m] = lane + 32 * m < nrs ? xall[rs - (ns + r0 + g0) + lane + 32 * m] : AT(0);
#pragma unroll
      for (int cc = 0; cc < 8; ++cc) {
        AT a = AT(0);
#pragma unroll
        for (int m = 0; m < 4; ++m) a += (AT)q[cc][m] * xv[m];
        kahan_add(sum[cc], comp[cc], a);
      }
    }
  }
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    AT t = sum[cc] - comp[cc];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) sm.dp[0][c0 + cc] = t;
  }
  __syncthreads();
  if (tid < w)
    st_relaxed_u64(sv.bpart + sv.part_off[s] + (int64_t)h * ns + k + tid,
                   ((unsigned long long)tag << 32) | __float_as_uint((float)sm.dp[0][tid]));
}

// dynamic shared memory: the block inverse (SB x (SB + 1)), then xcap
// solution values of the ancestor (struct) rows (0: gathered pass by pass)
template <typename T>
__global__ void __launch_bounds__(SBT, sizeof(T) == 4 ? 2 : 1)
    k_bwd_level(DevSym d, SV sv, const int32_t *__restrict__ lvl_fronts, const SolveItem *__restrict__ items, int nb,
                unsigned *ctl, int *status, double *__restrict__ sol, int xcap) {
  extern __shared__ __align__(16) unsigned char blk_raw[];
  __shared__ SolveShared<T> sm;
  if (solve_item_begin(ctl, status, sm)) {
    const unsigned tag = 2u * *(volatile unsigned *)ctl + 1u;
    const SolveItem itm = items[sm.item];
    bool part = false;
    if constexpr (sizeof(T) == 4) {
      if (itm.key < 0) {
        bwd_part<T>(d, sv, lvl_fronts, itm, tag, sol, sm, reinterpret_cast<T *>(blk_raw) + SB * (SB + 1), xcap);
        part = true;
      }
    }
    if (!part)
      bwd_item<T>(d, sv, lvl_fronts, itm, nb, tag, status, sol, reinterpret_cast<T(*)[SB + 1]>(blk_raw), sm,
                  reinterpret_cast<T *>(blk_raw) + SB * (SB + 1), xcap);
  }
  solve_item_end(ctl);
}

// the most ancestor rows a backward CTA keeps in shared memory (two FP32 CTAs,
// one FP64 CTA per SM)
template <typename T>
constexpr int bwd_xcap_max() {
  return sizeof(T) == 4 ? 9216 : 8192;
}

template <typename T>
void solve_impl(Ctx &c, Store &st, const double *b, double *x) {
  ProfScope ps(c, SGN_PROF_SOLVE);
  SV sv = view(st);
  const int nb = c.S.opts.panel;
  const int dpn = st.dpn;
  const size_t blk_smem = (size_t)SB * (SB + 1) * sizeof(T);
  k_solve_begin<<<1, 1, 0, c.stream>>>(st.ctl);
  c.count();
  for (int L = 0; L < c.S.n_levels; ++L) {
    const int64_t i0 = c.h_item_ptr[L], n = (c.h_item_ptr[L + 1] - i0) * dpn;
    if (n > 0) {
      k_fwd_gather<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(c.ds, sv, i0, n, b);
      c.count();
    }
    const int64_t t0 = st.h_fwd_lvl[L], nt = st.h_fwd_lvl[L + 1] - t0;
    if (nt == 0) continue;
    k_fwd_level<T><<<(unsigned)nt, SBT, blk_smem, c.stream>>>(c.ds, sv, c.ds.lvl_fronts, st.fwd_items + t0, nb,
                                                              st.ctl, c.status);
    c.count();
  }
  for (int L = c.S.n_levels - 1; L >= 0; --L) {
    const int64_t t0 = st.h_bwd_lvl[L], nt = st.h_bwd_lvl[L + 1] - t0;
    if (nt == 0) continue;
    // the most ancestor rows one CTA of the level gathers (a front's, or a
    // part's where the product is split); FP64 fronts beyond the shared
    // memory cap gather them 128 a pass (0)
    int xs = 0;
    for (int s : c.S.level_fronts[L]) {
      const int r = c.S.sn[s].nstruct * dpn;
      xs = std::max(xs, sizeof(T) == 4 && bwd_parts(r) > 0 ? bwd_part_rows(r) : r);
    }
    const int xcap = sizeof(T) == 4 ? std::min(xs, bwd_xcap_max<T>()) : (xs <= bwd_xcap_max<T>() ? xs : 0);
    k_bwd_level<T><<<(unsigned)nt, SBT, blk_smem + (size_t)xcap * sizeof(T), c.stream>>>(
        c.ds, sv, c.ds.lvl_fronts, st.bwd_items + t0, nb, st.ctl, c.status, x, xcap);
    c.count();
  }
}

}  // namespace

// one bounded wait on a block value that nothing publishes (tag 1 is never
// used: solves use 2e and 2e + 1, e >= 1): it must give up and record
// DEV_TIMEOUT in the status word
template <typename T>
__global__ void k_wait_selftest(SV sv, int *status) {
  __shared__ SolveShared<T> sm;
  if (threadIdx.x == 0) sm.abort = 0;
  __syncthreads();
  wait_block<T>(sv, 0, 1, 1u, sm.xs[0], status, &sm.abort);
}

void wait_selftest(Ctx &c, Store &s) {
  SV sv = view(s);
  if (s.fp32) k_wait_selftest<float><<<1, SB, 0, c.stream>>>(sv, c.status);
  else k_wait_selftest<double><<<1, SB, 0, c.stream>>>(sv, c.status);
}

void solve_direct(Ctx &c, Store &s, const double *b, double *x) {
  if (s.fp32) solve_impl<float>(c, s, b, x);
  else solve_impl<double>(c, s, b, x);
}

void solve_store(Ctx &c, Store &s, const double *b, double *x) {
  auto run = [&]() {
    if (s.fp32) solve_impl<float>(c, s, b, x);
    else solve_impl<double>(c, s, b, x);
  };
  if (!c.use_graphs || !c.cap_stream || c.prof_mask != 0) {
    run();
    return;
  }
  if (!s.sgraph || s.sgraph_b != b || s.sgraph_x != x) {
    if (s.sgraph) cudaGraphExecDestroy(s.sgraph);
    s.sgraph = capture_fn(c, run, &s.sgraph_launches, nullptr);
    s.sgraph_b = b;
    s.sgraph_x = x;
  }
  if (!s.sgraph) { run(); return; }
  cudaGraphLaunch(s.sgraph, c.stream);
  c.launches += s.sgraph_launches;
}

void launch_diag_inverse(Ctx &c, Store &st, const int32_t *fronts, int max_ns, int nfronts) {
  SV sv = view(st);
  dim3 gi((max_ns + SB - 1) / SB, (unsigned)nfronts);
  if (st.fp32) k_diag_inverse<float><<<gi, SB, (size_t)SB * (SB + 1) * sizeof(float), c.stream>>>(c.ds, sv, fronts);
  else k_diag_inverse<double><<<gi, SB, (size_t)SB * (SB + 1) * sizeof(double), c.stream>>>(c.ds, sv, fronts);
  c.count();
}

void set_solve_attributes() {
  cudaFuncSetAttribute(k_fwd_level<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(SB * (SB + 1) * 8));
  cudaFuncSetAttribute(k_fwd_level<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(SB * (SB + 1) * 4));
  cudaFuncSetAttribute(k_bwd_level<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)((SB * (SB + 1) + bwd_xcap_max<double>()) * 8));
  cudaFuncSetAttribute(k_bwd_level<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)((SB * (SB + 1) + bwd_xcap_max<float>()) * 4));
  cudaFuncSetAttribute(k_diag_inverse<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(SB * (SB + 1) * 8));
  cudaFuncSetAttribute(k_diag_inverse<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(SB * (SB + 1) * 4));
}

}  // namespace sgn
