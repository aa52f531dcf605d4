// The outer-block panel kernel of the multifrontal factorization (front.cu
// holds the factorization as a whole).  Included by one translation unit per
// front type (panels_f32.cu, panels_f64.cu), which instantiate the launchers
// at the end; the kernel itself has internal linkage in each.
//
// One launch factors the pivot panels of one 256-column outer block [K0,
// kend) of every active front of a level.  Each CTA (4 warps) owns a band of
// 128 rows of one front (rows K0 + 128 b ...).  For every panel [k, k + w):
//   * the band holding the panel's diagonal rows (the owner) keeps that
//     diagonal block up to date right-looking while it solves the earlier
//     panels' rows; as soon as the rows of the panel before have updated it,
//     the owner's warp 0 publishes that the panel's rows are final in the
//     block's earlier columns (flag fpre), factors the diagonal block with
//     Bunch-Kaufman (one warp) and publishes L11 / D / the permutation (flag
//     fflag; both are release stores of the factorization's epoch);
//   * every band with rows below the panel first updates its rows
//     left-looking by the block's earlier panels, each warp on its own, once
//     fpre is set (the owner's other warps do this while warp 0 factors the
//     block), then waits (bounded) for fflag, permutes and solves its rows
//     against L11 (W = L21 D and L21), and writes the K-major hi / lo copies
//     the tensor-core update reads.
// A CTA takes its (front, band) item by ticket; the items list every front's
// bands 0 and 1 (the only owners) before all other bands, so every CTA a
// band waits for has started before it.  A wait that expires records
// DEV_TIMEOUT and the CTA gives up.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "front_view.cuh"
#include "tc_update.cuh"

namespace sgn {

namespace {

constexpr int BAND = 128;                           // rows per CTA
constexpr long long PANEL_WAIT_CYCLES = 1ll << 31;  // ~1 s at 2 GHz
static_assert(PANEL_XS >= BAND && PANEL_XS % 4 == 0, "row pitch of the band buffers");

__device__ __forceinline__ unsigned ld_acquire_flag(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_flag(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// bounded wait (one thread) until *p == epoch; false (DEV_TIMEOUT recorded)
// if it never comes or another CTA already gave up
__device__ __forceinline__ bool wait_epoch(const unsigned *p, unsigned epoch, int *status) {
  if (ld_acquire_flag(p) == epoch) return true;
  const long long t0 = clock64();
  for (int n = 1;; ++n) {
    if (ld_acquire_flag(p) == epoch) return true;
    if ((n & 255) == 0 && ((*(volatile const int *)status & DEV_TIMEOUT) || clock64() - t0 > PANEL_WAIT_CYCLES)) {
      atomicOr(status, DEV_TIMEOUT);
      return false;
    }
  }
}

// The Bunch-Kaufman pivot tests, decided exactly as their FP64 evaluation:
//   ge_alpha(a, c):      a >= alpha * c                 (FP64 product)
//   ge_alpha_sq(a, r, c): a * r >= alpha * (c * c)       (FP64 products)
// with a, r, c values of the front's type.  For FP32 fronts the comparison is
// first made in FP32; the FP32 operands differ from the FP64 ones by less
// than 2^-22 relative, so a gap larger than 2^-20 of the larger side decides
// it, and only a near tie runs the FP64 arithmetic (the FP64 pipe of this
// part issues a warp instruction every ~64 cycles).
constexpr double BK_ALPHA = 0.6403882032022076;  // (1 + sqrt(17)) / 8
// the FP64 evaluations of near ties, out of line so that the common FP32
// decision does not issue (predicated) FP64 instructions
__device__ __noinline__ bool ge_alpha_fp64(double a, double c) { return a >= BK_ALPHA * c; }
__device__ __noinline__ bool ge_alpha_sq_fp64(double a, double r, double c) { return a * r >= BK_ALPHA * (c * c); }
__device__ __forceinline__ bool ge_alpha(float a, float c) {
  const float r = 0.64038820f * c;
  const float g = a - r;
  if (fabsf(g) > 0x1p-20f * fmaxf(a, r)) return g > 0.f;
  return ge_alpha_fp64((double)a, (double)c);
}
__device__ __forceinline__ bool ge_alpha(double a, double c) { return a >= BK_ALPHA * c; }
__device__ __forceinline__ bool ge_alpha_sq(float a, float r, float c) {
  const float lhs = a * r, rhs = (0.64038820f * c) * c;
  const float g = lhs - rhs;
  if (fabsf(g) > 0x1p-20f * fmaxf(lhs, rhs)) return g > 0.f;
  return ge_alpha_sq_fp64((double)a, (double)r, (double)c);
}
__device__ __forceinline__ bool ge_alpha_sq(double a, double r, double c) { return a * r >= BK_ALPHA * (c * c); }

// warp-wide max of non-negative magnitudes and the lowest lane holding it
// (valid lanes only; none valid: m = -1, idx = none).  FP32 magnitudes
// compare as their bit patterns, so one REDUX instruction each.
__device__ __forceinline__ void warp_argmax(float v, bool valid, int none, float &m, int &idx) {
  const unsigned key = valid ? __float_as_uint(v) + 1u : 0u;
  const unsigned mx = __reduce_max_sync(0xffffffffu, key);
  if (mx == 0u) { m = -1.f; idx = none; return; }
  m = __uint_as_float(mx - 1u);
  idx = (int)__reduce_min_sync(0xffffffffu, key == mx ? (unsigned)(threadIdx.x & 31) : 32u);
}
__device__ __forceinline__ void warp_argmax(double v, bool valid, int none, double &m, int &idx) {
  m = valid ? v : -1.0;
  idx = valid ? (int)(threadIdx.x & 31) : none;
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, m, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > m || (ov == m && oi < idx)) { m = ov; idx = oi; }
  }
}
__device__ __forceinline__ float warp_max0(float v) {  // v >= 0
  return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(v)));
}
__device__ __forceinline__ double warp_max0(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}


// four consecutive shared-memory values as one vector load (16-byte aligned)
__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4 *>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
  const double2 q0 = *reinterpret_cast<const double2 *>(p), q1 = *reinterpret_cast<const double2 *>(p + 2);
  v[0] = q0.x; v[1] = q0.y; v[2] = q1.x; v[3] = q1.y;
}

// m[c] = s[c] for all c < NBT: shared-memory broadcasts, four per vector load
template <typename CT, int NBT>
__device__ __forceinline__ void ld_bcast(const CT *s, CT (&m)[NBT]) {
#pragma unroll
  for (int g = 0; g < NBT / 4; ++g) {
    CT v[4];
    ld4(s + 4 * g, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) m[4 * g + q] = v[q];
  }
}

// symmetric interchange of kk and kp (> kk) in the trailing lower triangle
// of the shared block a (a[c][i] = A(i, c)) and in the already eliminated
// part of both rows; sperm follows
template <typename CT, int PITCH>
__device__ __noinline__ void bk_interchange(CT (*a)[PITCH], int *sperm, const int w, const int kk, const int kp) {
  const int lane = threadIdx.x & 31;
  const int n1 = w - kp - 1, n2 = kp - kk - 1, n3 = kk;
  for (int idx = lane; idx < 1 + n1 + n2 + n3; idx += 32) {
    if (idx == 0) {
      CT t0 = a[kk][kk]; a[kk][kk] = a[kp][kp]; a[kp][kp] = t0;
      int tp = sperm[kk]; sperm[kk] = sperm[kp]; sperm[kp] = tp;
    } else if (idx <= n1) {
      const int i = kp + idx;
      CT t0 = a[kk][i]; a[kk][i] = a[kp][i]; a[kp][i] = t0;
    } else if (idx <= n1 + n2) {
      const int i = kk + (idx - n1);
      CT t0 = a[kk][i]; a[kk][i] = a[i][kp]; a[i][kp] = t0;
    } else {
      const int cc = idx - n1 - n2 - 1;
      CT t0 = a[cc][kk]; a[cc][kk] = a[cc][kp]; a[cc][kp] = t0;
    }
  }
}

// Bunch-Kaufman LDL^T of the w x w diagonal block of a panel (w <= NBT <= 32)
// by one warp: 1x1 / 2x2 pivots, alpha = (1 + sqrt 17) / 8, pivot search
// restricted to the block, eliminations in CT, magnitudes compared exactly
// (max of |CT| values), pivot tests decided as in FP64 (ge_alpha,
// ge_alpha_sq).  Lane i holds row i of the lower triangle in registers
// (r[c] = A(i, c), c <= i; zero elsewhere) and mirrors every entry it
// changes into the shared block a (a[c][i] = A(i, c)), from which the
// dynamically indexed reads (column j, row imax of the pivot test, the
// pivots) are served; the multipliers of a step are broadcast through su / sv
// (32 entries, 16-byte aligned, four per vector load).  The pivot loop is not
// unrolled (the step stays small in the instruction cache); the updates
// unroll over the NBT columns with predicates.  On entry a and r hold the
// block; on return a[c][i] (i > c) holds W(i, c) = (L D)(i, c) unscaled,
// sD0 / sD1 the pivots (a 1x1 pivot below the static-pivot threshold
// replaced), stype their kinds (0: 1x1, 1 / 2: first / second of a pair) and
// sperm the block's permutation (position -> original index).
template <typename CT, int NBT>
__device__ __forceinline__ void bk_factor_regs(CT (&r)[NBT], CT (*a)[NBT + 1], const int w, const double eps_rel,
                                               int *sperm, int *stype, CT *sD0, CT *sD1, CT *su, CT *sv,
                                               unsigned long long *counters) {
  const int lane = threadIdx.x & 31;
  const int row = lane < NBT ? lane : 0;  // lanes >= NBT read a valid (unused) address
  sperm[lane] = lane; stype[lane] = 0; sD0[lane] = CT(0); sD1[lane] = CT(0);
  CT bm = CT(0);
#pragma unroll
  for (int c = 0; c < NBT; ++c) bm = max(bm, (CT)fabs(r[c]));
  bm = warp_max0(bm);
  const double thresh = eps_rel * fmax((double)bm, 1e-300);
  // the largest CT not above thresh: |x| > thresh  <=>  |x| > thresh_c
  CT thresh_c = (CT)thresh;
  if ((double)thresh_c > thresh) thresh_c = nextafter(thresh_c, CT(0));
  const CT thresh_v = (CT)thresh;  // the static pivot's magnitude
  unsigned long long n_pert = 0, n_pair = 0;  // counted in lane 0, added once at the end
  __syncwarp();
#pragma unroll 1
  for (int j = 0; j < w;) {
    // ---- pivot search: largest |A(i, j)|, i > j (ties to the lowest index)
    const bool below = lane > j && lane < w;
    CT cm;
    int imax;
    warp_argmax(below ? (CT)fabs(a[j][row]) : CT(0), below, w, cm, imax);
    const CT akk = a[j][j];
    const CT colmax = max(cm, CT(0)), absakk = (CT)fabs(akk);
    int kstep = 1, kp = j;
    if (!(!(max(absakk, colmax) > thresh_c) || ge_alpha(absakk, colmax))) {
      // largest off-diagonal |A(imax, t)|, t in [j, w), t != imax
      CT rm = CT(0);
      if (lane >= j && lane < w && lane != imax) rm = (CT)(lane < imax ? fabs(a[lane][imax]) : fabs(a[imax][lane]));
      rm = warp_max0(rm);
      const CT aii = (CT)fabs(a[imax][imax]);
      // 0: 1x1 at j, 1: 1x1 at imax, 2: 2x2 with imax
      const int dec = ge_alpha_sq(absakk, rm, colmax) ? 0 : (ge_alpha(aii, rm) ? 1 : 2);
      if (dec == 1) {
        kp = imax;
      } else if (dec == 2) {
        kstep = 2;
        kp = imax;
      }
    }
    const int kk = j + kstep - 1;
    if (kp != kk) {
      __syncwarp();  // every lane's reads of this step are done
      bk_interchange<CT, NBT + 1>(a, sperm, w, kk, kp);
      __syncwarp();
#pragma unroll
      for (int c = 0; c < NBT; ++c) r[c] = lane < NBT ? a[c][lane] : CT(0);
    }
    if (kstep == 1) {
      CT dj = a[j][j];
      const bool perturb = !(fabs(dj) > thresh_c);
      if (perturb) dj = (dj >= CT(0)) ? thresh_v : -thresh_v;
      if (lane == 0) {
        sD0[j] = dj; stype[j] = 0;
        if (perturb) ++n_pert;
      }
      const CT l = below ? a[j][row] : CT(0);
      su[lane] = l * (CT(1) / dj);
      __syncwarp();
      CT m[NBT];
      ld_bcast<CT, NBT>(su, m);
      // rows <= j and columns <= j have l = 0 / m = 0, so they stay as they
      // are; entries above the diagonal (c > lane) change but are never read
#pragma unroll
      for (int c = 0; c < NBT; ++c)
        if (c > j) {
          r[c] -= l * m[c];
          a[c][row] = r[c];
        }
    } else {
      const CT d11 = a[j][j], d21 = a[j][j + 1], d22 = a[j + 1][j + 1];
      const CT det = d11 * d22 - d21 * d21;
      const CT rdet = CT(1) / det;
      const CT i11 = d22 * rdet, i21 = -d21 * rdet, i22 = d11 * rdet;
      if (lane == 0) {
        sD0[j] = d11; sD1[j] = d21; sD0[j + 1] = d22;
        stype[j] = 1; stype[j + 1] = 2;
        ++n_pair;
      }
      const bool in = lane > j + 1 && lane < w;
      const CT u = in ? a[j][row] : CT(0), v = in ? a[j + 1][row] : CT(0);
      const CT p = u * i11 + v * i21, q = u * i21 + v * i22;  // (L1, L2) of row lane
      su[lane] = u;
      sv[lane] = v;
      __syncwarp();
      CT mu[NBT], mv[NBT];
      ld_bcast<CT, NBT>(su, mu);
      ld_bcast<CT, NBT>(sv, mv);
      // as for a 1x1 pivot: rows <= j + 1 have p = q = 0, columns <= j + 1
      // have u = v = 0, entries above the diagonal are never read
#pragma unroll
      for (int c = 0; c < NBT; ++c)
        if (c > j + 1) {
          r[c] -= p * mu[c] + q * mv[c];
          a[c][row] = r[c];
        }
    }
    __syncwarp();
    j += kstep;
  }
  if (lane == 0) {
    if (n_pert) atomicAdd(counters + 0, n_pert);
    if (n_pair) atomicAdd(counters + 1, n_pair);
  }
}

// the panel's diagonal block [k, k + w), already updated by every earlier
// panel of the outer block (the band holding it applied those updates
// right-looking, band_rows_solve), factored by the calling warp alone.  The
// block comes from the front, or (from_smem) from a, where the band's last
// diagonal-block update left it.  The results go to the band's own solve
// buffers (Ls: L11 transposed, pD0 / pD1 / pperm / ptype / pI0 / pI1, as
// band_rows_solve would load them), so that the band that factored the panel
// solves its rows without a round trip to memory; publish_panel_warp writes
// them out for the other bands.
template <typename T, int NBT>
__device__ __forceinline__ void owner_panel_warp(const SV &sv, int s, int f, int k, int w, double eps_rel,
                                                 unsigned long long *counters, T (*a)[NBT + 1], bool from_smem,
                                                 T *sD0, T *sD1, int *sperm, int *stype, T *su, T *svv, T *Ls,
                                                 T *pD0, T *pD1, T *pI0, T *pI1, int *pperm, int *ptype) {
  const int lane = threadIdx.x & 31;
  const T *F = (const T *)sv.F + sv.front_off[s];
  T r[NBT];
  if (from_smem) {
#pragma unroll
    for (int c = 0; c < NBT; ++c) r[c] = (c <= lane && lane < w) ? a[c][lane] : T(0);
  } else {
#pragma unroll
    for (int c = 0; c < NBT; ++c)
      r[c] = (c <= lane && lane < w) ? __ldcg(F + (int64_t)(k + lane) + (int64_t)(k + c) * f) : T(0);
  }
  __syncwarp();
#pragma unroll
  for (int c = 0; c < NBT; ++c)
    if (lane < NBT) a[c][lane] = r[c];
  bk_factor_regs<T, NBT>(r, a, w, eps_rel, sperm, stype, sD0, sD1, su, svv, counters);
  // D^{-1} of lane c's pivot: 1 / d for 1x1; for a pair, entry (0,0) of its
  // inverse for the first column, (1,1) for the second, i1 = entry (0,1)
  T i0 = T(1), i1 = T(0);
  if (lane < w) {
    const int ty = stype[lane];
    if (ty == 0) {
      i0 = T(1) / sD0[lane];
    } else {
      const int q = ty == 1 ? lane : lane - 1;
      const T d11 = sD0[q], d21 = sD1[q], d22 = sD0[q + 1];
      const T det = d11 * d22 - d21 * d21;
      i0 = (ty == 1 ? d22 : d11) / det;
      i1 = -d21 / det;
    }
  }
  if (lane < NBT) {
    const bool in = lane < w;
    pD0[lane] = in ? sD0[lane] : T(1);
    pD1[lane] = in ? sD1[lane] : T(0);
    pperm[lane] = in ? sperm[lane] : lane;
    ptype[lane] = in ? stype[lane] : 0;
    pI0[lane] = i0;
    pI1[lane] = i1;
    // column lane of L11 (Ls[c NBT + t] = L(t, c), t > c; zeros elsewhere):
    // from the unscaled W columns in a and the pivot's inverse
    const int ty = in ? stype[lane] : 0;
    const int cp = ty == 1 ? lane + 1 : (ty == 2 ? lane - 1 : lane);  // the pair's other column
#pragma unroll 4
    for (int ii = 0; ii < NBT; ++ii) {
      T val = T(0);
      if (in && ii < w && ii > lane && !(ty == 1 && ii == lane + 1)) {
        const T wc = a[lane][ii], wo = a[cp][ii];
        val = ty == 0 ? wc * i0 : wc * i0 + wo * i1;
      }
      Ls[lane * NBT + ii] = val;
    }
  }
}

// writes the panel [k, k + w) that this band factored to memory for the other
// bands, from the band's buffers (owner_panel_warp): lane c column c of
// stage (row-major, nb per row, L11 with D on its diagonal, zeros above; so
// every store instruction covers one row of the block) and the pivot arrays;
// lane 0 then publishes the panel (fflag = epoch) once every lane's writes
// are ordered before it
template <typename T, int NBT>
__device__ __forceinline__ void publish_panel_warp(const SV &sv, int s, int k, int w, int nb, const T *Ls,
                                                   const T *pD0, const T *pD1, const int *pperm, const int *ptype,
                                                   unsigned *flag, unsigned epoch) {
  const int lane = threadIdx.x & 31;
  T *stage = (T *)sv.Ldg + (sv.piv_off[s] + k) * (int64_t)nb;
  if (lane < w) {
    const T dl = pD0[lane];
#pragma unroll 4
    for (int ii = 0; ii < w; ++ii) stage[(int64_t)ii * nb + lane] = ii == lane ? dl : Ls[lane * NBT + ii];
    const int64_t po = sv.piv_off[s] + k;
    sv.piv_type[po + lane] = ptype[lane];
    sv.piv_perm[po + lane] = pperm[lane];
    sv.D0[po + lane] = (double)dl;
    sv.D1[po + lane] = (double)pD1[lane];
  }
  __syncwarp();
  if (lane == 0) {
    __threadfence();
    st_release_flag(flag + k, epoch);
  }
}

// Rows of one panel [k, k + w): the band's rows i in [max(rb0, k + w), rb1),
// one row per thread (row rb0 + tid), in two phases.
//
// band_rows_left, per warp (needs only data final before the panel's
// diagonal block is factored): the warp's rows of the panel's columns,
// updated left-looking by the block's earlier panels,
// F21 -= W[rows, K0:k] L[k:k+w, K0:k]^T, into xs; the warp stages each
// 32-wide chunk of L in its own buffer Lpw (the next chunk, and the next
// chunk of W, loaded into registers while the current one is applied).
template <typename T, int NBT>
__device__ __forceinline__ void band_rows_left(const SV &sv, int s, int f, int K0, int k, int w, int rb0, int rb1,
                                               T *Lpw, T *xs) {
  using CT = T;
  constexpr int KC = 32, XS = PANEL_XS, LPER = KC * NBT / 32;
  const T *F = (const T *)sv.F + sv.front_off[s];
  const T *W = (const T *)sv.W + sv.w_off[s];
  const int64_t ldw = f - K0;
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t i = (int64_t)rb0 + tid;
  const bool row_ok = i >= k + w && i < rb1;
  const int kp_in = k - K0;
  {
    CT v[NBT];
#pragma unroll
    for (int t = 0; t < NBT; ++t) v[t] = (row_ok && t < w) ? (CT)__ldcg(F + i + (int64_t)(k + t) * f) : CT(0);
#pragma unroll
    for (int t = 0; t < NBT; ++t) xs[t * XS + tid] = v[t];
  }
  auto load_lp = [&](int cu, CT (&r)[LPER]) {
    const int kc = min(KC, kp_in - cu);
#pragma unroll
    for (int m = 0; m < LPER; ++m) {
      const int idx = lane + m * 32;
      const int u = idx / NBT, t = idx - u * NBT;
      r[m] = (u < kc && t < w) ? (CT)__ldcg(F + (int64_t)(k + t) + (int64_t)(K0 + cu + u) * f) : CT(0);
    }
  };
  CT lpr[LPER];
  if (kp_in > 0) load_lp(0, lpr);
  CT wr[KC];
#pragma unroll
  for (int u = 0; u < KC; ++u) wr[u] = (row_ok && u < kp_in) ? (CT)__ldcg(W + (i - K0) + (int64_t)u * ldw) : CT(0);
  for (int cu = 0; cu < kp_in; cu += KC) {
    __syncwarp();
#pragma unroll
    for (int m = 0; m < LPER; ++m) Lpw[lane + m * 32] = lpr[m];
    __syncwarp();
    if (cu + KC < kp_in) load_lp(cu + KC, lpr);
    CT wn[KC];
    const int nx = cu + KC;
#pragma unroll
    for (int u = 0; u < KC; ++u)
      wn[u] = (row_ok && nx + u < kp_in) ? (CT)__ldcg(W + (i - K0) + (int64_t)(nx + u) * ldw) : CT(0);
#pragma unroll 4
    for (int t0 = 0; t0 < NBT; t0 += 4) {
      CT acc[4] = {CT(0), CT(0), CT(0), CT(0)};
#pragma unroll
      for (int u = 0; u < KC; ++u) {
        CT lv[4];
        ld4(Lpw + u * NBT + t0, lv);
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] += wr[u] * lv[q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) xs[(t0 + q) * XS + tid] -= acc[q];
    }
#pragma unroll
    for (int u = 0; u < KC; ++u) wr[u] = wn[u];
  }
}

// band_rows_solve, the whole CTA, once the panel's diagonal block is
// published (and every warp with rows has run band_rows_left): permutation
// and forward substitution with L11 (x = F21 P^T L11^{-T} = L21 D); L21 =
// x D^{-1}.  Writes L21 to the front and x to the block's W, leaves both in
// xs / xw for the operand copies (band_row_copies), and applies the panel to
// the diagonal blocks of the later panels in the band (the next panel's one
// also to anext, unless null).  Reads of data other
// CTAs wrote go through L2 (ld.global.cg).
template <typename T, int NBT>
__device__ __forceinline__ void band_rows_solve(const SV &sv, int s, int f, int ns, int K0, int k, int w, int nb,
                                                int rb0, int rb1, T *L11T, T *xs, T *xw, T *sD0, T *sD1, T *sI0,
                                                T *sI1, int *sperm, int *stype, bool own, T (*anext)[NBT + 1]) {
  using CT = T;
  constexpr int XS = PANEL_XS;
  T *F = (T *)sv.F + sv.front_off[s];
  T *W = (T *)sv.W + sv.w_off[s];
  const int64_t ldw = f - K0;
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)rb0 + tid;
  const bool row_ok = i >= k + w && i < rb1;
  const T *stage = (const T *)sv.Ldg + (sv.piv_off[s] + k) * (int64_t)nb;
  if (!own) {  // a band that factored the panel has L11 and the pivots here already
    constexpr int PER = (NBT * NBT + 127) / 128;
    CT lt[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = tid + q * 128;
      const int c = idx / NBT, t = idx - c * NBT;
      lt[q] = (idx < NBT * NBT && c < t && t < w) ? (CT)__ldcg(stage + (int64_t)t * nb + c) : CT(0);
    }
    const int64_t po = sv.piv_off[s] + k;
    if (tid < NBT) {
      const bool in = tid < w;
      sD0[tid] = in ? (CT)__ldcg(sv.D0 + po + tid) : CT(1);
      sD1[tid] = in ? (CT)__ldcg(sv.D1 + po + tid) : CT(0);
      sperm[tid] = in ? __ldcg(sv.piv_perm + po + tid) : tid;
      stype[tid] = in ? __ldcg(sv.piv_type + po + tid) : 0;
    }
#pragma unroll
    for (int q = 0; q < PER; ++q)
      if (tid + q * 128 < NBT * NBT) L11T[tid + q * 128] = lt[q];
    __syncthreads();
    // D^{-1} per pivot: 1 / d for 1x1, the inverse of the 2x2 block for pairs
    // (entry (0,0) in sI0 of the first, (1,1) in sI0 of the second, (0,1) in sI1)
    if (tid < NBT) {
      const int t = tid;
      CT i0 = CT(1), i1 = CT(0);
      if (stype[t] == 0) {
        i0 = CT(1) / sD0[t];
      } else {
        const int a = stype[t] == 1 ? t : t - 1;
        const CT d11 = sD0[a], d21 = sD1[a], d22 = sD0[a + 1];
        const CT det = d11 * d22 - d21 * d21;
        i0 = (stype[t] == 1 ? d22 : d11) / det;
        i1 = -d21 / det;
      }
      sI0[t] = i0;
      sI1[t] = i1;
    }
    __syncthreads();
  }
  // permutation and forward substitution, x in registers
  CT x[NBT];
#pragma unroll
  for (int t = 0; t < NBT; ++t) x[t] = (row_ok && t < w) ? xs[sperm[t] * XS + tid] : CT(0);
#pragma unroll
  for (int c = 0; c < NBT - 1; ++c) {
    const CT xc = x[c];
#pragma unroll
    for (int t0 = ((c + 1) / 4) * 4; t0 < NBT; t0 += 4) {
      CT lv[4];
      ld4(L11T + c * NBT + t0, lv);
#pragma unroll
      for (int q = 0; q < 4; ++q) x[t0 + q] -= lv[q] * xc;
    }
  }
  // x = L21 D: to the outer block's W; L21 = x D^{-1} to the front
  if (row_ok) {
#pragma unroll
    for (int t = 0; t < NBT; ++t) {
      if (t >= w) break;
      W[(i - K0) + (int64_t)(k - K0 + t) * ldw] = T(x[t]);
      CT l;
      if (stype[t] == 0) {
        l = x[t] * sI0[t];
      } else if (stype[t] == 1) {  // first of a 2x2 pair (t + 1 < w)
        const int tn = t + 1 < NBT ? t + 1 : t;
        l = x[t] * sI0[t] + x[tn] * sI1[t];
      } else {
        const int tp = t > 0 ? t - 1 : 0;
        l = x[tp] * sI1[t] + x[t] * sI0[t];
      }
      F[i + (int64_t)(k + t) * f] = T(l);
      xs[t * XS + tid] = l;
      xw[t * XS + tid] = x[t];
    }
  }
  __syncthreads();
  {
    // rows of later panels of this block (bands 0 and 1): apply this panel's
    // contribution to their panel's diagonal block right away,
    // A(i, j) -= sum_t W(i, t) L(j, t) for rows i >= j of one panel; both
    // rows belong to this band (panels are nb-aligned from K0, bands
    // 128-aligned, nb divides 128), their L in xs, W in xw
    const int kend_blk = min(K0 + FACTOR_BLOCK, ns);
    if (row_ok && i < kend_blk) {
      const int pa = K0 + ((int)(i - K0) / nb) * nb;  // first row of the panel holding row i
      const int pl = pa - rb0;                         // its local row in the band
      const int ni = (int)i - pa;                      // columns pa .. i: ni + 1 of them
      CT cur[NBT];
#pragma unroll
      for (int q = 0; q < NBT; ++q) cur[q] = q <= ni ? (CT)__ldcg(F + i + (int64_t)(pa + q) * f) : CT(0);
#pragma unroll 1
      for (int t = 0; t < w; ++t) {
        const CT xt = xw[t * XS + tid];
        const T *lt = xs + t * XS + pl;  // 16-byte aligned (XS, pl multiples of 4)
#pragma unroll
        for (int q0 = 0; q0 < NBT; q0 += 4) {
          CT lv[4];
          ld4(lt + q0, lv);
#pragma unroll
          for (int u = 0; u < 4; ++u) cur[q0 + u] -= xt * lv[u];
        }
      }
#pragma unroll
      for (int q = 0; q < NBT; ++q)
        if (q <= ni) F[i + (int64_t)(pa + q) * f] = T(cur[q]);
      if (anext && pa == k + w) {  // the next panel's block, for its factorization in this CTA
#pragma unroll
        for (int q = 0; q < NBT; ++q)
          if (q <= ni) anext[q][ni] = T(cur[q]);
      }
    }
  }
  // every row's right-looking updates are in the front (the next panel's
  // diagonal block may be factored now); L and W of the rows in xs / xw
  __syncthreads();
}

// the K-major hi / lo operand copies of the calling warp's own 32 rows of a
// panel (FP32 fronts with tensor cores), from xs (L) and xw (W) as
// band_rows_solve left them, written warp-cooperatively (lanes along t)
template <typename T>
__device__ __forceinline__ void band_row_copies(const SV &sv, int s, int ns, int K0, int k, int w, int rb0, int rb1,
                                                const T *xs, const T *xw) {
  constexpr int XS = PANEL_XS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int wpad = (k + w == ns) ? ((k - K0 + w + 31) / 32) * 32 - (k - K0) : w;
  for (int pass = 0; pass < 2; ++pass) {
    const T *src = pass == 1 ? xw : xs;
    float *hi = pass == 1 ? sv.wk0 : sv.wk2, *lo = pass == 1 ? sv.wk1 : sv.wk3;
    // rows are FACTOR_BLOCK floats apart and k - K0, wpad are multiples of 4:
    // every lane stores 4 consecutive entries as one 16-byte vector
    const int q4 = wpad / 4;  // vectors per row
    const int rows_per_it = 32 / q4 > 0 ? 32 / q4 : 1;
    const int sub = lane / q4, t4 = (lane % q4) * 4;
    for (int rr = 0; rr < 32; rr += rows_per_it) {
      const int rloc = warp * 32 + rr + sub;
      const int64_t ig = (int64_t)rb0 + rloc;
      if (sub >= rows_per_it || rr + sub >= 32 || ig < k + w || ig >= rb1) continue;
      const int64_t base = sv.w_off[s] + ig * FACTOR_BLOCK + (k - K0);
      for (int t = t4; t < wpad; t += 4 * q4) {
        float v[4], h[4], l[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          v[q] = t + q < w ? (float)src[(t + q) * XS + rloc] : 0.f;
          h[q] = tc::tf32_hi(v[q]);
          l[q] = v[q] - h[q];
        }
        *reinterpret_cast<float4 *>(hi + base + t) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(lo + base + t) = make_float4(l[0], l[1], l[2], l[3]);
      }
    }
  }
}

template <typename T, int NBT>
__global__ void __launch_bounds__(128) k_block_panels(DevSym d, SV sv, const int32_t *__restrict__ fronts,
                                                      const BandItem *__restrict__ items, int K0, int nb,
                                                      double eps_rel, unsigned long long *counters, unsigned *ctl,
                                                      int *status) {
  extern __shared__ __align__(16) unsigned char rows_raw[];
  T *Lp = reinterpret_cast<T *>(rows_raw);  // [4 warps][32][NBT]
  T *L11T = Lp + 4 * 32 * NBT;               // [NBT][NBT]
  T *xs = L11T + NBT * NBT;                  // [NBT][PANEL_XS] + 4: L of the band's rows
  T *xw = xs + NBT * PANEL_XS + 4;           // [NBT][PANEL_XS] + 4: W of the band's rows
  __shared__ T a[2][NBT][NBT + 1];  // diagonal blocks of alternate panels
  __shared__ T bD0[32], bD1[32];  // the warp's Bunch-Kaufman writes 32 entries
  __shared__ __align__(16) T bU[32], bV[32];
  __shared__ int bperm[32], btype[32];
  __shared__ T sD0[NBT], sD1[NBT], sI0[NBT], sI1[NBT];
  __shared__ int sperm[NBT], stype[NBT];
  __shared__ int s_item, s_abort;
  const int tid = threadIdx.x;
  if (tid == 0) {
    s_item = (int)atomicAdd(&ctl[5], 1u);
    s_abort = 0;
    if (s_item >= (int)gridDim.x) {  // counters not reset by the previous launch
      atomicOr(status, DEV_TIMEOUT);
      s_abort = 1;
    } else if (*(volatile const int *)status & DEV_TIMEOUT) {
      s_abort = 1;
    }
  }
  __syncthreads();
  if (!s_abort) {
    const unsigned epoch = *(volatile const unsigned *)&ctl[4];
    const BandItem it = items[s_item];
    const int s = fronts[it.q];
    const int dpn = sv.dpn;
    const int ns = d.sn_nown[s] * dpn;
    const int f = front_order(d, s, dpn);
    const int kend = min(K0 + FACTOR_BLOCK, ns);
    const int rb0 = K0 + BAND * it.band, rb1 = min(rb0 + BAND, f);
    unsigned *flag = sv.fflag + sv.piv_off[s];
    unsigned *pre = sv.fpre + sv.piv_off[s];
    // The diagonal block of panel k is factored by warp 0 of the band holding
    // it as soon as the rows of the panel before it have updated it: after
    // the rows of panel k - w (iteration k - w); it first publishes that the
    // panel's rows are final in the block's earlier columns (pre).  Meanwhile
    // the other warps write those rows' operand copies and go on with the
    // left-looking phase of panel k, which needs only pre.  Warp 0 writes the
    // factored panel out for the other bands (and sets its fflag) after the
    // CTA's next barrier, so that the band's own solve of the panel's rows
    // does not wait for that.  Iteration K0 - nb has no rows and only factors
    // the first panel's block (band 0).
    const int warp = tid >> 5, lane = tid & 31;
    int pend = -1;  // warp 0: the panel factored here and not yet published
    auto publish = [&]() {
      if (pend >= 0)
        publish_panel_warp<T, NBT>(sv, s, pend, min(nb, ns - pend), nb, L11T, sD0, sD1, sperm, stype, flag, epoch);
      pend = -1;
    };
    for (int k = K0 - nb; k < kend; k += nb) {
      const int w = k < K0 ? nb : min(nb, ns - k);
      bool rows = false;
      if (k >= K0) {
        const bool owner = (k - K0) / BAND == it.band;
        if (!owner && rb1 <= k + w) break;  // no rows below this panel (nor below later ones)
        rows = rb1 > k + w;
        if (rows) {
          const int64_t wr0 = (int64_t)rb0 + warp * 32;  // the warp's first row
          if (wr0 + 31 >= k + w && wr0 < rb1) {
            // a band that does not own the panel waits until the panel's rows
            // are final in the earlier columns
            int ok = 1;
            if (!owner && k > K0 && lane == 0) ok = wait_epoch(pre + k, epoch, status);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (ok) band_rows_left<T, NBT>(sv, s, f, K0, k, w, rb0, rb1, Lp + warp * 32 * NBT, xs);
            else if (lane == 0) s_abort = 1;
          }
          // then for the panel itself: a band that owns it factored it in its
          // own warp 0, which reaches the __syncthreads below only after that
          if (!owner && tid == 0 && !s_abort && !wait_epoch(flag + k, epoch, status)) s_abort = 1;
          __syncthreads();
          if (warp == 0) publish();
          if (s_abort) break;
          const int kn = k + w;
          const bool next_here = kn < kend && (kn - K0) / BAND == it.band;
          band_rows_solve<T, NBT>(sv, s, f, ns, K0, k, w, nb, rb0, rb1, L11T, xs, xw, sD0, sD1, sI0, sI1, sperm,
                                  stype, owner, next_here ? a[((kn - K0) / nb) & 1] : nullptr);
        } else if (warp == 0) {
          publish();
        }
      }
      // the next panel's diagonal block lies in this band's rows when this
      // band owns that panel (warp 1 publishes that its rows are final in
      // the earlier columns, so that warp 0 starts at once)
      const int kn = k + w;
      const bool next_owner = kn < kend && (kn - K0) / BAND == it.band;
      if (next_owner && warp == 1 && lane == 0 && kn > K0) {
        __threadfence();
        st_release_flag(pre + kn, epoch);
      }
      if (next_owner && warp == 0) {
        owner_panel_warp<T, NBT>(sv, s, f, kn, min(nb, ns - kn), eps_rel, counters, a[((kn - K0) / nb) & 1],
                                 k >= K0, bD0, bD1, bperm, btype, bU, bV, L11T, sD0, sD1, sI0, sI1, sperm, stype);
        pend = kn;
      }
      if (rows && sv.wk0) band_row_copies<T>(sv, s, ns, K0, k, w, rb0, rb1, xs, xw);
    }
    if (warp == 0) publish();
  }
  // the last CTA to finish resets the ticket counters for the next launch
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(&ctl[6], 1u) == gridDim.x - 1) {
      atomicExch(&ctl[5], 0u);
      atomicExch(&ctl[6], 0u);
    }
  }
}

}  // namespace

template <typename T, int NBT>
void launch_block_panels(unsigned grid, size_t smem, cudaStream_t stream, const DevSym &d, const SV &sv,
                         const int32_t *fronts, const BandItem *items, int K0, int nb, double eps_rel,
                         unsigned long long *counters, unsigned *ctl, int *status) {
  k_block_panels<T, NBT><<<grid, 128, smem, stream>>>(d, sv, fronts, items, K0, nb, eps_rel, counters, ctl, status);
}

template <typename T, int NBT>
void set_block_panels_smem(int bytes) {
  cudaFuncSetAttribute(k_block_panels<T, NBT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace sgn
