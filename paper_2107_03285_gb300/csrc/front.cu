// Multifrontal LDL^T of the (p-eliminated) saddle-point system and of K, and
// the matching forward / diagonal / backward solves.
//
// Fronts are processed level by level of the elimination tree (all fronts of
// a level are independent).  A front of order f with ns fully-summed DOFs is
// a dense column-major f x f matrix (lower triangle used).  It is assembled
// by pulling (no atomics) the original entries of its own columns and the
// trailing (update) blocks of its children, then partially factored panel by
// panel (width nb, even):
//   1. diag:   Bunch-Kaufman (1x1 / 2x2, alpha = (1 + sqrt 17) / 8) on the
//              nb x nb diagonal block in FP64, pivot search restricted to the
//              panel; symmetric swaps are applied to the panel and to the
//              already factored rows of the front.
//   2. trsm:   W = F21 P^T L11^{-T} (= L21 D) and L21 = W D^{-1}, row-parallel.
//   3. update: F22 -= W L21^T on the lower triangle (tiled GEMM).
// Restricting the pivot search to a panel never needs delayed pivots here:
// every panel starts at an even DOF of the pair-interleaved order, so the
// matrix eliminated so far is a principal submatrix over whole (x, lambda)
// pairs, and every such submatrix [[A, K], [K, -G]] (K SPD, A, G PSD) is
// nonsingular; hence each panel's trailing block is nonsingular too.
#include <cmath>
#include <cstdio>
#include <functional>
#include <type_traits>

#include "common.cuh"
#include "front_view.cuh"
#include "tc_update.cuh"

namespace sgn {

namespace {

constexpr int MAXNB = 64;

// ---------------------------------------------------------------- assembly
// One CTA per (front, node column group P): zero the group's DPN columns,
// add the original entries of K (and, for the saddle-point store, A and -G)
// and extend-add the children's contribution blocks.  Column k of the group
// lives in one region (factor columns or contribution block), so it is
// addressed as region[off0_k + row] without a per-element test.
template <typename T, int D, int DPN>
__global__ void __launch_bounds__(256) k_front_assemble(DevSym d, SV sv, int64_t item_base,
                                                        const double *__restrict__ Kv,
                                                        const double *__restrict__ Gv,
                                                        const double *__restrict__ wA, double eps_x,
                                                        double eps_l) {
  const int64_t item = item_base + blockIdx.x;
  const int s = d.item_sn[item], P = d.item_P[item];
  const int nown = d.sn_nown[s];
  const int f = (nown + d.sn_nstruct[s]) * DPN;
  const FrontMat<T> F = front_mat<T>(d, sv, s);
  const int col0 = P * DPN;
  const bool in_cb = col0 >= F.ns;
  T *const R = in_cb ? F.C : F.L;
  int64_t off0[DPN];
#pragma unroll
  for (int k = 0; k < DPN; ++k)
    off0[k] = in_cb ? (int64_t)(col0 + k - F.ns) * (F.f - F.ns) - F.ns : (int64_t)(col0 + k) * F.f;
#pragma unroll
  for (int k = 0; k < DPN; ++k)
    for (int i = col0 + threadIdx.x; i < f; i += blockDim.x) R[off0[k] + i] = T(0);
  __syncthreads();
  if (P < nown) {
    const int r = d.sn_first[s] + P;
    const int k0 = d.bsr_ptr[r], nsl = d.bsr_ptr[r + 1] - k0;
    for (int idx = threadIdx.x; idx < nsl * D * D; idx += blockDim.x) {
      int sl = idx / (D * D), ab = idx - sl * D * D;
      int a = ab / D, b = ab - a * D;
      int kk = k0 + sl;
      int Q = d.bsr_orig_pos[kk];
      if (Q < 0) continue;
      double kv = Kv[(int64_t)kk * D * D + b * D + a];  // K[(c,a),(r,b)]
      if (sv.kkt) {
        int rx = Q * DPN + 2 * a, cx = P * DPN + 2 * b;
        double gv = Gv[(int64_t)kk * D * D + b * D + a];
        if (rx >= cx + 1) *F.at(rx, cx + 1) += T(kv);        // (x row, lambda col)
        if (rx + 1 >= cx) *F.at(rx + 1, cx) += T(kv);        // (lambda row, x col)
        if (rx + 1 >= cx + 1) *F.at(rx + 1, cx + 1) += T(-gv);
        // A on the x diagonal; the optional stabilization eps_x (x) and
        // -eps_l (lambda) of a preconditioning factor
        if (Q == P && a == b) {
          *F.at(rx, cx) += T(wA[(int64_t)r * D + a] + eps_x);
          if (eps_l != 0.0) *F.at(rx + 1, cx + 1) += T(-eps_l);
        }
      } else {
        int ri = Q * D + a, ci = P * D + b;
        if (ri >= ci) *F.at(ri, ci) += T(kv);
      }
    }
  }
  __syncthreads();
  const int coff = d.sn_child_off[s], nch = d.sn_nchild[s];
  for (int j = 0; j < nch; ++j) {
    const int c = d.children[coff + j];
    const int q = d.cmap[d.cmap_off[coff + j] + P];
    if (q >= 0) {
      const int nstc = d.sn_nstruct[c];
      const int fcb = nstc * DPN;  // the child's contribution block is fcb x fcb
      const T *Cc = (const T *)sv.CB + sv.cb_off[c];
      const int32_t *relc = d.relpos + d.sn_struct_off[c];
      const int rows = (nstc - q) * DPN;  // child rows q*DPN .. fcb-1 of its column q*DPN + k
#pragma unroll
      for (int k = 0; k < DPN; ++k) {
        const int64_t jc = (int64_t)q * DPN + k;
        const T *ccol = Cc + jc * fcb;
        for (int rr0 = threadIdx.x + k; rr0 < rows; rr0 += 4 * blockDim.x) {
          // rows rr >= k (lower triangle of the child's block: ic >= jc)
          T v[4], o[4];
          int64_t dst[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int rr = rr0 + u * blockDim.x;
            dst[u] = -1;
            v[u] = T(0);
            if (rr < rows) {
              const int qq = q + rr / DPN, kp = rr % DPN;
              dst[u] = off0[k] + (int64_t)relc[qq] * DPN + kp;
              v[u] = ccol[(int64_t)q * DPN + rr];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) o[u] = dst[u] >= 0 ? R[dst[u]] : T(0);
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (dst[u] >= 0) R[dst[u]] = o[u] + v[u];
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------- outer-block panel kernel
// One launch factors the pivot panels of one 256-column outer block [K0,
// kend) of every active front of a level.  Each CTA owns a band of 128 rows
// of one front (rows K0 + 128 b ...).  For every panel [k, k + w) in turn:
//   * the band holding the panel's diagonal rows (the owner) forms the
//     panel's diagonal block left-looking from the rows it factored itself
//     (A11 = F11 - W[k:k+w, K0:k] L[k:k+w, K0:k]^T), factors it with
//     Bunch-Kaufman in one warp, stages L11 / D / the permutation and
//     publishes the panel (a release store of the factorization's epoch);
//   * every band with rows below the panel waits (bounded) for that
//     publication, then updates its rows left-looking by the block's earlier
//     panels, permutes and solves them against L11 (W = L21 D and L21), and
//     writes the K-major hi / lo copies the tensor-core update reads.
// A CTA takes its (front, band) item by ticket; the items list every front's
// bands 0 and 1 (the only owners) before all other bands, so every CTA a
// band waits for has started before it.  A wait that expires records
// DEV_TIMEOUT and the CTA gives up.

constexpr int BAND = 128;                           // rows per CTA
constexpr long long PANEL_WAIT_CYCLES = 1ll << 31;  // ~1 s at 2 GHz

__device__ __forceinline__ unsigned ld_acquire_flag(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_flag(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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
__device__ __forceinline__ bool ge_alpha(float a, float c) {
  const float r = 0.64038820f * c;
  const float g = a - r;
  if (fabsf(g) > 0x1p-20f * fmaxf(a, r)) return g > 0.f;
  return (double)a >= BK_ALPHA * (double)c;
}
__device__ __forceinline__ bool ge_alpha(double a, double c) { return a >= BK_ALPHA * c; }
__device__ __forceinline__ bool ge_alpha_sq(float a, float r, float c) {
  const float lhs = a * r, rhs = (0.64038820f * c) * c;
  const float g = lhs - rhs;
  if (fabsf(g) > 0x1p-20f * fmaxf(lhs, rhs)) return g > 0.f;
  return (double)a * (double)r >= BK_ALPHA * ((double)c * (double)c);
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

// Bunch-Kaufman LDL^T of the w x w block a (w <= 32; a[j][i] = A(i, j), lower
// triangle) by one warp, lane i holding row i: 1x1 / 2x2 pivots, alpha =
// (1 + sqrt 17) / 8, pivot search restricted to the block, eliminations in
// CT, magnitudes compared exactly (max of |CT| values), pivot tests decided
// as in FP64 (ge_alpha, ge_alpha_sq) in lane 0.  On return column j of a
// holds W(:, j) = L(:, j) D_j unscaled, sD0 / sD1 (32 entries) the 1x1 and
// 2x2 pivots (a 1x1 pivot below the static-pivot threshold replaced), stype
// their kinds (0: 1x1, 1 / 2: first / second of a pair) and sperm the
// block's permutation (position -> original index).
template <typename CT, int PITCH>
__device__ void bk_factor_warp(CT (*a)[PITCH], const int w, const double eps_rel, int *sperm, int *stype,
                               CT *sD0, CT *sD1, CT *su, CT *sv, unsigned long long *counters) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  sperm[lane] = lane; stype[lane] = 0; sD0[lane] = CT(0); sD1[lane] = CT(0);
  CT bm = CT(0);
  for (int jj = 0; jj < w; ++jj)
    if (lane >= jj && lane < w) bm = max(bm, (CT)fabs(a[jj][lane]));
  bm = warp_max0(bm);
  const double thresh = eps_rel * fmax((double)bm, 1e-300);
  // the largest CT not above thresh: |x| > thresh  <=>  |x| > thresh_c
  CT thresh_c = (CT)thresh;
  if ((double)thresh_c > thresh) thresh_c = nextafter(thresh_c, CT(0));
  const CT thresh_v = (CT)thresh;  // the static pivot's magnitude
  __syncwarp();
  unsigned long long n_pert = 0, n_pair = 0;  // counted in lane 0, added once at the end
  (void)su; (void)sv;
  int j = 0;
  while (j < w) {
    // ---- pivot search: largest |A(i, j)|, i > j (ties to the lowest index)
    CT cm;
    int imax;
    const bool below = lane > j && lane < w;
    warp_argmax(below ? (CT)fabs(a[j][lane]) : CT(0), below, w, cm, imax);
    const CT akk = a[j][j];
    const CT colmax = max(cm, CT(0)), absakk = (CT)fabs(akk);
    // every lane takes the same decisions on the same (warp-uniform) values,
    // so no broadcast is needed; 0: 1x1 at j, 1: needs the row of imax
    const int code = (!(max(absakk, colmax) > thresh_c) || ge_alpha(absakk, colmax)) ? 0 : 1;
    int kstep = 1, kp = j;
    if (code == 1) {
      // largest off-diagonal |A(imax, t)|, t in [j, w), t != imax
      CT rm = CT(0);
      if (lane >= j && lane < w && lane != imax) rm = (CT)(lane < imax ? fabs(a[lane][imax]) : fabs(a[imax][lane]));
      rm = warp_max0(rm);
      const CT aii = (CT)fabs(a[imax][imax]);
      // 0: 1x1 at j, 1: 1x1 at imax, 2: 2x2 with imax
      const int dec = ge_alpha_sq(absakk, rm, colmax) ? 0 : (ge_alpha(aii, rm) ? 1 : 2);
      if (dec == 1) { kstep = 1; kp = imax; }
      else if (dec == 2) { kstep = 2; kp = imax; }
    }
    const int kk = j + kstep - 1;
    __syncwarp();
    if (kp != kk) {
      // symmetric interchange of kk and kp (> kk) in the trailing lower
      // triangle and in the already eliminated part of both rows
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
      __syncwarp();
    }
    if (kstep == 1) {
      CT dj = a[j][j];
      const bool perturb = !(fabs(dj) > thresh_c);
      if (perturb) dj = (dj >= CT(0)) ? thresh_v : -thresh_v;
      if (lane == 0) {
        sD0[j] = dj; stype[j] = 0;
        if (perturb) ++n_pert;
      }
      const CT rd = CT(1) / dj;
      const CT l = (lane > j && lane < w) ? a[j][lane] : CT(0);
      const CT lr = l * rd;
      // every column cc > j of row lane at once: all loads first, the
      // multipliers by shuffles, then the stores (unrolled, predicated)
      const int row = lane < w ? lane : 0;
      CT av[32];
#pragma unroll
      for (int cc = 0; cc < 32; ++cc) av[cc] = cc < PITCH - 1 ? a[cc < PITCH - 1 ? cc : 0][row] : CT(0);
#pragma unroll
      for (int cc = 0; cc < 32; ++cc) {
        const CT m = __shfl_sync(FULL, lr, cc);
        if (cc > j && cc <= lane && lane < w) a[cc < PITCH - 1 ? cc : 0][lane] = av[cc] - l * m;
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
      const CT u = in ? a[j][lane] : CT(0), v = in ? a[j + 1][lane] : CT(0);
      const CT p = u * i11 + v * i21, q = u * i21 + v * i22;  // (L1, L2) of row lane
      const int row = lane < w ? lane : 0;
      CT av[32];
#pragma unroll
      for (int cc = 0; cc < 32; ++cc) av[cc] = cc < PITCH - 1 ? a[cc < PITCH - 1 ? cc : 0][row] : CT(0);
#pragma unroll
      for (int cc = 0; cc < 32; ++cc) {
        const CT w1 = __shfl_sync(FULL, u, cc), w2 = __shfl_sync(FULL, v, cc);
        if (cc > j + 1 && cc <= lane && lane < w) a[cc < PITCH - 1 ? cc : 0][lane] = av[cc] - (p * w1 + q * w2);
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

// L(i, j) (i > j) of a block factored by bk_factor_warp, from its unscaled
// columns and pivots: a 1x1 column is divided by its pivot, a 2x2 pair is
// multiplied by the pair's inverse; L is zero inside a 2x2 pivot
template <typename CT, int PITCH>
__device__ __forceinline__ CT bk_unit_lower(const CT (*a)[PITCH], int i, int j, const int *stype, const CT *sD0,
                                            const CT *sD1) {
  const int ty = stype[j];
  if (ty == 0) return a[j][i] * (CT(1) / sD0[j]);
  const int j0 = ty == 1 ? j : j - 1;  // first column of the pair
  if (i == j0 + 1) return CT(0);
  const CT d11 = sD0[j0], d21 = sD1[j0], d22 = sD0[j0 + 1];
  const CT det = d11 * d22 - d21 * d21;
  const CT i11 = d22 / det, i21 = -d21 / det, i22 = d11 / det;
  const CT u = a[j0][i], v = a[j0 + 1][i];
  return ty == 1 ? u * i11 + v * i21 : u * i21 + v * i22;
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

// the panel's diagonal block, already updated by every earlier panel (the
// band holding it applied those updates right-looking, band_panel_rows),
// factored by warp 0; stage (L11 with D on its diagonal) and the pivot
// arrays are written for the bands
template <typename T, int NBT>
__device__ void owner_panel(const DevSym &d, const SV &sv, int s, int f, int k, int w, int nb, double eps_rel,
                            unsigned long long *counters, T (*a)[NBT + 1], T *sD0, T *sD1, int *sperm, int *stype,
                            T *su, T *svv) {
  const int tid = threadIdx.x;
  const T *F = (const T *)sv.F + sv.front_off[s];
  __syncthreads();  // the band's right-looking updates of this block are complete
  for (int idx = tid; idx < NBT * NBT; idx += blockDim.x) {
    const int jj = idx / NBT, ii = idx - jj * NBT;
    a[jj][ii] = (ii >= jj && ii < w) ? __ldcg(F + (int64_t)(k + ii) + (int64_t)(k + jj) * f) : T(0);
  }
  __syncthreads();
  if (tid < 32) bk_factor_warp<T, NBT + 1>(a, w, eps_rel, sperm, stype, sD0, sD1, su, svv, counters);
  __syncthreads();
  T *stage = (T *)sv.Ldg + (sv.piv_off[s] + k) * (int64_t)nb;
  for (int idx = tid; idx < w * w; idx += blockDim.x) {
    const int jj = idx / w, ii = idx - jj * w;
    if (ii >= jj)
      stage[(int64_t)ii * nb + jj] = (ii == jj) ? sD0[jj] : bk_unit_lower<T, NBT + 1>(a, ii, jj, stype, sD0, sD1);
  }
  const int64_t po = sv.piv_off[s] + k;
  if (tid < w) {
    sv.piv_type[po + tid] = stype[tid];
    sv.piv_perm[po + tid] = sperm[tid];
    sv.D0[po + tid] = (double)sD0[tid];
    sv.D1[po + tid] = (double)sD1[tid];
  }
}

// one panel [k, k + w) of the band's rows i in [max(rb0, k + w), rb1), one
// row per thread (row rb0 + tid): left-looking update by the earlier panels
// of the block, F21 -= W[rows, K0:k] L[k:k+w, K0:k]^T (the next chunk of W
// prefetched while the current one is applied); permutation and forward
// substitution with L11 (x = F21 P^T L11^{-T} = L21 D); L21 = x D^{-1}.
// Writes L21 to the front, x to the block's W and (FP32 fronts with tensor
// cores) both as K-major hi / lo operand copies.  Reads of data other CTAs
// wrote go through L2 (ld.global.cg).
template <typename T, int NBT>
__device__ void band_panel_rows(const DevSym &d, const SV &sv, int s, int f, int ns, int K0, int k, int w, int nb,
                                int rb0, int rb1, T *Lp, T *L11T, T *xs, T *sD0, T *sD1, T *sI0, T *sI1,
                                int *sperm, int *stype) {
  using CT = T;
  constexpr int RB = BAND, KC = 32, XS = RB + 1;
  T *F = (T *)sv.F + sv.front_off[s];
  T *W = (T *)sv.W + sv.w_off[s];
  const int64_t ldw = f - K0;
  const int tid = threadIdx.x;
  const int64_t i = (int64_t)rb0 + tid;
  const bool row_ok = i >= k + w && i < rb1;
  const int kp_in = k - K0;
  const T *stage = (const T *)sv.Ldg + (sv.piv_off[s] + k) * (int64_t)nb;
  __syncthreads();  // the shared buffers may still be read by the previous panel
  {
    CT v[NBT];
#pragma unroll
    for (int t = 0; t < NBT; ++t) v[t] = (row_ok && t < w) ? (CT)__ldcg(F + i + (int64_t)(k + t) * f) : CT(0);
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
#pragma unroll
    for (int t = 0; t < NBT; ++t) xs[t * XS + tid] = v[t];
  }
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
  // left-looking update; the next chunk of L (and of W) is loaded into
  // registers while the current one is applied
  constexpr int LPER = KC * NBT / 128;
  auto load_lp = [&](int cu, CT (&r)[LPER]) {
    const int kc = min(KC, kp_in - cu);
#pragma unroll
    for (int m = 0; m < LPER; ++m) {
      const int idx = tid + m * 128;
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
    __syncthreads();
#pragma unroll
    for (int m = 0; m < LPER; ++m) Lp[tid + m * 128] = lpr[m];
    __syncthreads();
    if (cu + KC < kp_in) load_lp(cu + KC, lpr);
    CT wn[KC];
    const int nx = cu + KC;
#pragma unroll
    for (int u = 0; u < KC; ++u)
      wn[u] = (row_ok && nx + u < kp_in) ? (CT)__ldcg(W + (i - K0) + (int64_t)(nx + u) * ldw) : CT(0);
    if (row_ok) {
#pragma unroll 4
      for (int t0 = 0; t0 < NBT; t0 += 4) {
        CT acc[4] = {CT(0), CT(0), CT(0), CT(0)};
#pragma unroll
        for (int u = 0; u < KC; ++u) {
          CT lv[4];
          ld4(Lp + u * NBT + t0, lv);
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] += wr[u] * lv[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) xs[(t0 + q) * XS + tid] -= acc[q];
      }
    }
#pragma unroll
    for (int u = 0; u < KC; ++u) wr[u] = wn[u];
  }
  __syncthreads();
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
    }
  }
  __syncthreads();
  {
    // rows of later panels of this block (bands 0 and 1): apply this panel's
    // contribution to their panel's diagonal block right away,
    // A(i, j) -= sum_t W(i, t) L(j, t) for rows i >= j of one panel; both
    // rows belong to this band (panels are nb-aligned from K0, bands
    // 128-aligned, nb divides 128), their L in xs, W(i, .) in x
    const int kend_blk = min(K0 + FACTOR_BLOCK, ns);
    if (row_ok && i < kend_blk) {
      const int pa = K0 + ((int)(i - K0) / nb) * nb;  // first row of the panel holding row i
      const int pl = pa - rb0;                         // its local row in the band
      const int ni = (int)i - pa;                      // columns pa .. i: ni + 1 of them
      CT cur[NBT];
#pragma unroll
      for (int q = 0; q < NBT; ++q) cur[q] = q <= ni ? (CT)__ldcg(F + i + (int64_t)(pa + q) * f) : CT(0);
#pragma unroll
      for (int t = 0; t < NBT; ++t) {
        if (t >= w) break;
        const CT xt = x[t];
#pragma unroll
        for (int q = 0; q < NBT; ++q) cur[q] -= xt * xs[t * XS + min(pl + q, RB - 1)];
      }
#pragma unroll
      for (int q = 0; q < NBT; ++q)
        if (q <= ni) F[i + (int64_t)(pa + q) * f] = T(cur[q]);
    }
  }
  if (sv.wk0) {
    // K-major hi / lo copies, written warp-cooperatively (lanes along t):
    // first L (already in xs), then W
    const int warp = tid >> 5, lane = tid & 31;
    const int wpad = (k + w == ns) ? ((k - K0 + w + 31) / 32) * 32 - (k - K0) : w;
    for (int pass = 0; pass < 2; ++pass) {
      __syncthreads();
      if (pass == 1 && row_ok) {
#pragma unroll
        for (int t = 0; t < NBT; ++t) {
          if (t >= w) break;
          xs[t * XS + tid] = x[t];
        }
      }
      __syncthreads();
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
            v[q] = t + q < w ? (float)xs[(t + q) * XS + rloc] : 0.f;
            h[q] = tc::tf32_hi(v[q]);
            l[q] = v[q] - h[q];
          }
          *reinterpret_cast<float4 *>(hi + base + t) = make_float4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<float4 *>(lo + base + t) = make_float4(l[0], l[1], l[2], l[3]);
        }
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
  T *Lp = reinterpret_cast<T *>(rows_raw);  // [32][NBT]
  T *L11T = Lp + 32 * NBT;                   // [NBT][NBT]
  T *xs = L11T + NBT * NBT;                  // [NBT][129]
  __shared__ T a[NBT][NBT + 1];
  __shared__ T bD0[32], bD1[32], bU[32], bV[32];  // the warp's Bunch-Kaufman writes 32 entries
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
    for (int k = K0; k < kend; k += nb) {
      const int w = min(nb, ns - k);
      const bool owner = (k - K0) / BAND == it.band;
      if (!owner && rb1 <= k + w) break;  // no rows below this panel (nor below later ones)
      if (owner) {
        owner_panel<T, NBT>(d, sv, s, f, k, w, nb, eps_rel, counters, a, bD0, bD1, bperm, btype, bU, bV);
        __syncthreads();
        if (tid == 0) {
          __threadfence();
          st_release_flag(flag + k, epoch);
        }
      } else {
        if (tid == 0 && ld_acquire_flag(flag + k) != epoch) {
          const long long t0 = clock64();
          for (int n = 1; ld_acquire_flag(flag + k) != epoch; ++n) {
            if ((n & 255) == 0 &&
                ((*(volatile const int *)status & DEV_TIMEOUT) || clock64() - t0 > PANEL_WAIT_CYCLES)) {
              atomicOr(status, DEV_TIMEOUT);
              s_abort = 1;
              break;
            }
          }
        }
        __syncthreads();
        if (s_abort) break;
      }
      if (rb1 > k + w)
        band_panel_rows<T, NBT>(d, sv, s, f, ns, K0, k, w, nb, rb0, rb1, Lp, L11T, xs, sD0, sD1, sI0, sI1, sperm,
                                stype);
    }
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

// a new factorization: a new epoch for the panel flags, ticket counters cleared
__global__ void k_factor_begin(unsigned *ctl) {
  ctl[4] += 1u;
  ctl[5] = 0u;
  ctl[6] = 0u;
}

// applies the pivot permutations of the panels of the outer block [K0, kend)
// to the already factored columns left of each panel, so that L ends up in
// the final (pivoted) row order.  Deferring this to the end of the block is
// valid: inside the block, a panel only ever reads the rows of its own and
// later panels, never rows of an earlier panel in earlier columns.
template <typename T>
__global__ void __launch_bounds__(256) k_row_swap(DevSym d, SV sv, const int32_t *__restrict__ fronts, int K0, int NB,
                                                   int nb) {
  __shared__ T buf[MAXNB][65];
  const int s = fronts[blockIdx.y];
  const int dpn = sv.dpn;
  const int ns = d.sn_nown[s] * dpn;
  if (K0 >= ns) return;
  const int f = front_order(d, s, dpn);
  const int kend = min(K0 + NB, ns);
  const int c0 = blockIdx.x * 64;
  if (c0 >= kend) return;
  T *F = (T *)sv.F + sv.front_off[s];
  const int32_t *perm = sv.piv_perm + sv.piv_off[s];
  const int tid = threadIdx.x;
  if (blockIdx.x == 0) {
    // the factored diagonal blocks of this outer block's panels
    for (int k = K0; k < kend; k += nb) {
      const int w = min(nb, ns - k);
      const T *stage = (const T *)sv.Ldg + (sv.piv_off[s] + k) * (int64_t)nb;
      for (int idx = tid; idx < w * w; idx += blockDim.x) {
        const int jj = idx / w, ii = idx - jj * w;
        if (ii >= jj) F[(int64_t)(k + ii) + (int64_t)(k + jj) * f] = stage[(int64_t)ii * nb + jj];
      }
    }
  }
  for (int k = K0; k < kend; k += nb) {
    // panel [k, k + w) needs columns [c0, min(c0 + 64, k))
    if (k <= c0) continue;
    const int w = min(nb, ns - k);
    const int cw = min(64, k - c0);
    __syncthreads();
    for (int base = tid; base < w * cw; base += 8 * blockDim.x) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * blockDim.x;
        const int cc = idx / w, t = idx - cc * w;
        v[u] = idx < w * cw ? F[(int64_t)(k + perm[k + t]) + (int64_t)(c0 + cc) * f] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = base + u * blockDim.x;
        if (idx < w * cw) buf[idx % w][idx / w] = v[u];
      }
    }
    __syncthreads();
    for (int idx = tid; idx < w * cw; idx += blockDim.x) {
      int cc = idx / w, t = idx - cc * w;
      F[(int64_t)(k + t) + (int64_t)(c0 + cc) * f] = buf[t][cc];
    }
  }
}

// C -= A B^T on a 64 x 64 output tile, 4 x 4 per thread, K staged in chunks
// of 32: A(r, t) = A[r + t * lda] (r < ma), B(c, t) = B[c + t * ldb] (c < nbc);
// C(r, c) is front element (row0 + r, col0 + c); only entries with
// row + roff >= col (lower triangle) are written
template <typename T>
__device__ __forceinline__ void tile_gemm_sub(const FrontMat<T> &Fm, int64_t row0, int64_t col0,
                                              const T *__restrict__ A, int64_t lda, int ma, const T *__restrict__ B,
                                              int64_t ldb, int nbc, int kk, int roff) {
  constexpr int KC = 32;
  __shared__ T As[KC][64];
  __shared__ T Bs[KC][64];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int n = 0; n < 4; ++n) acc[m][n] = T(0);
  for (int t0 = 0; t0 < kk; t0 += KC) {
    const int kc = min(KC, kk - t0);
    __syncthreads();
    {
      T va[8], vb[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = tid + u * 256;
        const int t = idx >> 6, ii = idx & 63;
        const bool ok = t < kc;
        va[u] = (ok && ii < ma) ? A[ii + (int64_t)(t0 + t) * lda] : T(0);
        vb[u] = (ok && ii < nbc) ? B[ii + (int64_t)(t0 + t) * ldb] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int idx = tid + u * 256;
        As[idx >> 6][idx & 63] = va[u];
        Bs[idx >> 6][idx & 63] = vb[u];
      }
    }
    __syncthreads();
    for (int t = 0; t < kc; ++t) {
      T av[4], bv[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) av[m] = As[t][tx + 16 * m];
#pragma unroll
      for (int n = 0; n < 4; ++n) bv[n] = Bs[t][ty + 16 * n];
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int n = 0; n < 4; ++n) acc[m][n] = fma(av[m], bv[n], acc[m][n]);
    }
  }
  // all 16 loads first, then the stores (distinct addresses)
  T cur[4][4];
  T *cp[4][4];
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const int jl = ty + 16 * n;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int il = tx + 16 * m;
      const bool ok = jl < nbc && il < ma && il + roff >= jl;
      cp[m][n] = ok ? Fm.at(row0 + il, col0 + jl) : nullptr;
      cur[m][n] = ok ? *cp[m][n] : T(0);
    }
  }
#pragma unroll
  for (int n = 0; n < 4; ++n)
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (cp[m][n]) *cp[m][n] = cur[m][n] - acc[m][n];
}

// trailing update after the outer block [K0, kend):
// F[kend:, kend:] -= W[kend:, block] L[kend:, block]^T (lower triangle)
template <typename T>
__global__ void __launch_bounds__(256) k_update(DevSym d, SV sv, const int32_t *__restrict__ fronts, int K0,
                                                 int NB) {
  const int s = fronts[blockIdx.y];
  const int dpn = sv.dpn;
  const int ns = d.sn_nown[s] * dpn;
  if (K0 >= ns) return;
  const int f = front_order(d, s, dpn);
  const int kend = min(K0 + NB, ns);
  const int kw = kend - K0;
  const int nrows = f - kend;
  const int nt = (nrows + 63) / 64;
  const int tile = blockIdx.x;
  if (tile >= nt * (nt + 1) / 2) return;
  int bi = (int)((sqrt(8.0 * tile + 1.0) - 1.0) * 0.5);
  while ((bi + 1) * (bi + 2) / 2 <= tile) ++bi;
  while (bi * (bi + 1) / 2 > tile) --bi;
  const int bj = tile - bi * (bi + 1) / 2;
  const FrontMat<T> Fm = front_mat<T>(d, sv, s);
  const T *W = (const T *)sv.W + sv.w_off[s];
  const int64_t ldw = f - K0;
  const int r = bi * 64, cc = bj * 64;
  tile_gemm_sub<T>(Fm, kend + r, kend + cc, W + (kend - K0 + r), ldw, min(64, nrows - r),
                   Fm.L + (int64_t)(kend + cc) + (int64_t)K0 * f, f, min(64, nrows - cc), kw, r - cc);
}

// persistent tensor-core trailing update: CTA x of front y walks tiles
// x, x + gridDim.x, ... of the window of tile columns [win0, win1) (win1 < 0:
// to the end) of that front's lower triangle
__global__ void __launch_bounds__(tc::PTHREADS, 1) k_update_tcp(DevSym d, SV sv, const int32_t *__restrict__ fronts,
                                                                 int K0, int NB, const tc::Maps *__restrict__ maps,
                                                                 int win0, int win1, int *status) {
  const int s = fronts[blockIdx.y];
  const int dpn = sv.dpn;
  const int ns = d.sn_nown[s] * dpn;
  if (K0 >= ns) return;
  const int f = front_order(d, s, dpn);
  const int kend = min(K0 + NB, ns);
  const int nrows = f - kend;
  const int nt = (nrows + tc::TILE - 1) / tc::TILE;
  tc::TileJob job;
  job.win0 = win0;
  job.m = min(win1 < 0 ? nt : win1, nt) - win0;
  if (job.m <= 0) return;
  const int n = nt - win0;  // tile rows of the window
  job.ntiles = job.m * (job.m + 1) / 2 + (n - job.m) * job.m;
  if ((int)blockIdx.x >= job.ntiles) return;
  job.L = (float *)sv.F + sv.front_off[s];
  job.CB = (float *)sv.CB + sv.cb_off[s];
  job.f = f;
  job.ns = ns;
  job.nrows = nrows;
  job.kend = kend;
  job.kchunks = (kend - K0 + 31) / 32;
  tc::tile_loop_tc(&maps[s], job, blockIdx.x, gridDim.x, status, DEV_TIMEOUT);
}


__global__ void k_pivot_counts(int64_t n, const int32_t *__restrict__ type, const double *__restrict__ D0,
                               const double *__restrict__ D1, unsigned long long *counters) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  int ty = type[t];
  unsigned long long pos = 0, neg = 0, zer = 0;
  if (ty == 0) {
    double v = D0[t];
    if (v > 0) pos = 1; else if (v < 0) neg = 1; else zer = 1;
  } else if (ty == 1) {
    double det = D0[t] * D0[t + 1] - D1[t] * D1[t];
    if (det < 0) { pos = 1; neg = 1; }
    else if (det > 0) { if (D0[t] > 0) pos = 2; else neg = 2; }
    else zer = 2;
  }
  if (pos) atomicAdd(counters + 2, pos);
  if (neg) atomicAdd(counters + 3, neg);
  if (zer) atomicAdd(counters + 4, zer);
}

// host helpers ---------------------------------------------------------------
struct LevelInfo {
  int64_t f0, f1;          // range in lvl_fronts
  int64_t i0, i1;          // item range
  std::vector<int> ns, f;  // per front (sorted order)
};

LevelInfo level_info(Ctx &c, int L, int dpn) {
  LevelInfo li;
  li.f0 = c.h_lvl_ptr[L]; li.f1 = c.h_lvl_ptr[L + 1];
  li.i0 = c.h_item_ptr[L]; li.i1 = c.h_item_ptr[L + 1];
  for (int s : c.S.level_fronts[L]) {
    li.ns.push_back(c.S.sn[s].nown * dpn);
    li.f.push_back(c.S.sn[s].fnodes() * dpn);
  }
  return li;
}

int n_active(const LevelInfo &li, int k) {
  int n = 0;
  while (n < (int)li.ns.size() && li.ns[n] > k) ++n;
  return n;
}

// SMs the rest of a split trailing update leaves to the next block's panels
constexpr int PANEL_RESERVE_SMS = 32;

template <typename T>
void factor_impl(Ctx &c, Store &st) {
  const SV sv0 = view(st);
  const int nb = c.S.opts.panel;
  const int D = c.S.dim;
  const double eps_rel = sizeof(T) == 8 ? 1e-14 : 1e-7;
  unsigned long long *ctr = (unsigned long long *)c.counters;
  cudaMemsetAsync(c.counters, 0, 8 * sizeof(int64_t), c.stream);
  // panel kernels compiled for 16 and 32 columns
  const int nbt = nb <= 16 ? 16 : 32;
  const size_t panels_smem = (size_t)(32 * nbt + nbt * nbt + nbt * 129) * sizeof(T);
  k_factor_begin<<<1, 1, 0, c.stream>>>(st.ctl);
  c.count();
  int64_t blk = 0;  // index into the store's per-(level, outer block) item ranges
  for (int L = 0; L < c.S.n_levels; ++L) {
    LevelInfo li = level_info(c, L, st.dpn);
    int64_t nitems = li.i1 - li.i0;
    {
      ProfScope ps(c, SGN_PROF_FRONT_ASSEMBLY);
      const dim3 ga((unsigned)nitems);
      const double ex = st.kkt ? st.eps_x : 0.0, el = st.kkt ? st.eps_l : 0.0;
      if (D == 2 && st.dpn == 4) k_front_assemble<T, 2, 4><<<ga, 256, 0, c.stream>>>(c.ds, sv0, li.i0, c.Kv, c.Gv, c.wA, ex, el);
      else if (D == 2) k_front_assemble<T, 2, 2><<<ga, 256, 0, c.stream>>>(c.ds, sv0, li.i0, c.Kv, c.Gv, c.wA, ex, el);
      else if (st.dpn == 6) k_front_assemble<T, 3, 6><<<ga, 256, 0, c.stream>>>(c.ds, sv0, li.i0, c.Kv, c.Gv, c.wA, ex, el);
      else k_front_assemble<T, 3, 3><<<ga, 256, 0, c.stream>>>(c.ds, sv0, li.i0, c.Kv, c.Gv, c.wA, ex, el);
      c.count();
    }
    const int32_t *fronts = c.ds.lvl_fronts + li.f0;
    int max_ns = li.ns.empty() ? 0 : li.ns[0];
    bool side_pending = false;  // the rest of the last trailing update runs on the side stream
    for (int K0 = 0; K0 < max_ns; K0 += FACTOR_BLOCK) {
      const int kstop = std::min(K0 + FACTOR_BLOCK, max_ns);
      const int parity = (K0 / FACTOR_BLOCK) & 1;  // which operand set this block writes
      const SV sv = view(st, parity);
      {
        // every panel of the block in one launch (one CTA per 128-row band)
        int na = n_active(li, K0);
        double fl = 0.0;
        for (int q = 0; q < na; ++q)
          for (int k = K0; k < std::min(K0 + FACTOR_BLOCK, li.ns[q]); k += nb) {
            const double w = std::min(nb, li.ns[q] - k), nr = li.f[q] - k;
            fl += 2.0 * (nr * w - w * (w - 1) / 2.0) * (k - K0);  // left-looking panel updates
          }
        const int64_t b0 = st.h_blk_off[blk], b1 = st.h_blk_off[blk + 1];
        ++blk;
        ProfScope ps(c, SGN_PROF_TRSM, fl);
        if (nbt == 16)
          k_block_panels<T, 16><<<(unsigned)(b1 - b0), 128, panels_smem, c.stream>>>(
              c.ds, sv, fronts, st.blk_items + b0, K0, nb, eps_rel, ctr, st.ctl, c.status);
        else
          k_block_panels<T, 32><<<(unsigned)(b1 - b0), 128, panels_smem, c.stream>>>(
              c.ds, sv, fronts, st.blk_items + b0, K0, nb, eps_rel, ctr, st.ctl, c.status);
        c.count();
      }
      int na = n_active(li, K0);
      {
        // the permutations of this block's panels (rows [K0, kend), columns
        // left of each panel): independent of the trailing update
        ProfScope ps(c, SGN_PROF_PIVOT);
        dim3 gs((kstop + 63) / 64, na);
        k_row_swap<T><<<gs, 256, 0, c.stream>>>(c.ds, sv, fronts, K0, FACTOR_BLOCK, nb);
        c.count();
      }
      int max_rows = 0;
      for (int q = 0; q < na; ++q) max_rows = std::max(max_rows, li.f[q] - std::min(K0 + FACTOR_BLOCK, li.ns[q]));
      if (max_rows > 0) {
        auto flops_cols = [&](int c0, int c1) {  // trailing-update flops of tile columns [c0, c1) (c1 < 0: all)
          double fl = 0.0;
          for (int q = 0; q < na; ++q) {
            const double kend = std::min(K0 + FACTOR_BLOCK, li.ns[q]), nr = li.f[q] - kend;
            const double a = std::min<double>(nr, (double)c0 * tc::TILE);
            const double b = c1 < 0 ? nr : std::min<double>(nr, (double)c1 * tc::TILE);
            if (b <= a) continue;
            // lower-triangle entries of columns [a, b): sum_{j=a}^{b-1} (nr - j)
            fl += 2.0 * (kend - K0) * ((b - a) * nr - (b * (b - 1) - a * (a - 1)) / 2.0);
          }
          return fl;
        };
        if (std::is_same<T, float>::value && st.tc) {
          // one CTA per SM (192 KB shared memory); spread the SMs over the
          // active fronts and let every CTA loop over its front's tiles.  The
          // tile columns holding the next outer block's columns go first on
          // this stream; the rest runs on the side stream, next to the next
          // block's panels (which write the other operand set), on fewer SMs
          // so that those panels find room
          const int nt128 = (max_rows + tc::TILE - 1) / tc::TILE;
          const int ctas = c.update_ctas > 0 ? c.update_ctas : c.num_sms;
          const int next_w = FACTOR_BLOCK / tc::TILE;
          const tc::Maps *maps = (const tc::Maps *)st.maps + (size_t)parity * c.S.sn.size();
          if (side_pending) cudaStreamWaitEvent(c.stream, c.ev_join, 0);  // the previous block's rest
          const bool split = nt128 > next_w && c.side_stream && K0 + FACTOR_BLOCK < max_ns;
          {
            const int m = std::min(next_w, nt128);
            const int tiles = m * (m + 1) / 2 + (nt128 - m) * m;
            int g = std::max(1, std::min(split ? tiles : nt128 * (nt128 + 1) / 2, (ctas + na - 1) / na));
            ProfScope ps(c, SGN_PROF_UPDATE, split ? flops_cols(0, next_w) : flops_cols(0, -1));
            k_update_tcp<<<dim3(g, na), tc::PTHREADS, tc::PSMEM_BYTES, c.stream>>>(
                c.ds, sv, fronts, K0, FACTOR_BLOCK, maps, 0, split ? next_w : -1, c.status);
            c.tc_launches++;
            c.count();
          }
          if (split) {
            cudaEventRecord(c.ev_fork, c.stream);
            cudaStream_t main = c.stream;
            c.stream = c.side_stream;
            cudaStreamWaitEvent(c.stream, c.ev_fork, 0);
            {
              const int m = nt128 - next_w;
              const int tiles = m * (m + 1) / 2;
              const int rest = std::max(1, ctas - std::min(ctas / 4, PANEL_RESERVE_SMS));
              int g = std::max(1, std::min(tiles, (rest + na - 1) / na));
              ProfScope ps(c, SGN_PROF_UPDATE, flops_cols(next_w, -1));
              k_update_tcp<<<dim3(g, na), tc::PTHREADS, tc::PSMEM_BYTES, c.stream>>>(
                  c.ds, sv, fronts, K0, FACTOR_BLOCK, maps, next_w, -1, c.status);
              c.tc_launches++;
              c.count();
            }
            cudaEventRecord(c.ev_join, c.stream);
            c.stream = main;
            side_pending = true;
          } else {
            side_pending = false;
          }
        } else {
          int nt = (max_rows + 63) / 64;
          dim3 gu(nt * (nt + 1) / 2, na);
          ProfScope ps(c, SGN_PROF_UPDATE, flops_cols(0, -1));
          k_update<T><<<gu, 256, 0, c.stream>>>(c.ds, sv, fronts, K0, FACTOR_BLOCK);
          c.count();
        }
      }
    }
    if (side_pending) {  // the level's contribution blocks are complete before the next level
      cudaStreamWaitEvent(c.stream, c.ev_join, 0);
      side_pending = false;
    }
    if (max_ns > 0) {
      ProfScope ps(c, SGN_PROF_SOLVE);
      launch_diag_inverse(c, st, fronts, max_ns, (int)(li.f1 - li.f0));
    }
  }
  st.factored = true;
}

}  // namespace

cudaEvent_t *Ctx::prof_pair(int kind, double flops) {
  if (!((prof_mask >> kind) & 1)) return nullptr;
  if (capture_events) {
    GraphEv g{kind, flops, nullptr, nullptr};
    if (cudaEventCreate(&g.e0) != cudaSuccess || cudaEventCreate(&g.e1) != cudaSuccess) return nullptr;
    capture_events->push_back(g);
    return &capture_events->back().e0;  // e0 and e1 are adjacent members
  }
  if (2 * (prof_used + 1) > (int64_t)prof_ev.size()) {
    for (int i = 0; i < 512; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { prof_mask = 0; prof_err = "event pool"; return nullptr; }
      prof_ev.push_back(e);
    }
  }
  cudaEvent_t *p = prof_ev.data() + 2 * prof_used;
  prof_kind.push_back(kind);
  prof_fl.push_back(flops);
  ++prof_used;
  return p;
}

void factor_direct(Ctx &c, Store &s) {
  if (s.fp32) factor_impl<float>(c, s);
  else factor_impl<double>(c, s);
}


void Ctx::harvest_graph_events() {
  if (!pending_events) return;
  cudaEventSynchronize(pending_events->back().e1);
  for (const GraphEv &g : *pending_events) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g.e0, g.e1) == cudaSuccess) {
      gacc_sec[g.kind] += ms * 1e-3;
      gacc_fl[g.kind] += g.flops;
      gacc_n[g.kind] += 1;
    }
  }
  pending_events = nullptr;
}

// captures `body` (which launches on c.stream) into an executable graph
template <typename Body>
cudaGraphExec_t capture(Ctx &c, Body body, int64_t *launches, int64_t *tc) {
  cudaStream_t save = c.stream;
  const int64_t l0 = c.launches, t0 = c.tc_launches;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  c.stream = c.cap_stream;
  if (cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    c.stream = save;
    return nullptr;
  }
  body();
  cudaError_t e = cudaStreamEndCapture(c.cap_stream, &g);
  c.stream = save;
  if (e != cudaSuccess || !g) return nullptr;
  if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
  cudaGraphDestroy(g);
  *launches = c.launches - l0;
  if (tc) *tc = c.tc_launches - t0;
  c.launches = l0;  // counted again at every replay
  c.tc_launches = t0;
  return ex;
}

cudaGraphExec_t capture_fn(Ctx &c, const std::function<void()> &body, int64_t *launches, int64_t *tc) {
  return capture(c, body, launches, tc);
}

void factor_store(Ctx &c, Store &s) {
  auto run = [&]() {
    if (s.fp32) factor_impl<float>(c, s);
    else factor_impl<double>(c, s);
  };
  c.harvest_graph_events();
  const int only_update = 1 << SGN_PROF_UPDATE;
  if (!c.use_graphs || !c.cap_stream || (c.prof_mask != 0 && c.prof_mask != only_update)) {
    run();
    return;
  }
  if (c.prof_mask == 0) {
    if (!s.fgraph) s.fgraph = capture(c, run, &s.fgraph_launches, &s.fgraph_tc);
    if (!s.fgraph) { run(); return; }
    cudaGraphLaunch(s.fgraph, c.stream);
  } else {
    if (!s.fgraph_prof) {
      c.capture_events = &s.fprof;
      int64_t l = 0, t = 0;
      s.fgraph_prof = capture(c, run, &l, &t);
      c.capture_events = nullptr;
      if (!s.fgraph) { s.fgraph_launches = l; s.fgraph_tc = t; }
    }
    if (!s.fgraph_prof) { run(); return; }
    cudaGraphLaunch(s.fgraph_prof, c.stream);
    c.pending_events = &s.fprof;
  }
  c.launches += s.fgraph_launches;
  c.tc_launches += s.fgraph_tc;
  s.factored = true;
}


void set_kernel_attributes() {
  static bool done = false;
  if (done) return;
  done = true;
  cudaFuncSetAttribute(k_block_panels<double, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)((32 * 32 + 32 * 32 + 32 * 129) * sizeof(double)));
  cudaFuncSetAttribute(k_update_tcp, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::PSMEM_BYTES);
  set_solve_attributes();
}

void destroy_graphs(Store &s) {
  if (s.fgraph) cudaGraphExecDestroy(s.fgraph);
  if (s.fgraph_prof) cudaGraphExecDestroy(s.fgraph_prof);
  if (s.sgraph) cudaGraphExecDestroy(s.sgraph);
  for (GraphEv &g : s.fprof) { cudaEventDestroy(g.e0); cudaEventDestroy(g.e1); }
  s.fgraph = s.fgraph_prof = s.sgraph = nullptr;
  s.fprof.clear();
}

void pivot_counts(Ctx &c, Store &s) {
  int64_t n = s.piv_elems;
  k_pivot_counts<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(n, s.piv_type, s.D0, s.D1,
                                                                     (unsigned long long *)c.counters);
  c.count();
}

}  // namespace sgn
