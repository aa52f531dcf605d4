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
//              nb x nb diagonal block in the front's precision (pivot tests
//              decided as in FP64), pivot search restricted to the panel;
//              symmetric swaps are applied to the panel and to the already
//              factored rows of the front (k_row_swap).
//   2. trsm:   W = F21 P^T L11^{-T} (= L21 D) and L21 = W D^{-1}, row-parallel.
//   3. update: F22 -= W L21^T on the lower triangle (tiled GEMM).
// Steps 1 and 2 of a 256-column outer block run as one dataflow launch
// (block_panels.cuh, compiled in panels_f32.cu / panels_f64.cu).
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
// later panels, never rows of an earlier panel in earlier columns; and
// nothing else of the level reads rows [K0, kend) (the trailing updates and
// later blocks use rows >= kend), so the launch may run beside them.
// One warp per panel and CTA column range: lane t gathers row perm(t) of a
// column and writes it to row t; a panel whose permutation is the identity
// is skipped.  CTA 0 also writes the factored diagonal blocks from the stage.
constexpr int RS_COLS = 64;  // columns per CTA
template <typename T>
__global__ void __launch_bounds__(256) k_row_swap(DevSym d, SV sv, const int32_t *__restrict__ fronts, int K0, int NB,
                                                   int nb) {
  const int s = fronts[blockIdx.y];
  const int dpn = sv.dpn;
  const int ns = d.sn_nown[s] * dpn;
  if (K0 >= ns) return;
  const int f = front_order(d, s, dpn);
  const int kend = min(K0 + NB, ns);
  const int c0 = blockIdx.x * RS_COLS;
  if (c0 >= kend) return;
  T *F = (T *)sv.F + sv.front_off[s];
  const int32_t *perm = sv.piv_perm + sv.piv_off[s];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (blockIdx.x == 0) {
    for (int k = K0; k < kend; k += nb) {
      const int w = min(nb, ns - k);
      const T *stage = (const T *)sv.Ldg + (sv.piv_off[s] + k) * (int64_t)nb;
      for (int idx = tid; idx < w * w; idx += blockDim.x) {
        const int jj = idx / w, ii = idx - jj * w;
        if (ii >= jj) F[(int64_t)(k + ii) + (int64_t)(k + jj) * f] = stage[(int64_t)ii * nb + jj];
      }
    }
  }
  const int nwarps = blockDim.x >> 5;
  for (int k = K0 + warp * nb; k < kend; k += nwarps * nb) {
    if (k <= c0) continue;  // no columns of this CTA left of the panel
    const int w = min(nb, ns - k);
    const int src = lane < w ? perm[k + lane] : lane;
    if (__all_sync(0xffffffffu, src == lane)) continue;
    const int cend = min(c0 + RS_COLS, k);
    for (int c = c0; c < cend; c += 8) {
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = (lane < w && c + u < cend) ? F[(int64_t)(k + src) + (int64_t)(c + u) * f] : T(0);
      __syncwarp();
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (lane < w && c + u < cend) F[(int64_t)(k + lane) + (int64_t)(c + u) * f] = v[u];
      __syncwarp();
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

// The tiles of one trailing-update launch: every active front's window of
// tile columns [win0, win1) (win1 < 0: to the end) of its lower triangle, in
// one list ordered by front; cum[q] = tiles of the fronts before front q of
// the level (cum[na] = all), so CTAs take equal shares of the list however
// unevenly the tiles fall on fronts.
struct UpdateTiles {
  DevSym d;
  SV sv;
  const int32_t *fronts;
  const tc::Maps *maps;
  const int32_t *cum;
  int na, K0, NB, win0, win1, pair;
  // list index g -> its front's job and tensor maps, and the unit's index in
  // the front's window
  __device__ __forceinline__ void get(int g, tc::TileJob &job, const tc::Maps *&mp, int &t) const {
    int lo = 0, hi = na;  // the front holding g: the last q with cum[q] <= g
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (__ldg(cum + mid) <= g) lo = mid;
      else hi = mid;
    }
    t = g - __ldg(cum + lo);
    const int s = __ldg(fronts + lo);
    const int dpn = sv.dpn;
    const int ns = d.sn_nown[s] * dpn;
    const int f = front_order(d, s, dpn);
    const int kend = min(K0 + NB, ns);
    const int nrows = f - kend;
    const int nt = (nrows + tc::TILE - 1) / tc::TILE;
    job.win0 = win0;
    job.m = min(win1 < 0 ? nt : win1, nt) - win0;
    job.pair = pair;
    job.ntiles = tc::window_units(job.m, nt - win0, pair != 0);
    job.L = (float *)sv.F + sv.front_off[s];
    job.CB = (float *)sv.CB + sv.cb_off[s];
    job.f = f;
    job.ns = ns;
    job.nrows = nrows;
    job.kend = kend;
    job.kchunks = (kend - K0 + 31) / 32;
    mp = maps + s;
  }
};

// persistent tensor-core trailing update: CTA x walks units x, x + gridDim.x,
// ... of the launch's list (UpdateTiles); PAIR = the units are tile pairs.
template <bool PAIR>
__global__ void __launch_bounds__(tc::PTHREADS, 1) k_update_tcp(DevSym d, SV sv, const int32_t *__restrict__ fronts,
                                                                 int K0, int NB, const tc::Maps *__restrict__ maps,
                                                                 int win0, int win1, const int32_t *__restrict__ cum,
                                                                 int na, int *status) {
  const int total = cum[na];
  if ((int)blockIdx.x >= total) return;
  const UpdateTiles src{d, sv, fronts, maps, cum, na, K0, NB, win0, win1, PAIR ? 1 : 0};
  tc::tile_loop_tc<PAIR>(src, total, blockIdx.x, gridDim.x, status, DEV_TIMEOUT);
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
constexpr int PANEL_RESERVE_SMS = 16;

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
  const size_t panels_smem = block_panels_smem(nbt, sizeof(T));
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
    bool side_used = false;     // the side stream holds work of this level
    for (int K0 = 0; K0 < max_ns; K0 += FACTOR_BLOCK) {
      const int kstop = std::min(K0 + FACTOR_BLOCK, max_ns);
      const int parity = (K0 / FACTOR_BLOCK) & 1;  // which operand set this block writes
      const int64_t bidx = blk;                     // this (level, outer block)
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
          launch_block_panels<T, 16>((unsigned)(b1 - b0), panels_smem, c.stream, c.ds, sv, fronts, st.blk_items + b0,
                                     K0, nb, eps_rel, ctr, st.ctl, c.status);
        else
          launch_block_panels<T, 32>((unsigned)(b1 - b0), panels_smem, c.stream, c.ds, sv, fronts, st.blk_items + b0,
                                     K0, nb, eps_rel, ctr, st.ctl, c.status);
        c.count();
      }
      int na = n_active(li, K0);
      {
        // the permutations of this block's panels (rows [K0, kend), columns
        // left of each panel): nothing else of the level touches those rows,
        // so they run on the side stream, off the chain of panels and
        // updates; the level ends by joining the side stream
        cudaStream_t main = c.stream;
        if (c.side_stream) {
          cudaEventRecord(c.ev_fork, main);
          c.stream = c.side_stream;
          cudaStreamWaitEvent(c.stream, c.ev_fork, 0);
          side_used = true;
        }
        {
          ProfScope ps(c, SGN_PROF_PIVOT);
          dim3 gs((kstop + RS_COLS - 1) / RS_COLS, na);
          k_row_swap<T><<<gs, 256, 0, c.stream>>>(c.ds, sv, fronts, K0, FACTOR_BLOCK, nb);
          c.count();
        }
        c.stream = main;
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
          // one CTA per SM (192 KB shared memory), each taking an equal share
          // of one list of the units of every active front.  The tile columns
          // holding the next outer block's columns go first on this stream, in
          // single tiles so that more SMs share that critical step;
          // the rest runs on the side stream, next to the next block's panels
          // (which write the other operand set), on fewer SMs so that those
          // panels find room
          const int nt128 = (max_rows + tc::TILE - 1) / tc::TILE;
          const int ctas = c.update_ctas > 0 ? c.update_ctas : c.num_sms;
          const int next_w = FACTOR_BLOCK / tc::TILE;
          const tc::Maps *maps = (const tc::Maps *)st.maps + (size_t)parity * c.S.sn.size();
          if (side_pending) cudaStreamWaitEvent(c.stream, c.ev_join, 0);  // the previous block's rest
          const bool split = nt128 > next_w && c.side_stream && K0 + FACTOR_BLOCK < max_ns;
          // the tile list of window w: its cumulative counts and its length
          auto tiles_of = [&](int wdw, const int32_t *&cum) {
            const int64_t off = st.h_upd_off[3 * bidx + wdw];
            cum = st.upd_cum + off;
            return (int)st.h_upd_cum[off + na];
          };
          {
            const int32_t *cum;
            const int tiles = tiles_of(split ? 0 : 2, cum);
            const int g = std::max(1, std::min(tiles, ctas));
            ProfScope ps(c, SGN_PROF_UPDATE, split ? flops_cols(0, next_w) : flops_cols(0, -1));
            if (split)
              k_update_tcp<false><<<g, tc::PTHREADS, tc::PSMEM_BYTES, c.stream>>>(
                  c.ds, sv, fronts, K0, FACTOR_BLOCK, maps, 0, next_w, cum, na, c.status);
            else
              k_update_tcp<true><<<g, tc::PTHREADS, tc::PSMEM_BYTES, c.stream>>>(
                  c.ds, sv, fronts, K0, FACTOR_BLOCK, maps, 0, -1, cum, na, c.status);
            c.tc_launches++;
            c.count();
          }
          if (split) {
            cudaEventRecord(c.ev_fork, c.stream);
            cudaStream_t main = c.stream;
            c.stream = c.side_stream;
            cudaStreamWaitEvent(c.stream, c.ev_fork, 0);
            {
              const int32_t *cum;
              const int tiles = tiles_of(1, cum);
              const int rest = std::max(1, ctas - std::min(ctas / 4, PANEL_RESERVE_SMS));
              const int g = std::max(1, std::min(tiles, rest));
              ProfScope ps(c, SGN_PROF_UPDATE, flops_cols(next_w, -1));
              k_update_tcp<true><<<g, tc::PTHREADS, tc::PSMEM_BYTES, c.stream>>>(
                  c.ds, sv, fronts, K0, FACTOR_BLOCK, maps, next_w, -1, cum, na, c.status);
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
    if (side_used || side_pending) {  // the level's side-stream work is complete before the next level
      cudaEventRecord(c.ev_join, c.side_stream);
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
  set_block_panels_smem<float, 16>((int)block_panels_smem(16, sizeof(float)));
  set_block_panels_smem<float, 32>((int)block_panels_smem(32, sizeof(float)));
  set_block_panels_smem<double, 16>((int)block_panels_smem(16, sizeof(double)));
  set_block_panels_smem<double, 32>((int)block_panels_smem(32, sizeof(double)));
  cudaFuncSetAttribute(k_update_tcp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::PSMEM_BYTES);
  cudaFuncSetAttribute(k_update_tcp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::PSMEM_BYTES);
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
