// Internal to the multifrontal factorization (front.cu) and the
// substitutions (solve.cu): the store view the kernels receive and the
// addressing of a front's lower triangle.
#pragma once

#include "common.cuh"

namespace sgn {

struct SV {  // store view passed to kernels
  void *F;                       // factor columns of every front (f x ns each)
  void *CB;                      // contribution-block arena
  void *Xinv;                    // diagonal-block inverses
  void *W;
  void *Ldg;                     // staged factored diagonal blocks (panel x panel per panel)
  float *wk0, *wk1, *wk2, *wk3;  // K-major hi/lo copies (FP32 fronts with tensor cores)
  double *rhs;
  int32_t *piv_type, *piv_perm;
  double *D0, *D1;
  double *yz;                    // y, z = D^{-1} y, v of the substitutions (pivot order)
  unsigned long long *pub;       // published block values of the substitutions
  unsigned *pflag;               // their tags (FP64 fronts)
  unsigned long long *bpart;     // published parts of the backward ancestor-row products (FP32)
  const int64_t *part_off;       // each front's first part word in bpart
  unsigned *fflag;               // panel-factored flags of the factorization (epoch tags)
  unsigned *fpre;                // panel-rows-ready flags (epoch tags)
  const int64_t *front_off, *cb_off, *w_off, *rhs_off, *piv_off, *xinv_off;
  int dpn;
  int kkt;
};

inline SV view(Store &s, int parity = 0) {
  SV v;
  v.F = s.F; v.CB = s.CB; v.cb_off = s.cb_off; v.W = s.W; v.rhs = s.rhs; v.Ldg = s.Ldg;
  v.Xinv = s.Xinv; v.xinv_off = s.xinv_off; v.pub = s.pub; v.pflag = s.pflag; v.yz = s.yz; v.fflag = s.fflag;
  v.fpre = s.fflag ? s.fflag + s.piv_elems : nullptr;
  const int o = 4 * (parity & 1);
  v.wk0 = s.tc ? s.wk[o] : nullptr; v.wk1 = s.wk[o + 1]; v.wk2 = s.wk[o + 2]; v.wk3 = s.wk[o + 3];
  v.piv_type = s.piv_type; v.piv_perm = s.piv_perm;
  v.D0 = s.D0; v.D1 = s.D1; v.front_off = s.front_off; v.w_off = s.w_off; v.rhs_off = s.rhs_off;
  v.piv_off = s.piv_off; v.dpn = s.dpn; v.kkt = s.kkt ? 1 : 0;
  v.bpart = s.bpart; v.part_off = s.part_off;
  return v;
}

__device__ __forceinline__ int front_order(const DevSym &d, int s, int dpn) {
  return (d.sn_nown[s] + d.sn_nstruct[s]) * dpn;
}

// The lower triangle of front s (order f, ns fully-summed columns): columns
// j < ns live in the front array (f x ns, column-major), the contribution
// block (rows and columns >= ns) in the arena ((f - ns) x (f - ns)).
template <typename T>
struct FrontMat {
  T *L, *C;
  int64_t f, ns;
  // element (i, j) of the lower triangle (i >= j)
  __device__ __forceinline__ T *at(int64_t i, int64_t j) const {
    return j < ns ? L + i + j * f : C + (i - ns) + (j - ns) * (f - ns);
  }
};

template <typename T>
__device__ __forceinline__ FrontMat<T> front_mat(const DevSym &d, const SV &sv, int s) {
  FrontMat<T> m;
  m.L = (T *)sv.F + sv.front_off[s];
  m.C = (T *)sv.CB + sv.cb_off[s];
  m.ns = (int64_t)d.sn_nown[s] * sv.dpn;
  m.f = m.ns + (int64_t)d.sn_nstruct[s] * sv.dpn;
  return m;
}

constexpr int SB = 128;  // solve block width (independent of the pivot panel width)

// host-side launchers shared by the translation units
void launch_diag_inverse(Ctx &c, Store &st, const int32_t *fronts, int max_ns, int nfronts);
void set_solve_attributes();

// the outer-block panel kernel (block_panels.cuh; T = float / double, NBT =
// 16 / 32 compiled panel width) and its dynamic shared memory: a chunk of L
// per warp (4 x 32 x NBT), L11 (NBT x NBT) and the band's L and W (NBT rows
// of PANEL_XS entries each, 4 entries of padding after each buffer so that
// 4-wide reads near a buffer's end stay inside it)
constexpr int PANEL_XS = 132;
inline size_t block_panels_smem(int nbt, size_t elt) {
  return (size_t)(4 * 32 * nbt + nbt * nbt + 2 * (nbt * PANEL_XS + 4)) * elt;
}
template <typename T, int NBT>
void launch_block_panels(unsigned grid, size_t smem, cudaStream_t stream, const DevSym &d, const SV &sv,
                         const int32_t *fronts, const BandItem *items, int K0, int nb, double eps_rel,
                         unsigned long long *counters, unsigned *ctl, int *status);
template <typename T, int NBT>
void set_block_panels_smem(int bytes);

}  // namespace sgn
