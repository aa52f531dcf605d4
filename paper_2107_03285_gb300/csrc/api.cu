// C ABI of libsgn: set-up, device binding, and the orchestration of the hot
// path (assemble -> factor -> solve + FP64 refinement), forward simulation and
// the adjoint gradient.  All device memory comes from the caller's buffer.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <map>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "tc_update.cuh"

using namespace sgn;


namespace {

thread_local std::string g_err;

// Newton equilibrium: a residual that a full-accuracy step no longer halves
// counts as converged once below this fraction of ||f_ext||.  Measured floors
// of ||c|| / ||f_ext|| with the displacement iterate: 1.3e-11 (60 x 60 grid),
// 8.5e-12 (40 x 40), below 1e-13 on the 3D cubes.
constexpr double kStagnationCap = 1e-10;

#define CUDA_TRY(h, call)                                                   \
  do {                                                                      \
    cudaError_t _e = (call);                                                \
    if (_e != cudaSuccess) {                                                \
      (h)->last_error = g_err = std::string(#call) + ": " + cudaGetErrorString(_e); \
      return SGN_ECUDA;                                                     \
    }                                                                       \
  } while (0)

struct V3 {  // a vector of the full saddle-point system: x, p, lambda parts
  double *x, *p, *l;
};

struct Carver {
  char *base;
  size_t off = 0;
  explicit Carver(char *b) : base(b) {}
  template <typename T>
  T *take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += std::max<size_t>(n, 1) * sizeof(T);
    return p;
  }
};

struct Upload {
  void *dst;
  const void *src;
  size_t bytes;
};

// Places every contribution block in one arena: the block of front s lives
// from the assembly of s's level (which writes it) to the assembly of its
// parent's level (which reads it).  Levels are walked in order; a level's
// blocks are placed best-fit in the free space (largest first) before its
// children's blocks are released.  Returns the arena size in elements.
int64_t plan_cb_arena(const Symbolic &S, int dpn, std::vector<int64_t> &cb_off, int64_t *cb_sum) {
  cb_off.assign(S.sn.size(), 0);
  std::map<int64_t, int64_t> free_blocks;  // offset -> size, below `end`
  int64_t end = 0, high = 0, sum = 0;
  auto cb_size = [&](int s) {
    const int64_t m = (int64_t)S.sn[s].nstruct * dpn;
    return ((m * m + 63) / 64) * 64;  // 256-byte granules (FP32)
  };
  auto release = [&](int64_t off, int64_t size) {
    auto it = free_blocks.emplace(off, size).first;
    auto nx = std::next(it);
    if (nx != free_blocks.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_blocks.erase(nx);
    }
    if (it != free_blocks.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_blocks.erase(it);
        it = pv;
      }
    }
    if (it->first + it->second == end) {  // free space at the top shrinks the arena
      end = it->first;
      free_blocks.erase(it);
    }
  };
  for (const auto &lv : S.level_fronts) {
    std::vector<int> order(lv.begin(), lv.end());
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cb_size(a) > cb_size(b); });
    for (int s : order) {
      const int64_t need = cb_size(s);
      sum += need;
      if (need == 0) continue;
      auto best = free_blocks.end();
      for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it)
        if (it->second >= need && (best == free_blocks.end() || it->second < best->second)) best = it;
      if (best != free_blocks.end()) {
        cb_off[s] = best->first;
        const int64_t rest = best->second - need, at = best->first + need;
        free_blocks.erase(best);
        if (rest > 0) free_blocks.emplace(at, rest);
      } else {
        cb_off[s] = end;
        end += need;
        high = std::max(high, end);
      }
    }
    for (int s : lv)
      for (int j = 0; j < S.sn[s].nchild; ++j) {
        const int ch = S.children[S.sn[s].child_off + j];
        if (cb_size(ch) > 0) release(cb_off[ch], cb_size(ch));
      }
  }
  *cb_sum = sum;
  // self-check: replay the lifetimes and verify that no two live blocks overlap
  std::map<int64_t, int64_t> live;  // offset -> end
  for (const auto &lv : S.level_fronts) {
    for (int s : lv) {
      const int64_t need = cb_size(s);
      if (need == 0) continue;
      const int64_t o = cb_off[s], e = o + need;
      if (e > high) return -1;
      auto it = live.lower_bound(o);
      if (it != live.end() && it->first < e) return -1;
      if (it != live.begin() && std::prev(it)->second > o) return -1;
      live.emplace(o, e);
    }
    for (int s : lv)
      for (int j = 0; j < S.sn[s].nchild; ++j) {
        const int ch = S.children[S.sn[s].child_off + j];
        if (cb_size(ch) > 0) live.erase(cb_off[ch]);
      }
  }
  return high;
}

void store_offsets(Ctx &c, Store &s, int dpn) {
  s.dpn = dpn;
  const int n_sn = (int)c.S.sn.size();
  s.h_front_off.assign(n_sn, 0); s.h_w_off.assign(n_sn, 0);
  s.h_rhs_off.assign(n_sn, 0); s.h_piv_off.assign(n_sn, 0); s.h_xinv_off.assign(n_sn, 0);
  s.h_part_off.assign(n_sn, 0);
  int64_t fo = 0, ro = 0, po = 0, xo = 0, pa = 0;
  constexpr int64_t SBK = 128;  // solve block width
  for (int i = 0; i < n_sn; ++i) {
    int64_t f = (int64_t)c.S.sn[i].fnodes() * dpn, ns = (int64_t)c.S.sn[i].nown * dpn;
    s.h_front_off[i] = fo; fo += ((f * ns + 63) / 64) * 64;
    s.h_rhs_off[i] = ro; ro += f;
    s.h_piv_off[i] = po; po += ns;
    s.h_part_off[i] = pa; pa += s.fp32 ? (int64_t)bwd_parts(f - ns) * ns : 0;
    // full blocks of SBK^2, the last one (w < SBK) of w^2, 16-byte aligned
    const int64_t nfull = ns / SBK, wl = ns - nfull * SBK;
    s.h_xinv_off[i] = xo; xo += nfull * SBK * SBK + ((wl * wl + 3) / 4) * 4;
  }
  s.xinv_elems = xo;
  // W (= L21 D of the current outer block) is only live while its level is
  // factored, so all levels share one workspace sized for the largest level
  int64_t wmax = 0;
  for (const auto &lv : c.S.level_fronts) {
    int64_t wo = 0;
    for (int i : lv) {
      s.h_w_off[i] = wo;
      wo += (int64_t)c.S.sn[i].fnodes() * dpn * FACTOR_BLOCK;
    }
    wmax = std::max(wmax, wo);
  }
  // substitution schedules (one CTA per item): forward items are the
  // front's 128-row bands, own bands (key b) before its struct bands (key
  // nbo + j), except that a front with one own block is a single item;
  // backward items its 128-column blocks, last first (key nbo - 1 - b),
  // and for an FP32 front with many ancestor rows the parts of each block's
  // ancestor-row product (key -1 - (b BWD_PARTS_MAX + h), which wait on
  // nothing).  Sorting a level's items by key puts every dependency first.
  s.h_fwd_items.clear(); s.h_bwd_items.clear();
  s.h_fwd_lvl.assign(1, 0); s.h_bwd_lvl.assign(1, 0);
  int32_t q = 0;
  for (const auto &lv : c.S.level_fronts) {
    const size_t f0 = s.h_fwd_items.size(), b0 = s.h_bwd_items.size();
    for (int i : lv) {
      const int64_t f = (int64_t)c.S.sn[i].fnodes() * dpn, ns = (int64_t)c.S.sn[i].nown * dpn;
      const int32_t nbo = (int32_t)((ns + SBK - 1) / SBK), nbs = (int32_t)((f - ns + SBK - 1) / SBK);
      if (ns > 0) {
        // a single-block front is one forward item (it also does its struct rows)
        const int32_t nfw = nbo > 1 ? nbo + nbs : 1;
        for (int32_t k = 0; k < nfw; ++k) s.h_fwd_items.push_back({q, k});
        for (int32_t k = 0; k < nbo; ++k) s.h_bwd_items.push_back({q, k});
        const int nparts = s.fp32 ? bwd_parts(f - ns) : 0;
        for (int32_t b = 0; b < nbo; ++b)
          for (int h = 0; h < nparts; ++h) s.h_bwd_items.push_back({q, -1 - (b * BWD_PARTS_MAX + h)});
      }
      ++q;
    }
    auto by_key = [](const SolveItem &a, const SolveItem &b) { return a.key != b.key ? a.key < b.key : a.q < b.q; };
    std::sort(s.h_fwd_items.begin() + f0, s.h_fwd_items.end(), by_key);
    std::sort(s.h_bwd_items.begin() + b0, s.h_bwd_items.end(), by_key);
    s.h_fwd_lvl.push_back((int64_t)s.h_fwd_items.size());
    s.h_bwd_lvl.push_back((int64_t)s.h_bwd_items.size());
  }
  // panel-kernel items per (level, outer block): band-major, so that the
  // owners of the block's panels (bands 0 and 1 of every front) come first
  s.h_blk_items.clear();
  s.h_blk_off.assign(1, 0);
  s.h_upd_cum.clear();
  s.h_upd_off.clear();
  for (const auto &lv : c.S.level_fronts) {
    int64_t max_ns = 0;
    for (int i : lv) max_ns = std::max<int64_t>(max_ns, (int64_t)c.S.sn[i].nown * dpn);
    for (int64_t K0 = 0; K0 < max_ns; K0 += FACTOR_BLOCK) {
      for (int32_t b = 0;; ++b) {
        bool any = false;
        int32_t q = 0;
        for (int i : lv) {
          const int64_t f = (int64_t)c.S.sn[i].fnodes() * dpn, ns = (int64_t)c.S.sn[i].nown * dpn;
          if (ns > K0 && f - K0 > (int64_t)128 * b) {
            s.h_blk_items.push_back({q, b});
            any = true;
          }
          ++q;
        }
        if (!any) break;
      }
      s.h_blk_off.push_back((int64_t)s.h_blk_items.size());
      // the trailing update's units per active front (fronts sorted by ns,
      // largest first, so the active ones come first), for each window: single
      // tiles for the next outer block's columns (window 0, on the critical
      // path: more CTAs), tile pairs for the rest (1) and the whole (2)
      const int next_w = FACTOR_BLOCK / 128;
      for (int wdw = 0; wdw < 3; ++wdw) {
        const int win0 = wdw == 1 ? next_w : 0, win1 = wdw == 0 ? next_w : -1;
        s.h_upd_off.push_back((int64_t)s.h_upd_cum.size());
        int32_t acc = 0;
        s.h_upd_cum.push_back(0);
        for (int i : lv) {
          const int64_t f = (int64_t)c.S.sn[i].fnodes() * dpn, ns = (int64_t)c.S.sn[i].nown * dpn;
          if (ns <= K0) break;
          const int64_t kend = std::min<int64_t>(K0 + FACTOR_BLOCK, ns);
          const int nt = (int)((f - kend + 127) / 128);
          const int m = std::min(win1 < 0 ? nt : win1, nt) - win0, n = nt - win0;
          acc += tc::window_units(m, n, wdw != 0);
          s.h_upd_cum.push_back(acc);
        }
      }
    }
  }
  // self-check (the substitutions' waits rely on it): an item of key k >= 0
  // waits only on keys 0 .. k - 1 and the negative keys (the parts, which
  // wait on nothing) of its own front, so within their level each front's
  // parts must come first and its other items with keys 0, 1, 2, ... in
  // list order
  s.sched_ok = true;
  for (const auto *lst : {&s.h_fwd_items, &s.h_bwd_items}) {
    const auto &lvl = lst == &s.h_fwd_items ? s.h_fwd_lvl : s.h_bwd_lvl;
    std::vector<int32_t> next(q, 0);
    for (size_t L = 0; L + 1 < lvl.size(); ++L)
      for (int64_t t = lvl[L]; t < lvl[L + 1]; ++t) {
        const SolveItem &it = (*lst)[t];
        if (it.q < 0 || it.q >= q) s.sched_ok = false;
        else if (it.key < 0) s.sched_ok = s.sched_ok && lst == &s.h_bwd_items && next[it.q] == 0;
        else if (it.key != next[it.q]) s.sched_ok = false;
        else ++next[it.q];
      }
  }
  s.front_elems = fo; s.w_elems = wmax; s.rhs_elems = ro; s.piv_elems = po; s.part_elems = pa;
  s.cb_elems = plan_cb_arena(c.S, dpn, s.h_cb_off, &s.cb_sum);
}

// lays out (base == nullptr: only measures) every device array
size_t carve(Ctx &c, char *base, int stores, std::vector<Upload> *up) {
  Carver cv(base);
  Symbolic &S = c.S;
  const int d = S.dim, nv = d + 1;
  const int64_t ne = S.n_elem, nf = S.n_free, nx = nf * d;
  auto st_up = [&](auto *&dst, const auto &vec) {
    using T = typename std::remove_reference<decltype(vec)>::type::value_type;
    T *p = cv.take<T>(vec.size());
    dst = p;
    if (up && p) up->push_back({p, vec.data(), vec.size() * sizeof(T)});
  };
  DevSym &ds = c.ds;
  ds.dim = d; ds.n_nodes = S.n_nodes; ds.n_elem = S.n_elem; ds.n_free = S.n_free;
  ds.n_sn = (int)S.sn.size(); ds.panel = S.opts.panel;
  // static symbolic data
  static thread_local std::vector<int32_t> sn_first, sn_nown, sn_nstruct, sn_child_off, sn_nchild, lvl_fronts,
      item_sn, item_P;
  static thread_local std::vector<int64_t> sn_struct_off;
  sn_first.clear(); sn_nown.clear(); sn_nstruct.clear(); sn_child_off.clear(); sn_nchild.clear();
  sn_struct_off.clear(); lvl_fronts.clear(); item_sn.clear(); item_P.clear();
  for (auto &s : S.sn) {
    sn_first.push_back(s.first); sn_nown.push_back(s.nown); sn_nstruct.push_back(s.nstruct);
    sn_child_off.push_back(s.child_off); sn_nchild.push_back(s.nchild); sn_struct_off.push_back(s.struct_off);
  }
  c.h_lvl_ptr.assign(1, 0); c.h_item_ptr.assign(1, 0);
  for (int L = 0; L < S.n_levels; ++L) {
    for (int s : S.level_fronts[L]) {
      lvl_fronts.push_back(s);
      for (int P = 0; P < S.sn[s].fnodes(); ++P) { item_sn.push_back(s); item_P.push_back(P); }
    }
    c.h_lvl_ptr.push_back((int64_t)lvl_fronts.size());
    c.h_item_ptr.push_back((int64_t)item_sn.size());
  }
  const int32_t *cp;
  const double *cd;
  const int64_t *c64;
#define UP32(field, vec) do { int32_t *p_; st_up(p_, vec); ds.field = p_; } while (0)
#define UPD(field, vec) do { double *p_; st_up(p_, vec); ds.field = p_; } while (0)
#define UP64(field, vec) do { int64_t *p_; st_up(p_, vec); ds.field = p_; } while (0)
  (void)cp; (void)cd; (void)c64;
  UP32(elem_node, S.elem_node); UP32(elem_rank, S.elem_rank);
  UPD(elem_B, S.elem_B); UPD(elem_vol, S.elem_vol); UPD(X, S.X);
  UP32(node_rank, S.node_rank); UP32(rank_node, S.rank_node);
  UP32(bsr_ptr, S.bsr_ptr); UP32(bsr_col, S.bsr_col); UP32(bsr_orig_pos, S.bsr_orig_pos);
  UP32(up_slot, S.up_slot); UP32(up_slot_t, S.up_slot_t); UP32(up_ptr, S.up_ptr); UP32(up_contrib, S.up_contrib);
  UP32(inc_ptr, S.inc_ptr); UP32(inc, S.inc);
  UP32(sn_first, sn_first); UP32(sn_nown, sn_nown); UP32(sn_nstruct, sn_nstruct);
  UP32(sn_child_off, sn_child_off); UP32(sn_nchild, sn_nchild); UP64(sn_struct_off, sn_struct_off);
  UP32(struct_ranks, S.struct_ranks); UP32(relpos, S.relpos); UP32(children, S.children);
  UP64(cmap_off, S.cmap_off); UP32(cmap, S.cmap);
  UP32(lvl_fronts, lvl_fronts); UP32(item_sn, item_sn); UP32(item_P, item_P);
#undef UP32
#undef UPD
#undef UP64
  // dynamic arrays
  c.n_state = 3 + nv * d;
  c.st = cv.take<double>((size_t)c.n_state * ne);
  c.cpv = cv.take<double>((size_t)nv * d * ne);
  c.Kv = cv.take<double>(S.bsr_col.size() * d * d);
  c.Gv = cv.take<double>(S.bsr_col.size() * d * d);
  c.wA = cv.take<double>(nx); c.tgt = cv.take<double>(nx);
  c.fx = cv.take<double>(nx); c.fp = cv.take<double>(ne); c.xr = cv.take<double>(nx);
  c.bx = cv.take<double>(nx); c.bp = cv.take<double>(ne); c.bl = cv.take<double>(nx);
  c.zx = cv.take<double>(nx); c.zp = cv.take<double>(ne); c.zl = cv.take<double>(nx);
  c.rx = cv.take<double>(nx); c.rp = cv.take<double>(ne); c.rl = cv.take<double>(nx);
  c.red = cv.take<double>(2 * nx * 2);  // reduced rhs and solution
  c.kry = cv.take<double>((size_t)Ctx::KRY_VECS * (2 * nx + ne));  // BiCGSTAB vectors
  c.n_partial = 1024;
  c.partial = cv.take<double>(c.n_partial);
  c.partial2 = cv.take<double>(2 * c.n_partial);
  c.status = cv.take<int>(4);
  c.counters = cv.take<int64_t>(8);
  const size_t nn = (size_t)S.n_nodes * d;
  c.eq = cv.take<double>(4 * nx);
  c.xsave = cv.take<double>(nn); c.xrt = cv.take<double>(nx); c.ueq = cv.take<double>(nn);
  c.hx = cv.take<double>(nn); c.hdx = cv.take<double>(nn); c.hdl = cv.take<double>(nn);
  c.hp = cv.take<double>(ne); c.hdp = cv.take<double>(ne);
  c.lbq = cv.take<double>(ne); c.lbr = cv.take<double>(ne);
  if (c.n_inst > 0) {
    int32_t *p_;
    st_up(p_, c.h_rank_inst); c.rank_inst = p_;
    st_up(p_, c.h_elem_inst); c.elem_inst = p_;
    c.inst_acc = cv.take<double>(4 * (size_t)c.n_inst);
  }
  bool plan_ok = true;
  auto store = [&](Store &s, bool on, int dpn, bool kkt, bool fp32) {
    s.enabled = on;
    s.kkt = kkt; s.fp32 = fp32;
    store_offsets(c, s, dpn);
    if (!on) return;
    if (s.cb_elems < 0) { plan_ok = false; s.cb_elems = 0; }
    if (!s.sched_ok) plan_ok = false;
    size_t es = fp32 ? 4 : 8;
    s.F = cv.take<char>((size_t)s.front_elems * es);
    s.CB = cv.take<char>((size_t)s.cb_elems * es);
    s.Xinv = cv.take<char>((size_t)s.xinv_elems * es);
    s.W = cv.take<char>((size_t)s.w_elems * es);
    s.Ldg = cv.take<char>((size_t)s.piv_elems * c.S.opts.panel * es);
    s.rhs = cv.take<double>(s.rhs_elems);
    s.piv_type = cv.take<int32_t>(s.piv_elems); s.piv_perm = cv.take<int32_t>(s.piv_elems);
    s.D0 = cv.take<double>(s.piv_elems); s.D1 = cv.take<double>(s.piv_elems);
    s.yz = cv.take<double>(s.piv_elems);
    s.pub = cv.take<unsigned long long>(s.piv_elems);
    s.pflag = fp32 ? nullptr : cv.take<unsigned>(s.piv_elems);
    s.bpart = s.part_elems > 0 ? cv.take<unsigned long long>((size_t)s.part_elems) : nullptr;
    s.fflag = cv.take<unsigned>(2 * s.piv_elems);  // panel-factored, then panel-rows-ready flags
    s.ctl = cv.take<unsigned>(16);
    {
      SolveItem *it;
      st_up(it, s.h_fwd_items); s.fwd_items = it;
      st_up(it, s.h_bwd_items); s.bwd_items = it;
      BandItem *bi;
      st_up(bi, s.h_blk_items); s.blk_items = bi;
      int32_t *uc;
      st_up(uc, s.h_upd_cum); s.upd_cum = uc;
    }
    if (fp32) {
      for (int q = 0; q < 8; ++q) s.wk[q] = cv.take<float>(s.w_elems);
      s.maps = cv.take<char>(2 * S.sn.size() * sizeof(tc::Maps));
    }
    int64_t *p;
    st_up(p, s.h_front_off); s.front_off = p;
    st_up(p, s.h_cb_off); s.cb_off = p;
    st_up(p, s.h_xinv_off); s.xinv_off = p;
    st_up(p, s.h_w_off); s.w_off = p;
    st_up(p, s.h_rhs_off); s.rhs_off = p;
    st_up(p, s.h_piv_off); s.piv_off = p;
    st_up(p, s.h_part_off); s.part_off = p;
  };
  store(c.kkt64, (stores & SGN_STORE_FP64) != 0, 2 * d, true, false);
  store(c.kkt32, (stores & SGN_STORE_MIXED) != 0, 2 * d, true, true);
  store(c.kf, (stores & SGN_STORE_KFACT) != 0, d, false, false);
  store(c.kf32, (stores & SGN_STORE_KFACT_MIXED) != 0, d, false, true);
  return plan_ok ? cv.off + 256 : 0;  // 0: a host plan failed its self-check
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// TMA tensor maps of the four K-major operand arrays of every front: rows =
// the front's rows, 256 K columns (1 KB rows), box 32 x 128 with 128B swizzle,
// out-of-range rows read as zero
bool encode_maps(Ctx &c, Store &st, std::vector<tc::Maps> &out) {
  void *fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn)
    return false;
  EncodeTiledFn enc = (EncodeTiledFn)fn;
  const size_t nsn = c.S.sn.size();
  out.assign(2 * nsn, tc::Maps());
  for (size_t pi = 0; pi < 2 * nsn; ++pi) {
    const size_t i = pi % nsn, par = pi / nsn;
    const cuuint64_t f = (cuuint64_t)c.S.sn[i].fnodes() * st.dpn;
    cuuint64_t dims[2] = {(cuuint64_t)FACTOR_BLOCK, f};
    cuuint64_t strides[1] = {(cuuint64_t)FACTOR_BLOCK * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)tc::KCH, (cuuint32_t)tc::TILE};
    cuuint32_t estr[2] = {1, 1};
    CUtensorMap *m[4] = {&out[pi].whi, &out[pi].wlo, &out[pi].lhi, &out[pi].llo};
    for (int k = 0; k < 4; ++k) {
      void *addr = st.wk[4 * par + k] + st.h_w_off[i];
      CUresult r = enc(m[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, addr, dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return false;
    }
  }
  return true;
}

sgn_status check_status(sgn_ctx *h) {
  int st = 0;
  CUDA_TRY(h, cudaMemcpyAsync(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (st) {
    CUDA_TRY(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream));
    if (st & DEV_INVERTED) { h->last_error = "inverted element (det F <= 0)"; return SGN_EINVERTED; }
    if (st & DEV_TIMEOUT) { h->last_error = "a bounded device wait expired"; return SGN_ETIMEOUT; }
    h->last_error = "non-finite value in element evaluation";
    return SGN_ENONFINITE;
  }
  return SGN_OK;
}

sgn_status launch_check(sgn_ctx *h) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    h->last_error = g_err = std::string("kernel launch: ") + cudaGetErrorString(e);
    return SGN_ECUDA;
  }
  return SGN_OK;
}

}  // namespace

namespace sgn {
void set_error(Ctx *h, const std::string &msg) {
  g_err = msg;
  if (h) h->last_error = msg;
}
}  // namespace sgn

extern "C" {

const char *sgn_last_error(sgn_t h) { return h ? h->last_error.c_str() : ""; }

sgn_status sgn_selftest_wait_timeout(sgn_t h) {
  if (!h) return SGN_EINVAL;
  if (!h->bound) return SGN_ESTATE;
  Store *st = nullptr;
  for (Store *s : {&h->kkt32, &h->kkt64, &h->kf32, &h->kf})
    if (s->enabled) { st = s; break; }
  if (!st) return SGN_ESTATE;
  sgn_status s = check_status(h);  // start from a clean status word
  if (s != SGN_OK) return s;
  wait_selftest(*h, *st);
  s = launch_check(h);
  if (s != SGN_OK) return s;
  return check_status(h);  // SGN_ETIMEOUT expected; the word is cleared
}

const char *sgn_strerror(sgn_status s) {
  switch (s) {
    case SGN_OK: return "ok";
    case SGN_EINVAL: return g_err.empty() ? "invalid argument" : g_err.c_str();
    case SGN_ECUDA: return g_err.empty() ? "CUDA error" : g_err.c_str();
    case SGN_ENOMEM: return "device buffer too small or host allocation failed";
    case SGN_EINVERTED: return "inverted element (det F <= 0)";
    case SGN_ENEWTON: return "equilibrium Newton did not converge";
    case SGN_EPIVOT: return "perturbed pivot not recovered by refinement";
    case SGN_EREFINE: return "iterative refinement did not reach its tolerance";
    case SGN_ESTATE: return "call out of order";
    case SGN_ENONFINITE: return "non-finite value";
    case SGN_ETIMEOUT: return "a bounded device-side wait expired";
  }
  return "unknown status";
}

sgn_status sgn_setup(const sgn_mesh *mesh, const sgn_setup_opts *opts, sgn_t *out) {
  if (!mesh || !out) return SGN_EINVAL;
  *out = nullptr;
  sgn_ctx *h = new (std::nothrow) sgn_ctx();
  if (!h) return SGN_ENOMEM;
  SymbolicOptions so;
  if (opts) { so.leaf_nodes = opts->leaf_nodes; so.panel = opts->panel; }
  if (opts && opts->update_ctas < 0) { g_err = "update_ctas must be >= 0"; delete h; return SGN_EINVAL; }
  if (so.leaf_nodes <= 0) so.leaf_nodes = 16;
  if (so.panel <= 0) so.panel = 32;
  if (!(mesh->nu > -1.0 && mesh->nu < 0.5) || !(mesh->E0 > 0.0)) {
    g_err = "material: need E0 > 0 and -1 < nu < 0.5";
    delete h;
    return SGN_EINVAL;
  }
  std::string err;
  try {
    err = analyze(mesh->dim, mesh->n_nodes, mesh->n_elem, mesh->X_h, mesh->conn_h, mesh->fixed_h, so, h->S);
  } catch (const std::bad_alloc &) {
    delete h;
    return SGN_ENOMEM;
  }
  if (!err.empty()) {
    g_err = err;
    delete h;
    return SGN_EINVAL;
  }
  h->E0 = mesh->E0; h->nu = mesh->nu;
  h->update_ctas = opts ? opts->update_ctas : 0;
  *out = h;
  return SGN_OK;
}

sgn_status sgn_get_info(sgn_t h, sgn_info *o) {
  if (!h || !o) return SGN_EINVAL;
  const Symbolic &S = h->S;
  o->n_nodes = S.n_nodes; o->n_free = S.n_free; o->n_elem = S.n_elem;
  o->n_x = (int64_t)S.n_free * S.dim; o->n_p = S.n_elem; o->n_kkt = 2 * o->n_x + o->n_p;
  // full symmetric saddle point without A: 2 (K) + 2 (cp) + C diag
  int64_t nnzK = (int64_t)S.bsr_col.size() * S.dim * S.dim;
  int64_t nnzcp = 0;
  for (int64_t i = 0; i < (int64_t)S.elem_rank.size(); ++i) nnzcp += S.elem_rank[i] >= 0 ? S.dim : 0;
  o->nnz_kkt = 2 * nnzK + 2 * nnzcp + o->n_p;
  o->n_supernodes = (int64_t)S.sn.size(); o->n_levels = S.n_levels;
  o->max_front = S.max_front_nodes * 2 * S.dim;
  o->nnz_factor = S.nnz_factor_kkt;
  o->factor_flops = S.flops_kkt; o->kfactor_flops = S.flops_k;
  o->setup_seconds = S.seconds;
  return SGN_OK;
}

sgn_status sgn_device_bytes(sgn_t h, int32_t stores, size_t *bytes) {
  if (!h || !bytes) return SGN_EINVAL;
  *bytes = carve(*h, nullptr, stores, nullptr);
  if (*bytes == 0) { g_err = "internal: a host plan (contribution-block arena, substitution schedule) failed its self-check"; return SGN_EINVAL; }
  return SGN_OK;
}

sgn_status sgn_set_stream(sgn_t h, void *stream) {
  if (!h) return SGN_EINVAL;
  h->stream = (cudaStream_t)stream;
  return SGN_OK;
}

sgn_status sgn_bind(sgn_t h, void *dev_buf, size_t bytes, int32_t stores, void *stream) {
  if (!h || !dev_buf) return SGN_EINVAL;
  if (((uintptr_t)dev_buf & 255) != 0) { g_err = "device buffer must be 256-byte aligned"; return SGN_EINVAL; }
  size_t need = carve(*h, nullptr, stores, nullptr);
  if (need == 0) { g_err = "internal: a host plan (contribution-block arena, substitution schedule) failed its self-check"; return SGN_EINVAL; }
  if (bytes < need) return SGN_ENOMEM;
  h->stream = (cudaStream_t)stream;
  CUDA_TRY(h, cudaGetDevice(&h->device));
  CUDA_TRY(h, cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  // the fixed element-scratch array of sgn_assemble_static is resolved (and,
  // under lazy module loading, set up) here, never inside an assembly
  CUDA_TRY(h, static_scratch_bind(h->device));
  std::vector<Upload> ups;
  h->base = (char *)dev_buf;
  h->bytes = bytes;
  carve(*h, h->base, stores, &ups);
  std::vector<tc::Maps> maps32, mapsk;
  const char *tc_off = getenv("SGN_DISABLE_TC");
  const bool tc_ok = !(tc_off && tc_off[0] == '1');
  for (auto sm : {std::make_pair(&h->kkt32, &maps32), std::make_pair(&h->kf32, &mapsk)}) {
    Store &st = *sm.first;
    st.tc = false;
    if (st.enabled && tc_ok && encode_maps(*h, st, *sm.second)) {
      ups.push_back({st.maps, sm.second->data(), sm.second->size() * sizeof(tc::Maps)});
      st.tc = true;
    }
  }
  for (auto &u : ups) CUDA_TRY(h, cudaMemcpyAsync(u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->status, 0, 4 * sizeof(int), h->stream));
  // published solve values start untagged (no solve uses tag 0)
  for (Store *st : {&h->kkt64, &h->kkt32, &h->kf, &h->kf32}) {
    if (!st->enabled) continue;
    CUDA_TRY(h, cudaMemsetAsync(st->pub, 0, (size_t)st->piv_elems * sizeof(unsigned long long), h->stream));
    if (st->pflag) CUDA_TRY(h, cudaMemsetAsync(st->pflag, 0, (size_t)st->piv_elems * sizeof(unsigned), h->stream));
    if (st->bpart)
      CUDA_TRY(h, cudaMemsetAsync(st->bpart, 0, (size_t)st->part_elems * sizeof(unsigned long long), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(st->fflag, 0, 2 * (size_t)st->piv_elems * sizeof(unsigned), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(st->ctl, 0, 16 * sizeof(unsigned), h->stream));
  }
  // uploads read host vectors owned by h->S or by the carve's thread-local
  // staging; wait for them before those can change
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->stores = stores;
  set_kernel_attributes();
  if (!h->cap_stream) CUDA_TRY(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  if (!h->side_stream) CUDA_TRY(h, cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking));
  if (!h->ev_fork) CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  if (!h->ev_join) CUDA_TRY(h, cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  {
    const char *g = getenv("SGN_DISABLE_GRAPHS");
    h->use_graphs = !(g && g[0] == '1');
  }
  destroy_graphs(h->kkt64); destroy_graphs(h->kkt32); destroy_graphs(h->kf); destroy_graphs(h->kf32);
  if (h->step_graph) { cudaGraphExecDestroy(h->step_graph); h->step_graph = nullptr; }
  h->bound = true;
  h->assembled = false;
  h->inst_have_eq = h->inst_have_kkt = false;
  h->kkt64.factored = h->kkt32.factored = h->kf.factored = h->kf32.factored = false;
  if (h->pending_obj) {  // the joined objective of sgn_batch_setup
    sgn_objective o{(int32_t)h->pobj_track.size(), h->pobj_track.data(), h->pobj_target.data(),
                    h->pobj_weight.data(), h->pobj_alpha};
    sgn_status s = sgn_set_objective(h, &o);
    if (s != SGN_OK) return s;
  }
  return SGN_OK;
}

sgn_status sgn_set_objective(sgn_t h, const sgn_objective *obj) {
  if (!h || !obj || !h->bound) return h ? (h->bound ? SGN_EINVAL : SGN_ESTATE) : SGN_EINVAL;
  if (!(obj->alpha > 0.0) || obj->n_track < 0) { g_err = "objective: need alpha > 0"; return SGN_EINVAL; }
  const Symbolic &S = h->S;
  const int d = S.dim;
  std::vector<double> w((size_t)S.n_free * d, 0.0), t((size_t)S.n_free * d, 0.0);
  double wt2 = 0.0;  // sum w t^2 over the given entries
  for (int i = 0; i < obj->n_track; ++i) {
    int64_t g = obj->track_dof_h[i];
    if (g < 0 || g >= (int64_t)S.n_nodes * d) { g_err = "tracked DOF out of range"; return SGN_EINVAL; }
    int r = S.node_rank[g / d];
    if (r < 0) { g_err = "tracked DOF is fixed"; return SGN_EINVAL; }
    if (!std::isfinite(obj->weight_h[i])) { g_err = "weight is not finite"; return SGN_EINVAL; }
    int64_t rd = (int64_t)r * d + g % d;
    // repeated DOFs add up: sum_t w_t (x - target_t)^2 = (sum w)(x - wavg)^2 + const
    wt2 += obj->weight_h[i] * obj->target_h[i] * obj->target_h[i];
    double wn = w[rd] + obj->weight_h[i];
    t[rd] = wn != 0.0 ? (w[rd] * t[rd] + obj->weight_h[i] * obj->target_h[i]) / wn : 0.0;
    w[rd] = wn;
  }
  CUDA_TRY(h, cudaMemcpyAsync(h->wA, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->tgt, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  double merged = 0.0;
  for (size_t i = 0; i < w.size(); ++i) merged += w[i] * t[i] * t[i];
  h->f_const = 0.5 * (wt2 - merged);
  h->max_w = 0.0;
  for (double v : w) h->max_w = std::max(h->max_w, std::fabs(v));
  h->alpha = obj->alpha;
  h->have_objective = true;
  h->assembled = false;
  return SGN_OK;
}

void sgn_destroy(sgn_t h) {
  if (!h) return;
  if (h->bound) cudaStreamSynchronize(h->stream);
  destroy_graphs(h->kkt64); destroy_graphs(h->kkt32); destroy_graphs(h->kf); destroy_graphs(h->kf32);
  if (h->step_graph) cudaGraphExecDestroy(h->step_graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side_stream) cudaStreamDestroy(h->side_stream);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (cudaEvent_t e : h->prof_ev) cudaEventDestroy(e);
  delete h;
}

sgn_status sgn_assemble(sgn_t h, const double *x_d, const double *p_d) {
  if (!h || !x_d || !p_d) return SGN_EINVAL;
  if (!h->bound || !h->have_objective) return SGN_ESTATE;
  {
    ProfScope ps(*h, SGN_PROF_ELEMENTS);
    launch_elem_state(*h, x_d, p_d);
    launch_slot_gather(*h, true);
  }
  {
    ProfScope ps(*h, SGN_PROF_VECTOR);
    launch_objective_terms(*h, x_d, p_d);
  }
  h->assembled = true;
  h->kkt64.factored = h->kkt32.factored = h->kf.factored = h->kf32.factored = false;
  return launch_check(h);
}

sgn_status sgn_factor(sgn_t h, sgn_precision prec, sgn_factor_report *rep) {
  return sgn_factor_ex(h, prec, nullptr, rep);
}

sgn_status sgn_factor_ex(sgn_t h, sgn_precision prec, const sgn_factor_opts *opts, sgn_factor_report *rep) {
  if (!h) return SGN_EINVAL;
  const double ex = opts ? opts->eps_x : 0.0, el = opts ? opts->eps_lambda : 0.0;
  if (!(ex >= 0.0) || !(el >= 0.0)) { g_err = "stabilization must be >= 0"; return SGN_EINVAL; }
  if (!h->assembled) return SGN_ESTATE;
  Store &st = prec == SGN_MIXED ? h->kkt32 : h->kkt64;
  if (!st.enabled) { g_err = "store for this precision was not bound"; return SGN_ESTATE; }
  if (st.eps_x != ex || st.eps_l != el) {  // the captured factor graphs bake the old values in
    destroy_graphs(st);
    st.eps_x = ex;
    st.eps_l = el;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rep) {
    CUDA_TRY(h, cudaEventCreate(&e0)); CUDA_TRY(h, cudaEventCreate(&e1));
    CUDA_TRY(h, cudaEventRecord(e0, h->stream));
  }
  const int64_t tc0 = h->tc_launches;
  factor_store(*h, st);
  h->active = &st;
  sgn_status s = launch_check(h);
  if (s != SGN_OK) return s;
  if (rep) {
    CUDA_TRY(h, cudaEventRecord(e1, h->stream));
    pivot_counts(*h, st);
    int64_t ctr[8];
    CUDA_TRY(h, cudaMemcpyAsync(ctr, h->counters, sizeof(ctr), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    rep->n_perturbed = ctr[0]; rep->n_2x2 = ctr[1];
    rep->n_pos = ctr[2] + h->S.n_elem;  // p pivots: C = alpha I > 0
    rep->n_neg = ctr[3]; rep->n_zero = ctr[4];
    rep->seconds = ms * 1e-3;
    rep->tensor_core_updates = h->tc_launches - tc0;
    s = check_status(h);
    if (s != SGN_OK) return s;
  }
  return SGN_OK;
}

sgn_status sgn_factor_inertia(sgn_t h, sgn_precision prec, const sgn_inertia_opts *opts, double *delta_h,
                              sgn_factor_report *rep) {
  if (!h) return SGN_EINVAL;
  if (!h->assembled) return SGN_ESTATE;
  const double d0 = opts && opts->delta0 > 0 ? opts->delta0 : 1e-4 * std::max(h->max_w, 1e-300);
  const double grow = opts && opts->growth > 1 ? opts->growth : 10.0;
  const int tries = opts && opts->max_tries > 0 ? opts->max_tries : 30;
  const int64_t nx = (int64_t)h->S.n_free * h->S.dim, np = h->S.n_elem;
  double delta = 0.0;
  sgn_factor_report r{};
  for (int t = 0; t < tries; ++t) {
    sgn_factor_opts fo{delta, 0.0};
    sgn_status s = sgn_factor_ex(h, prec, &fo, &r);
    if (s != SGN_OK) return s;
    // the inertia (n_x + n_p, n_x, 0) <=> the reduced Hessian is positive
    // definite on the null space of the constraint Jacobian
    if (r.n_pos == nx + np && r.n_neg == nx && r.n_zero == 0) {
      if (delta_h) *delta_h = delta;
      if (rep) *rep = r;
      return SGN_OK;
    }
    delta = delta == 0.0 ? d0 : delta * grow;
  }
  set_error(h, "sgn_factor_inertia: no regularization up to the try limit gave the saddle-point inertia");
  if (delta_h) *delta_h = delta;
  if (rep) *rep = r;
  return SGN_EPIVOT;
}

sgn_status sgn_solve(sgn_t h, sgn_rhs_mode mode, const double *g_d, double *dx_d, double *dp_d, double *dl_d,
                     const sgn_solve_opts *opts, sgn_solve_report *rep) {
  if (!h || !dp_d) return SGN_EINVAL;
  if (mode == SGN_RHS_PAPER && !g_d) return SGN_EINVAL;
  Store *stp = (h->active && h->active->factored) ? h->active : nullptr;
  if (!stp) return SGN_ESTATE;
  Store &st = *stp;
  Ctx &c = *h;
  const int64_t nx = (int64_t)c.S.n_free * c.S.dim, ne = c.S.n_elem;
  int max_refine = opts && opts->max_refine > 0 ? opts->max_refine : (st.fp32 ? 30 : 2);
  double tol = opts && opts->tol > 0 ? opts->tol : 1e-12;
  const int method = opts ? opts->method : SGN_SOLVE_AUTO;
  if (method < SGN_SOLVE_AUTO || method > SGN_SOLVE_BICGSTAB) return SGN_EINVAL;
  // the system solved: M, or the factored M(delta) of an inertia correction
  struct ResEps {
    Ctx &c;
    ~ResEps() { c.res_eps_x = c.res_eps_l = 0.0; }
  } res_eps_reset{c};
  if (opts && opts->regularized) {
    c.res_eps_x = st.eps_x;
    c.res_eps_l = st.eps_l;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rep) {
    CUDA_TRY(h, cudaEventCreate(&e0)); CUDA_TRY(h, cudaEventCreate(&e1));
    CUDA_TRY(h, cudaEventRecord(e0, c.stream));
  }
  // right-hand side b = [b_x; b_p; b_l]
  if (mode == SGN_RHS_KKT) {
    CUDA_TRY(h, cudaMemsetAsync(c.bx, 0, nx * sizeof(double), c.stream));
    launch_axpy(c, c.bx, c.fx, -1.0, nx);
    CUDA_TRY(h, cudaMemsetAsync(c.bp, 0, ne * sizeof(double), c.stream));
    launch_axpy(c, c.bp, c.fp, -1.0, ne);
  } else {
    CUDA_TRY(h, cudaMemsetAsync(c.bx, 0, nx * sizeof(double), c.stream));
    CUDA_TRY(h, cudaMemsetAsync(c.bp, 0, ne * sizeof(double), c.stream));
    launch_axpy(c, c.bp, g_d, -1.0, ne);
  }
  CUDA_TRY(h, cudaMemsetAsync(c.bl, 0, nx * sizeof(double), c.stream));
  double *red_b = c.red, *red_x = c.red + 2 * nx;
  // z = M^{-1} b
  launch_reduce_rhs(c, c.bx, c.bp, c.bl, red_b, 2 * c.S.dim);
  solve_store(c, st, red_b, red_x);
  launch_recover(c, red_x, c.bp, c.zx, c.zp, c.zl);
  double bn = std::sqrt(device_sumsq3(c, c.bx, nx, c.bp, ne, c.bl, nx));
  double rn = 0.0, rn_prev = 0.0;
  int steps = 0, kits = 0;
  double hist[32];
  bool krylov = false;
  for (;;) {
    launch_residual(c, c.bx, c.bp, c.bl, c.zx, c.zp, c.zl, c.rx, c.rp, c.rl);
    rn = std::sqrt(device_sumsq3(c, c.rx, nx, c.rp, ne, c.rl, nx));
    if (steps < 32) hist[steps] = bn > 0 ? rn / bn : rn;
    if (!(rn == rn)) { h->last_error = "non-finite residual"; return SGN_ENONFINITE; }
    if (rn <= tol * bn) break;
    // stagnation at round-off level: the FP64 residual cannot fall further
    if (steps > 0 && rn > 0.5 * rn_prev && rn <= 1e-11 * bn) break;
    if (method == SGN_SOLVE_BICGSTAB || (method == SGN_SOLVE_AUTO && steps > 0 && rn > 0.5 * rn_prev)) {
      krylov = true;  // refinement no longer contracts: Krylov takes over from z
      break;
    }
    if (steps >= max_refine) {
      krylov = method == SGN_SOLVE_AUTO;
      break;
    }
    rn_prev = rn;
    launch_reduce_rhs(c, c.rx, c.rp, c.rl, red_b, 2 * c.S.dim);
    solve_store(c, st, red_b, red_x);
    // d = M^{-1} r, recovered into (rx, rp, rl) scratch then added
    launch_recover(c, red_x, c.rp, c.rx, c.rp, c.rl);
    launch_axpy(c, c.zx, c.rx, 1.0, nx);
    launch_axpy(c, c.zp, c.rp, 1.0, ne);
    launch_axpy(c, c.zl, c.rl, 1.0, nx);
    ++steps;
  }
  if (krylov) {
    // BiCGSTAB (van der Vorst 1992), right-preconditioned by the factor, on
    // M z = b from the current z; r = b - M z is in (rx, rp, rl).  Matrix
    // products go through the FP64 residual kernel with b = 0, which returns
    // -M v; the signs below account for it.
    const int max_k = opts && opts->max_krylov > 0 ? opts->max_krylov : 200;
    const int64_t n3 = 2 * nx + ne;
    auto vec = [&](int i) { return V3{c.kry + (size_t)i * n3, c.kry + (size_t)i * n3 + nx, c.kry + (size_t)i * n3 + nx + ne}; };
    const V3 R{c.rx, c.rp, c.rl}, Z{c.zx, c.zp, c.zl};
    const V3 Rh = vec(0), Pv = vec(1), Vn = vec(2), Y = vec(3), Sv = vec(4), Zt = vec(5), Tn = vec(6), O = vec(7);
    CUDA_TRY(h, cudaMemsetAsync(c.kry, 0, (size_t)Ctx::KRY_VECS * n3 * sizeof(double), c.stream));
    auto copy3 = [&](const V3 &d, const V3 &a) {
      cudaMemcpyAsync(d.x, a.x, nx * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
      cudaMemcpyAsync(d.p, a.p, ne * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
      cudaMemcpyAsync(d.l, a.l, nx * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
    };
    auto axpy3 = [&](const V3 &y, const V3 &x, double a) {
      launch_axpy(c, y.x, x.x, a, nx); launch_axpy(c, y.p, x.p, a, ne); launch_axpy(c, y.l, x.l, a, nx);
    };
    auto dot3 = [&](const V3 &a, const V3 &b) {
      return device_dot(c, a.x, b.x, nx) + device_dot(c, a.p, b.p, ne) + device_dot(c, a.l, b.l, nx);
    };
    auto neg_matvec = [&](const V3 &out, const V3 &in) {  // out = -M in
      launch_residual(c, O.x, O.p, O.l, in.x, in.p, in.l, out.x, out.p, out.l);
    };
    auto precond = [&](const V3 &out, const V3 &in) {  // out = (factor)^{-1} in
      launch_reduce_rhs(c, in.x, in.p, in.l, red_b, 2 * c.S.dim);
      solve_store(c, st, red_b, red_x);
      launch_recover(c, red_x, in.p, out.x, out.p, out.l);
    };
    copy3(Rh, R);
    double rho = 1.0, alpha = 1.0, omega = 1.0;
    for (kits = 0; kits < max_k;) {
      const double rho1 = dot3(Rh, R);
      if (rho1 == 0.0 || !std::isfinite(rho1)) break;  // breakdown
      const double beta = (rho1 / rho) * (alpha / omega);
      // p = r + beta (p - omega v), v = -Vn
      axpy3(Pv, Vn, beta == 0.0 ? 0.0 : omega);
      if (beta != 1.0) {  // p *= beta, then p += r
        V3 tmp = Pv;
        cudaMemsetAsync(Y.x, 0, nx * sizeof(double), c.stream);
        cudaMemsetAsync(Y.p, 0, ne * sizeof(double), c.stream);
        cudaMemsetAsync(Y.l, 0, nx * sizeof(double), c.stream);
        axpy3(Y, tmp, beta);
        copy3(Pv, Y);
      }
      axpy3(Pv, R, 1.0);
      precond(Y, Pv);
      neg_matvec(Vn, Y);
      const double rv = dot3(Rh, Vn);  // = -(rh . v)
      if (rv == 0.0 || !std::isfinite(rv)) break;
      alpha = -rho1 / rv;
      copy3(Sv, R);
      axpy3(Sv, Vn, alpha);  // s = r - alpha v
      axpy3(Z, Y, alpha);
      ++kits;
      const double sn = std::sqrt(dot3(Sv, Sv));
      if (sn <= tol * bn) { copy3(R, Sv); break; }
      precond(Zt, Sv);
      neg_matvec(Tn, Zt);
      const double tt = dot3(Tn, Tn);
      if (tt == 0.0 || !std::isfinite(tt)) { copy3(R, Sv); break; }
      omega = -dot3(Tn, Sv) / tt;  // (t . s) / (t . t)
      axpy3(Z, Zt, omega);
      copy3(R, Sv);
      axpy3(R, Tn, omega);  // r = s - omega t
      const double rk = std::sqrt(dot3(R, R));
      if (rk <= tol * bn || omega == 0.0) break;
      rho = rho1;
    }
    // the true FP64 residual of the final iterate
    launch_residual(c, c.bx, c.bp, c.bl, c.zx, c.zp, c.zl, c.rx, c.rp, c.rl);
    rn = std::sqrt(device_sumsq3(c, c.rx, nx, c.rp, ne, c.rl, nx));
    if (!(rn == rn)) { h->last_error = "non-finite residual"; return SGN_ENONFINITE; }
  }
  batch_record_solve(c);
  c.inst_have_kkt = c.n_inst > 0;
  if (dx_d) launch_to_nodes_plain(c, c.zx, dx_d);
  if (dl_d) launch_to_nodes_plain(c, c.zl, dl_d);
  CUDA_TRY(h, cudaMemcpyAsync(dp_d, c.zp, ne * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  sgn_status s = launch_check(h);
  if (s != SGN_OK) return s;
  s = check_status(h);  // bounded waits of the substitutions
  if (s != SGN_OK) return s;
  if (rep) {
    CUDA_TRY(h, cudaEventRecord(e1, c.stream));
    CUDA_TRY(h, cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    rep->refine_steps = steps;
    rep->krylov_iters = kits;
    rep->residual = bn > 0 ? rn / bn : rn;
    for (int i = 0; i < 32; ++i) rep->history[i] = i <= steps ? hist[i] : 0.0;
    rep->seconds = ms * 1e-3;
  }
  if (bn > 0 && rn > 1e-8 * bn) {
    h->last_error = "refinement left a residual above 1e-8 relative";
    return SGN_EREFINE;
  }
  return SGN_OK;
}

sgn_status sgn_step_host(sgn_t h, sgn_precision prec, const double *x_h, const double *p_h, double *dx_h,
                         double *dp_h, double *dl_h, sgn_solve_report *rep) {
  if (!h || !x_h || !p_h || !dp_h) return SGN_EINVAL;
  if (!h->bound) return SGN_ESTATE;
  Ctx &c = *h;
  const int64_t nn = (int64_t)c.S.n_nodes * c.S.dim, ne = c.S.n_elem;
  double *xd = c.hx, *dxd = c.hdx, *dld = c.hdl, *pd = c.hp, *dpd = c.hdp;
  CUDA_TRY(h, cudaMemcpyAsync(xd, x_h, nn * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  CUDA_TRY(h, cudaMemcpyAsync(pd, p_h, ne * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  sgn_status s = sgn_assemble(h, xd, pd);
  if (s != SGN_OK) return s;
  s = sgn_factor(h, prec, nullptr);
  if (s != SGN_OK) return s;
  s = sgn_solve(h, SGN_RHS_KKT, nullptr, dxd, dpd, dld, nullptr, rep);
  if (s != SGN_OK && s != SGN_EREFINE) return s;
  sgn_status s2 = s;
  CUDA_TRY(h, cudaMemcpyAsync(dp_h, dpd, ne * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  if (dx_h) CUDA_TRY(h, cudaMemcpyAsync(dx_h, dxd, nn * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  if (dl_h) CUDA_TRY(h, cudaMemcpyAsync(dl_h, dld, nn * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  CUDA_TRY(h, cudaStreamSynchronize(c.stream));
  s = check_status(h);
  return s != SGN_OK ? s : s2;
}

sgn_status sgn_export_kkt(sgn_t h, int64_t *nnz, int64_t *rows, int64_t *cols, double *vals) {
  if (!h || !nnz) return SGN_EINVAL;
  if (!h->assembled) return SGN_ESTATE;
  const Symbolic &S = h->S;
  const int d = S.dim, nv = d + 1;
  const int64_t ne = S.n_elem, nx = (int64_t)S.n_free * d, nnd = (int64_t)S.n_nodes * d;
  std::vector<double> wA(nx), Kv(S.bsr_col.size() * d * d), cpv((size_t)nv * d * ne);
  CUDA_TRY(h, cudaMemcpyAsync(wA.data(), h->wA, wA.size() * 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(Kv.data(), h->Kv, Kv.size() * 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(cpv.data(), h->cpv, cpv.size() * 8, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  int64_t n = 0;
  auto put = [&](int64_t r, int64_t c, double v) {
    if (rows) { rows[n] = r; cols[n] = c; vals[n] = v; }
    ++n;
  };
  auto xid = [&](int rank, int a) { return (int64_t)S.rank_node[rank] * d + a; };
  const int64_t pbase = nnd, lbase = nnd + ne;
  for (int r = 0; r < S.n_free; ++r)
    for (int a = 0; a < d; ++a)
      if (wA[(int64_t)r * d + a] != 0.0) put(xid(r, a), xid(r, a), wA[(int64_t)r * d + a]);
  for (int r = 0; r < S.n_free; ++r)
    for (int k = S.bsr_ptr[r]; k < S.bsr_ptr[r + 1]; ++k) {
      int c = S.bsr_col[k];
      for (int a = 0; a < d; ++a)
        for (int b = 0; b < d; ++b) {
          double v = Kv[(size_t)k * d * d + a * d + b];
          put(xid(r, a), lbase + xid(c, b), v);  // (x, lambda) block: K^T
          put(lbase + xid(r, a), xid(c, b), v);  // (lambda, x) block: K
        }
    }
  for (int64_t e = 0; e < ne; ++e) {
    put(pbase + e, pbase + e, h->alpha);
    for (int a = 0; a < nv; ++a) {
      int r = S.elem_rank[(size_t)a * ne + e];
      if (r < 0) continue;
      for (int i = 0; i < d; ++i) {
        double v = cpv[(size_t)(a * d + i) * ne + e];
        put(lbase + xid(r, i), pbase + e, v);
        put(pbase + e, lbase + xid(r, i), v);
      }
    }
  }
  if (rows && n != *nnz) return SGN_EINVAL;
  *nnz = n;
  return SGN_OK;
}

sgn_status sgn_profile(sgn_t h, int32_t mask) {
  if (!h) return SGN_EINVAL;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->harvest_graph_events();
  h->prof_mask = mask;
  h->prof_used = 0;
  h->prof_kind.clear();
  h->prof_fl.clear();
  for (int k = 0; k < 8; ++k) { h->gacc_sec[k] = 0.0; h->gacc_fl[k] = 0.0; h->gacc_n[k] = 0; }
  return SGN_OK;
}

sgn_status sgn_profile_read(sgn_t h, sgn_kernel_profile *out, int32_t n) {
  if (!h || !out || n < 0) return SGN_EINVAL;
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  h->harvest_graph_events();
  for (int k = 0; k < n; ++k)
    out[k] = sgn_kernel_profile{k < 8 ? h->gacc_n[k] : 0, k < 8 ? h->gacc_sec[k] : 0.0, k < 8 ? h->gacc_fl[k] : 0.0};
  for (int64_t i = 0; i < h->prof_used; ++i) {
    int k = h->prof_kind[i];
    if (k >= n) continue;
    float ms = 0.f;
    CUDA_TRY(h, cudaEventElapsedTime(&ms, h->prof_ev[2 * i], h->prof_ev[2 * i + 1]));
    out[k].launches += 1;
    out[k].seconds += ms * 1e-3;
    out[k].flops += h->prof_fl[i];
  }
  return SGN_OK;
}

int64_t sgn_launch_count(sgn_t h) { return h ? h->launches : -1; }

sgn_status sgn_step_graph(sgn_t h, sgn_precision prec, int32_t refine_steps, const double *x_d, const double *p_d,
                          double *dx_d, double *dp_d, double *dl_d, double *residual_h) {
  if (!h || !x_d || !p_d || !dp_d || refine_steps < 0 || refine_steps > 64) return SGN_EINVAL;
  if (!h->bound || !h->have_objective) return SGN_ESTATE;
  Store &st = prec == SGN_MIXED ? h->kkt32 : h->kkt64;
  if (!st.enabled) return SGN_ESTATE;
  if (!h->cap_stream) return SGN_ECUDA;
  if (st.eps_x != 0.0 || st.eps_l != 0.0) {  // the step graph factors M itself
    destroy_graphs(st);
    st.eps_x = st.eps_l = 0.0;
    if (h->step_graph) { cudaGraphExecDestroy(h->step_graph); h->step_graph = nullptr; }
  }
  Ctx &c = *h;
  const int64_t nx = (int64_t)c.S.n_free * c.S.dim, ne = c.S.n_elem;
  const void *key[6] = {x_d, p_d, dx_d, dp_d, dl_d, &st};
  bool same = h->step_graph && h->step_prec == (int)prec && h->step_refine == refine_steps;
  for (int i = 0; i < 6 && same; ++i) same = h->step_key[i] == key[i];
  if (!same) {
    if (h->step_graph) { cudaGraphExecDestroy(h->step_graph); h->step_graph = nullptr; }
    double *red_b = c.red, *red_x = c.red + 2 * nx;
    auto body = [&]() {
      launch_elem_state(c, x_d, p_d);
      launch_slot_gather(c, true);
      launch_objective_terms(c, x_d, p_d);
      factor_direct(c, st);
      cudaMemsetAsync(c.bx, 0, nx * sizeof(double), c.stream);
      launch_axpy(c, c.bx, c.fx, -1.0, nx);
      cudaMemsetAsync(c.bp, 0, ne * sizeof(double), c.stream);
      launch_axpy(c, c.bp, c.fp, -1.0, ne);
      cudaMemsetAsync(c.bl, 0, nx * sizeof(double), c.stream);
      launch_reduce_rhs(c, c.bx, c.bp, c.bl, red_b, 2 * c.S.dim);
      solve_direct(c, st, red_b, red_x);
      launch_recover(c, red_x, c.bp, c.zx, c.zp, c.zl);
      for (int it = 0; it < refine_steps; ++it) {
        launch_residual(c, c.bx, c.bp, c.bl, c.zx, c.zp, c.zl, c.rx, c.rp, c.rl);
        launch_reduce_rhs(c, c.rx, c.rp, c.rl, red_b, 2 * c.S.dim);
        solve_direct(c, st, red_b, red_x);
        launch_recover(c, red_x, c.rp, c.rx, c.rp, c.rl);
        launch_axpy(c, c.zx, c.rx, 1.0, nx);
        launch_axpy(c, c.zp, c.rp, 1.0, ne);
        launch_axpy(c, c.zl, c.rl, 1.0, nx);
      }
      launch_residual(c, c.bx, c.bp, c.bl, c.zx, c.zp, c.zl, c.rx, c.rp, c.rl);
      launch_sumsq3(c, c.rx, nx, c.rp, ne, c.rl, nx, c.partial2);
      launch_sumsq3(c, c.bx, nx, c.bp, ne, c.bl, nx, c.partial2 + c.n_partial);
      batch_record_solve(c);
      if (dx_d) launch_to_nodes_plain(c, c.zx, dx_d);
      if (dl_d) launch_to_nodes_plain(c, c.zl, dl_d);
      cudaMemcpyAsync(dp_d, c.zp, ne * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
    };
    const int mask = h->prof_mask;
    h->prof_mask = 0;  // no profiling events inside the step graph
    h->step_graph = capture_fn(c, body, &h->step_launches, &h->step_tc);
    h->prof_mask = mask;
    if (!h->step_graph) { h->last_error = "graph capture failed"; return SGN_ECUDA; }
    for (int i = 0; i < 6; ++i) h->step_key[i] = key[i];
    h->step_prec = (int)prec;
    h->step_refine = refine_steps;
  }
  CUDA_TRY(h, cudaGraphLaunch(h->step_graph, c.stream));
  c.inst_have_kkt = c.n_inst > 0;
  c.launches += h->step_launches;
  c.tc_launches += h->step_tc;
  c.assembled = true;
  st.factored = true;
  c.active = &st;
  if (residual_h) {
    std::vector<double> part(2 * c.n_partial);
    CUDA_TRY(h, cudaMemcpyAsync(part.data(), c.partial2, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                c.stream));
    CUDA_TRY(h, cudaStreamSynchronize(c.stream));
    double rr = 0.0, bb = 0.0;
    for (int i = 0; i < c.n_partial; ++i) { rr += part[i]; bb += part[c.n_partial + i]; }
    *residual_h = bb > 0 ? std::sqrt(rr / bb) : std::sqrt(rr);
    sgn_status s = check_status(h);
    if (s != SGN_OK) return s;
  }
  return SGN_OK;
}

sgn_status sgn_factor_k(sgn_t h) {
  if (!h) return SGN_EINVAL;
  if (!h->assembled) return SGN_ESTATE;
  if (!h->kf.enabled) { g_err = "K store was not bound"; return SGN_ESTATE; }
  factor_store(*h, h->kf);
  return launch_check(h);
}

sgn_status sgn_gradient(sgn_t h, double *g_d) {
  if (!h || !g_d) return SGN_EINVAL;
  if (!h->assembled || !h->kf.factored) return SGN_ESTATE;
  Ctx &c = *h;
  const int64_t nx = (int64_t)c.S.n_free * c.S.dim;
  double *b = c.eq, *lam = c.eq + nx;
  CUDA_TRY(h, cudaMemsetAsync(b, 0, nx * sizeof(double), c.stream));
  launch_axpy(c, b, c.fx, -1.0, nx);
  solve_store(c, c.kf, b, lam);  // lam = -K^{-1} f_x (K symmetric)
  launch_gradient_finish(c, lam, g_d);
  return launch_check(h);
}

sgn_status sgn_equilibrium(sgn_t h, const double *p_d, const double *fext_d, double *x_d,
                           const sgn_newton_opts *opts, sgn_newton_report *rep) {
  if (!h || !p_d || !fext_d || !x_d) return SGN_EINVAL;
  if (!h->bound) return SGN_ESTATE;
  const bool mixed = opts && opts->precision == SGN_MIXED;
  if (opts && opts->precision != SGN_FP64 && opts->precision != SGN_MIXED) return SGN_EINVAL;
  Store &kst = mixed ? h->kf32 : h->kf;
  if (!kst.enabled) {
    h->last_error = mixed ? "K FP32 store (SGN_STORE_KFACT_MIXED) was not bound" : "K store was not bound";
    return SGN_ESTATE;
  }
  Ctx &c = *h;
  auto t0 = std::chrono::steady_clock::now();
  const int d = c.S.dim;
  const int64_t nx = (int64_t)c.S.n_free * d, nn = (int64_t)c.S.n_nodes * d;
  const int max_iter = opts && opts->max_iter > 0 ? opts->max_iter : 50;
  const double tol = opts && opts->tol > 0 ? opts->tol : 1e-10;
  // The iterate is the displacement u = x - X (node-major, in c.ueq): F is
  // formed from it, so the round-off floor of ||c|| does not depend on where
  // the body sits (an absolute position carries eps |x| of representation
  // error, which alone floors ||c|| at a few 1e-10 ||f_ext|| here).
  double *fr = c.eq, *cr = fr + nx, *dxr = cr + nx, *tmp = dxr + nx;
  double *usave = c.xsave, *ur_tmp = c.xrt, *u = c.ueq;
  launch_from_nodes(c, fext_d, fr);
  launch_shift_rest(c, x_d, -1.0, u);
  const double fnorm = std::sqrt(device_sumsq3(c, fr, nx, nullptr, 0, nullptr, 0));
  const double scale = fnorm > 0 ? fnorm : 1.0;
  // Pi(u) = sum_e vol_e Psi(F_e) - f_ext . u  (the constant f_ext . X left out)
  auto potential = [&](const double *uu, bool *valid) -> double {
    int nbk = energy_blocks(c);
    launch_energy_partials(c, uu, p_d, c.partial, nbk, true);
    std::vector<double> hp(nbk);
    cudaMemcpyAsync(hp.data(), c.partial, nbk * sizeof(double), cudaMemcpyDeviceToHost, c.stream);
    cudaStreamSynchronize(c.stream);
    double e = 0.0;
    for (double v : hp) e += v;
    *valid = std::isfinite(e);
    launch_from_nodes(c, uu, ur_tmp);
    double w = device_dot(c, fr, ur_tmp, nx);
    return e - w;
  };
  auto residual = [&](const double *uu) -> double {
    launch_elem_state_disp(c, uu, p_d);
    launch_internal_force(c, cr);
    launch_axpy(c, cr, fr, -1.0, nx);
    return std::sqrt(device_sumsq3(c, cr, nx, nullptr, 0, nullptr, 0));
  };
  bool valid = true;
  double Pi = potential(u, &valid);
  if (!valid) { c.last_error = "initial guess has an inverted element"; return SGN_EINVERTED; }
  double cn = residual(u);
  double init = cn / scale;
  int it = 0, solves = 0;
  bool conv = false, dir_ok = true;
  double cn_prev = -1.0;
  double hist[32] = {0}, tstep[32] = {0};
  for (;; ++it) {
    if (it < 32) hist[it] = cn / scale;
    // converged, or (for a tolerance below the round-off floor) stagnating:
    // a full-accuracy Newton step no longer halves ||c|| and it is already
    // below kStagnationCap ||f_ext||
    if (cn <= tol * scale || (dir_ok && cn_prev > 0 && cn > 0.5 * cn_prev && cn <= kStagnationCap * scale)) {
      conv = true;
      break;
    }
    cn_prev = cn;
    if (it >= max_iter) break;
    // Newton direction: K du = -c.  Every solve goes through (c.rx -> c.zx)
    // so that the captured substitution graph is reused; with FP32 fronts the
    // direction is refined against the FP64 K until ||K du + c|| <= eta ||c||
    launch_slot_gather(c, false);
    c.assembled = true;
    factor_store(c, kst);
    CUDA_TRY(h, cudaMemsetAsync(tmp, 0, nx * sizeof(double), c.stream));
    launch_axpy(c, tmp, cr, -1.0, nx);
    CUDA_TRY(h, cudaMemsetAsync(dxr, 0, nx * sizeof(double), c.stream));
    CUDA_TRY(h, cudaMemcpyAsync(c.rx, tmp, nx * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    const double eta = std::min(0.1, cn / scale);
    dir_ok = !mixed;
    for (int q = 0;; ++q) {
      solve_store(c, kst, c.rx, c.zx);
      launch_axpy(c, dxr, c.zx, 1.0, nx);
      ++solves;
      if (!mixed || q >= 9) break;
      launch_residual_k(c, tmp, dxr, c.rx);
      if (std::sqrt(device_sumsq3(c, c.rx, nx, nullptr, 0, nullptr, 0)) <= eta * cn) {
        dir_ok = true;
        break;
      }
    }
    double slope = device_dot(c, cr, dxr, nx);
    CUDA_TRY(h, cudaMemcpyAsync(usave, u, nn * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    double t = 1.0, Pit = 0.0;
    bool acc = false;
    for (int hv = 0; hv < 40; ++hv) {
      launch_positions_update(c, usave, dxr, t, u);
      bool ok = true;
      Pit = potential(u, &ok);
      if (ok) {
        if (Pit <= Pi + 1e-4 * t * slope) { acc = true; break; }
        if (std::fabs(t * slope) <= 1e-13 * std::max(std::fabs(Pi), 1e-300)) {
          double cnt = residual(u);
          if (cnt < cn) { acc = true; break; }
        }
      }
      t *= 0.5;
    }
    if (!acc) {
      launch_positions_update(c, usave, dxr, 1.0, u);
      bool ok = true;
      Pit = potential(u, &ok);
      if (!ok) {
        CUDA_TRY(h, cudaMemcpyAsync(u, usave, nn * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        break;
      }
    }
    if (it < 32) tstep[it] = acc ? t : 1.0;
    Pi = Pit;
    cn = residual(u);
  }
  launch_shift_rest(c, u, 1.0, x_d);  // x = X + u
  batch_record_equilibrium(c, cr, fr);
  c.inst_have_eq = c.n_inst > 0;
  c.kf.factored = c.kf32.factored = false;  // K factor belongs to an earlier iterate
  c.assembled = false;
  if (c.active) c.active->factored = false;
  sgn_status s = launch_check(h);
  if (s != SGN_OK) return s;
  CUDA_TRY(h, cudaStreamSynchronize(c.stream));
  if (rep) {
    rep->iters = it; rep->converged = conv ? 1 : 0;
    rep->residual = cn / scale; rep->initial_residual = init;
    rep->solves = solves;
    for (int q = 0; q < 32; ++q) { rep->history[q] = hist[q]; rep->step_length[q] = tstep[q]; }
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  int stw = 0;
  CUDA_TRY(h, cudaMemcpy(&stw, c.status, sizeof(int), cudaMemcpyDeviceToHost));
  if (stw) CUDA_TRY(h, cudaMemset(c.status, 0, sizeof(int)));
  return conv ? SGN_OK : SGN_ENEWTON;
}

}  // extern "C"
