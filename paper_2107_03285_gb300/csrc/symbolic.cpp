// Host symbolic phase: node graph, geometric nested dissection, elimination
// tree, supernodes, front maps, block pattern of K and element slot maps.
#include "symbolic.h"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

namespace sgn {

namespace {

struct NDBuilder {
  int dim;
  const double *X;
  const std::vector<std::vector<int>> &adj;   // over original node ids (free nodes only)
  int leaf;
  std::vector<uint8_t> mark;                  // scratch: 0 none, 1 L, 2 R
  std::vector<int> comp;                      // scratch: component label, -1 outside the current set
  // output: supernodes as lists of original node ids in postorder
  std::vector<std::vector<int>> groups;

  NDBuilder(int d, const double *x, const std::vector<std::vector<int>> &a, int lf, int n)
      : dim(d), X(x), adj(a), leaf(lf), mark(n, 0), comp(n, -1) {}

  // A disconnected node set (e.g. many independent design instances in one
  // mesh) needs no separator: each connected component is dissected on its
  // own and becomes its own subtree of the elimination forest.  Returns
  // false (and leaves the scratch clean) when ids is connected.
  bool split_components(const std::vector<int> &ids) {
    for (int v : ids) comp[v] = -2;  // member, not yet labelled
    std::vector<std::vector<int>> parts;
    std::vector<int> stack;
    for (int v0 : ids) {
      if (comp[v0] != -2) continue;
      const int label = (int)parts.size();
      parts.emplace_back();
      comp[v0] = label;
      stack.push_back(v0);
      while (!stack.empty()) {
        const int u = stack.back();
        stack.pop_back();
        parts[label].push_back(u);
        for (int w : adj[u])
          if (comp[w] == -2) { comp[w] = label; stack.push_back(w); }
      }
    }
    for (int v : ids) comp[v] = -1;
    if (parts.size() < 2) return false;
    for (auto &p : parts) build(std::move(p));
    return true;
  }

  double coord(int v, int ax) const { return X[(int64_t)v * dim + ax]; }

  void sort_lex(std::vector<int> &ids, int first_axis) const {
    std::sort(ids.begin(), ids.end(), [&](int a, int b) {
      for (int k = 0; k < dim; ++k) {
        int ax = (first_axis + k) % dim;
        double ca = coord(a, ax), cb = coord(b, ax);
        if (ca < cb) return true;
        if (ca > cb) return false;
      }
      return a < b;
    });
  }

  void build(std::vector<int> ids) {
    if ((int)ids.size() <= leaf) {
      sort_lex(ids, dim - 1);
      groups.push_back(std::move(ids));
      return;
    }
    if (split_components(ids)) return;
    // split along the axis of largest extent
    int axis = 0;
    double best = -1.0;
    for (int ax = 0; ax < dim; ++ax) {
      double lo = 1e300, hi = -1e300;
      for (int v : ids) { lo = std::min(lo, coord(v, ax)); hi = std::max(hi, coord(v, ax)); }
      if (hi - lo > best * (1.0 + 1e-12)) { best = hi - lo; axis = ax; }
    }
    sort_lex(ids, axis);
    size_t h = ids.size() / 2;
    double v = coord(ids[h], axis);
    double eps = 1e-9 * std::max(best, 1e-300);
    std::vector<int> L, R, S;
    for (int u : ids) {
      double c = coord(u, axis);
      if (c < v - eps) L.push_back(u);
      else if (c > v + eps) R.push_back(u);
      else S.push_back(u);
    }
    // the plane of nodes at the median coordinate separates the two sides
    // on structured meshes; check it, else fall back to the boundary of the
    // first half as a vertex separator
    bool ok = !S.empty();
    if (ok) {
      for (int u : R) mark[u] = 2;
      for (int u : L) {
        for (int w : adj[u]) if (mark[w] == 2) { ok = false; break; }
        if (!ok) break;
      }
      for (int u : R) mark[u] = 0;
    }
    if (!ok) {
      L.assign(ids.begin(), ids.begin() + h);
      R.assign(ids.begin() + h, ids.end());
      S.clear();
      for (int u : R) mark[u] = 2;
      std::vector<int> L2;
      for (int u : L) {
        bool b = false;
        for (int w : adj[u]) if (mark[w] == 2) { b = true; break; }
        (b ? S : L2).push_back(u);
      }
      for (int u : R) mark[u] = 0;
      L.swap(L2);
    }
    if (L.empty() && R.empty()) {
      sort_lex(S, dim - 1);
      groups.push_back(std::move(S));
      return;
    }
    if (!L.empty()) build(std::move(L));
    if (!R.empty()) build(std::move(R));
    if (!S.empty()) {
      sort_lex(S, (axis + 1) % dim);
      groups.push_back(std::move(S));
    }
  }
};

template <typename T>
void sort_unique(std::vector<T> &v) {
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
}

}  // namespace

std::string analyze(int dim, int n_nodes, int n_elem, const double *X, const int32_t *conn,
                    const uint8_t *fixed, const SymbolicOptions &opts_in, Symbolic &S) {
  auto t0 = std::chrono::steady_clock::now();
  if (dim != 2 && dim != 3) return "dim must be 2 or 3";
  if (n_nodes <= 0 || n_elem <= 0) return "empty mesh";
  if (!X || !conn || !fixed) return "null mesh array";
  SymbolicOptions opts = opts_in;
  if (opts.leaf_nodes <= 0) opts.leaf_nodes = 16;
  if (opts.panel <= 0) opts.panel = 32;
  // panels tile the 256-column outer blocks exactly: 8, 16 or 32
  if (opts.panel != 8 && opts.panel != 16 && opts.panel != 32)
    return "panel must be 8, 16 or 32";
  const int nv = dim + 1;
  S = Symbolic();
  S.dim = dim; S.n_nodes = n_nodes; S.n_elem = n_elem; S.opts = opts;
  S.X.assign(X, X + (int64_t)n_nodes * dim);
  for (int64_t i = 0; i < (int64_t)n_elem * nv; ++i)
    if (conn[i] < 0 || conn[i] >= n_nodes) return "connectivity index out of range";

  // ---- element rest geometry: D_m, vol, shape-function gradients B
  S.elem_B.assign((int64_t)nv * dim * n_elem, 0.0);
  S.elem_vol.assign(n_elem, 0.0);
  for (int e = 0; e < n_elem; ++e) {
    const int32_t *c = conn + (int64_t)e * nv;
    double Dm[3][3] = {{0}};
    for (int a = 1; a <= dim; ++a)
      for (int i = 0; i < dim; ++i) Dm[i][a - 1] = X[(int64_t)c[a] * dim + i] - X[(int64_t)c[0] * dim + i];
    double det, inv[3][3];
    if (dim == 2) {
      det = Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0];
      if (!(std::fabs(det) > 0.0)) return "degenerate element";
      inv[0][0] = Dm[1][1] / det; inv[0][1] = -Dm[0][1] / det;
      inv[1][0] = -Dm[1][0] / det; inv[1][1] = Dm[0][0] / det;
      S.elem_vol[e] = std::fabs(det) / 2.0;
    } else {
      double c00 = Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1];
      double c01 = Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2];
      double c02 = Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0];
      det = Dm[0][0] * c00 + Dm[0][1] * c01 + Dm[0][2] * c02;
      if (!(std::fabs(det) > 0.0)) return "degenerate element";
      inv[0][0] = c00 / det;
      inv[1][0] = c01 / det;
      inv[2][0] = c02 / det;
      inv[0][1] = (Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2]) / det;
      inv[1][1] = (Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0]) / det;
      inv[2][1] = (Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1]) / det;
      inv[0][2] = (Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1]) / det;
      inv[1][2] = (Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2]) / det;
      inv[2][2] = (Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0]) / det;
      S.elem_vol[e] = std::fabs(det) / 6.0;
    }
    // F_ij = sum_a x_{a,i} B_{a,j}: B_a = row a-1 of D_m^{-1}, B_0 = -sum
    for (int j = 0; j < dim; ++j) {
      double s = 0.0;
      for (int a = 1; a <= dim; ++a) {
        S.elem_B[((int64_t)(a * dim + j)) * n_elem + e] = inv[a - 1][j];
        s += inv[a - 1][j];
      }
      S.elem_B[((int64_t)j) * n_elem + e] = -s;
    }
  }

  // ---- free nodes and their graph
  std::vector<std::vector<int>> adj(n_nodes);
  for (int e = 0; e < n_elem; ++e) {
    const int32_t *c = conn + (int64_t)e * nv;
    for (int a = 0; a < nv; ++a) {
      if (fixed[c[a]]) continue;
      for (int b = 0; b < nv; ++b)
        if (b != a && !fixed[c[b]]) adj[c[a]].push_back(c[b]);
    }
  }
  std::vector<int> free_ids;
  for (int v = 0; v < n_nodes; ++v) {
    if (!fixed[v]) free_ids.push_back(v);
    sort_unique(adj[v]);
  }
  S.n_free = (int)free_ids.size();
  if (S.n_free == 0) return "no free nodes";
  {
    // every free node must belong to an element with another free node or be
    // in some element at all (a node in no element has a singular K row)
    std::vector<uint8_t> used(n_nodes, 0);
    for (int64_t i = 0; i < (int64_t)n_elem * nv; ++i) used[conn[i]] = 1;
    for (int v : free_ids) if (!used[v]) return "free node in no element";
  }

  // ---- nested dissection ordering (geometric bisection of the node graph)
  NDBuilder nd(dim, X, adj, opts.leaf_nodes, n_nodes);
  nd.build(free_ids);
  S.node_rank.assign(n_nodes, -1);
  S.rank_node.resize(S.n_free);
  {
    int r = 0;
    for (auto &g : nd.groups) {
      Supernode s;
      s.first = r;
      s.nown = (int)g.size();
      for (int v : g) { S.node_rank[v] = r; S.rank_node[r] = v; ++r; }
      S.sn.push_back(s);
    }
  }
  const int n_sn = (int)S.sn.size();
  S.sn_of_rank.resize(S.n_free);
  for (int s = 0; s < n_sn; ++s)
    for (int i = 0; i < S.sn[s].nown; ++i) S.sn_of_rank[S.sn[s].first + i] = s;

  // ---- block pattern of K in rank space
  std::vector<std::vector<int>> radj(S.n_free);
  for (int r = 0; r < S.n_free; ++r) {
    int v = S.rank_node[r];
    radj[r].push_back(r);
    for (int w : adj[v]) radj[r].push_back(S.node_rank[w]);
    std::sort(radj[r].begin(), radj[r].end());
  }
  S.bsr_ptr.assign(S.n_free + 1, 0);
  for (int r = 0; r < S.n_free; ++r) S.bsr_ptr[r + 1] = S.bsr_ptr[r] + (int)radj[r].size();
  S.bsr_col.resize(S.bsr_ptr[S.n_free]);
  S.bsr_diag.resize(S.n_free);
  for (int r = 0; r < S.n_free; ++r) {
    std::copy(radj[r].begin(), radj[r].end(), S.bsr_col.begin() + S.bsr_ptr[r]);
    for (int k = S.bsr_ptr[r]; k < S.bsr_ptr[r + 1]; ++k)
      if (S.bsr_col[k] == r) S.bsr_diag[r] = k;
  }
  auto slot_of = [&](int r, int c) -> int {
    auto b = S.bsr_col.begin() + S.bsr_ptr[r], en = S.bsr_col.begin() + S.bsr_ptr[r + 1];
    auto it = std::lower_bound(b, en, c);
    return (it != en && *it == c) ? (int)(it - S.bsr_col.begin()) : -1;
  };

  // ---- supernodal symbolic factorization: struct(s), etree, levels
  std::vector<std::vector<int>> sstruct(n_sn);
  std::vector<std::vector<int>> kids(n_sn);
  std::vector<int> mark(S.n_free, -1);
  for (int s = 0; s < n_sn; ++s) {
    Supernode &sn = S.sn[s];
    int last = sn.first + sn.nown - 1;
    std::vector<int> st;
    for (int i = 0; i < sn.nown; ++i) {
      int r = sn.first + i;
      for (int c : radj[r]) if (c > last && mark[c] != s) { mark[c] = s; st.push_back(c); }
    }
    for (int c : kids[s])
      for (int r : sstruct[c]) if (r > last && mark[r] != s) { mark[r] = s; st.push_back(r); }
    std::sort(st.begin(), st.end());
    sstruct[s] = st;
    if (!st.empty()) {
      int p = S.sn_of_rank[st[0]];
      sn.parent = p;
      kids[p].push_back(s);
    }
    int lv = 0;
    for (int c : kids[s]) lv = std::max(lv, S.sn[c].level + 1);
    sn.level = lv;
  }
  int64_t off = 0;
  for (int s = 0; s < n_sn; ++s) {
    S.sn[s].nstruct = (int)sstruct[s].size();
    S.sn[s].struct_off = off;
    off += S.sn[s].nstruct;
  }
  S.struct_ranks.resize(off);
  S.relpos.assign(off, -1);
  for (int s = 0; s < n_sn; ++s)
    std::copy(sstruct[s].begin(), sstruct[s].end(), S.struct_ranks.begin() + S.sn[s].struct_off);

  // front position of rank r inside the front of supernode s (-1 if absent)
  auto front_pos = [&](int s, int r) -> int {
    const Supernode &sn = S.sn[s];
    if (r >= sn.first && r < sn.first + sn.nown) return r - sn.first;
    auto b = sstruct[s].begin(), en = sstruct[s].end();
    auto it = std::lower_bound(b, en, r);
    if (it != en && *it == r) return sn.nown + (int)(it - b);
    return -1;
  };
  for (int s = 0; s < n_sn; ++s) {
    int p = S.sn[s].parent;
    if (p < 0) continue;
    for (int q = 0; q < S.sn[s].nstruct; ++q) {
      int pos = front_pos(p, sstruct[s][q]);
      if (pos < 0) return "internal error: struct not contained in parent front";
      S.relpos[S.sn[s].struct_off + q] = pos;
    }
  }
  // children lists and inverse maps
  for (int s = 0; s < n_sn; ++s) {
    S.sn[s].child_off = (int)S.children.size();
    S.sn[s].nchild = (int)kids[s].size();
    for (int c : kids[s]) {
      S.children.push_back(c);
      S.cmap_off.push_back((int64_t)S.cmap.size());
      size_t base = S.cmap.size();
      S.cmap.resize(base + S.sn[s].fnodes(), -1);
      for (int q = 0; q < S.sn[c].nstruct; ++q) S.cmap[base + S.relpos[S.sn[c].struct_off + q]] = q;
    }
  }
  // original entries: slot (r, c), c >= r, lands in owner(r)'s front
  S.bsr_orig_pos.assign(S.bsr_col.size(), -1);
  for (int r = 0; r < S.n_free; ++r) {
    int s = S.sn_of_rank[r];
    for (int k = S.bsr_ptr[r]; k < S.bsr_ptr[r + 1]; ++k) {
      int c = S.bsr_col[k];
      if (c < r) continue;
      int pos = front_pos(s, c);
      if (pos < 0) return "internal error: original entry outside its front";
      S.bsr_orig_pos[k] = pos;
    }
  }
  // levels
  S.n_levels = 0;
  for (auto &sn : S.sn) S.n_levels = std::max(S.n_levels, sn.level + 1);
  S.level_fronts.assign(S.n_levels, {});
  for (int s = 0; s < n_sn; ++s) S.level_fronts[S.sn[s].level].push_back(s);
  for (auto &lf : S.level_fronts)
    std::stable_sort(lf.begin(), lf.end(), [&](int a, int b) { return S.sn[a].nown > S.sn[b].nown; });

  // ---- element ranks, gather map for upper slots, incidence
  S.elem_node.resize((int64_t)nv * n_elem);
  S.elem_rank.resize((int64_t)nv * n_elem);
  for (int e = 0; e < n_elem; ++e)
    for (int a = 0; a < nv; ++a) {
      int v = conn[(int64_t)e * nv + a];
      S.elem_node[(int64_t)a * n_elem + e] = v;
      S.elem_rank[(int64_t)a * n_elem + e] = S.node_rank[v];
    }
  // upper slot numbering
  std::vector<int32_t> upper_id(S.bsr_col.size(), -1);
  for (int r = 0; r < S.n_free; ++r)
    for (int k = S.bsr_ptr[r]; k < S.bsr_ptr[r + 1]; ++k)
      if (S.bsr_col[k] >= r) {
        upper_id[k] = (int)S.up_slot.size();
        S.up_slot.push_back(k);
        S.up_slot_t.push_back(slot_of(S.bsr_col[k], r));
      }
  const int n_up = (int)S.up_slot.size();
  std::vector<int32_t> cnt(n_up + 1, 0);
  std::vector<std::pair<int, int32_t>> contribs;
  contribs.reserve((size_t)n_elem * nv * (nv + 1) / 2);
  for (int e = 0; e < n_elem; ++e)
    for (int a = 0; a < nv; ++a) {
      int ra = S.elem_rank[(int64_t)a * n_elem + e];
      if (ra < 0) continue;
      for (int b = 0; b < nv; ++b) {
        int rb = S.elem_rank[(int64_t)b * n_elem + e];
        if (rb < 0 || rb < ra || (rb == ra && b != a)) continue;
        int k = slot_of(ra, rb);
        int u = upper_id[k];
        contribs.emplace_back(u, e * 16 + a * 4 + b);
      }
    }
  std::stable_sort(contribs.begin(), contribs.end(),
                   [](const std::pair<int, int32_t> &x, const std::pair<int, int32_t> &y) { return x.first < y.first; });
  S.up_ptr.assign(n_up + 1, 0);
  for (auto &c : contribs) S.up_ptr[c.first + 1]++;
  for (int u = 0; u < n_up; ++u) S.up_ptr[u + 1] += S.up_ptr[u];
  S.up_contrib.resize(contribs.size());
  for (size_t i = 0; i < contribs.size(); ++i) S.up_contrib[i] = contribs[i].second;

  S.inc_ptr.assign(S.n_free + 1, 0);
  for (int e = 0; e < n_elem; ++e)
    for (int a = 0; a < nv; ++a) {
      int r = S.elem_rank[(int64_t)a * n_elem + e];
      if (r >= 0) S.inc_ptr[r + 1]++;
    }
  for (int r = 0; r < S.n_free; ++r) S.inc_ptr[r + 1] += S.inc_ptr[r];
  S.inc.resize(S.inc_ptr[S.n_free]);
  {
    std::vector<int32_t> fill(S.inc_ptr.begin(), S.inc_ptr.end() - 1);
    for (int e = 0; e < n_elem; ++e)
      for (int a = 0; a < nv; ++a) {
        int r = S.elem_rank[(int64_t)a * n_elem + e];
        if (r >= 0) S.inc[fill[r]++] = e * 4 + a;
      }
  }

  // ---- statistics
  auto flops_of = [](double f, double ns) {
    double fl = 0.0;
    for (int64_t j = 0; j < (int64_t)ns; ++j) {
      double t = f - j - 1;
      fl += t * (t + 1) + t;
    }
    return fl;
  };
  const int dkkt = 2 * dim;
  for (auto &sn : S.sn) {
    int64_t fn = sn.fnodes();
    S.max_front_nodes = std::max(S.max_front_nodes, fn);
    S.sum_f2_nodes += fn * fn;
    int64_t f = fn * dkkt, ns = (int64_t)sn.nown * dkkt;
    S.nnz_factor_kkt += ns * (ns + 1) / 2 + ns * (f - ns);
    S.flops_kkt += flops_of((double)f, (double)ns);
    S.flops_k += flops_of((double)fn * dim, (double)sn.nown * dim);
  }
  S.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return "";
}

}  // namespace sgn
