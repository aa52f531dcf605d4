// Batched design instances behind one handle: sgn_batch_setup joins n
// independent meshes (and their objectives) into one disjoint system, whose
// saddle-point matrix is block diagonal by instance.  The symbolic phase
// splits the node graph into its connected components before any separator
// is sought, so every instance is its own subtree of one elimination forest
// and every level's fronts of every instance share the same launches.
// Instances keep their own coordinates (they may overlap in space).
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

namespace sgn {

namespace {

constexpr int TPB = 256;

// acc[inst[i / per]] += v[i]^2 over n entries (per consecutive entries share
// one owner); lanes of a warp that share an instance add once
__global__ void k_inst_sumsq(int64_t n, int per, const double *__restrict__ v, const int32_t *__restrict__ inst,
                             double *__restrict__ acc) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool ok = i < n;
  const int key = ok ? inst[i / per] : -1;
  double x = ok ? v[i] * v[i] : 0.0;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  // sum over the peer lanes (a segmented reduction inside the warp)
  double s = 0.0;
  for (unsigned m = peers; m; m &= m - 1) s += __shfl_sync(peers, x, __ffs(m) - 1);
  if (ok && lane == leader) atomicAdd(acc + key, s);
}

}  // namespace

void launch_inst_sumsq(Ctx &c, const double *v, int64_t n, int per, const int32_t *inst, double *acc) {
  if (n <= 0) return;
  k_inst_sumsq<<<(unsigned)((n + TPB - 1) / TPB), TPB, 0, c.stream>>>(n, per, v, inst, acc);
  c.count();
}

// per-instance ||c_i||^2 and ||f_ext,i||^2 of the last Newton iterate
void batch_record_equilibrium(Ctx &c, const double *cr, const double *fr) {
  if (c.n_inst <= 0) return;
  const int d = c.S.dim;
  cudaMemsetAsync(c.inst_acc, 0, 2 * (size_t)c.n_inst * sizeof(double), c.stream);
  launch_inst_sumsq(c, cr, (int64_t)c.S.n_free * d, d, c.rank_inst, c.inst_acc);
  launch_inst_sumsq(c, fr, (int64_t)c.S.n_free * d, d, c.rank_inst, c.inst_acc + c.n_inst);
}

// per-instance ||r_i||^2 and ||b_i||^2 of the last solve of the saddle-point
// system (r in rx / rp / rl, b in bx / bp / bl)
void batch_record_solve(Ctx &c) {
  if (c.n_inst <= 0) return;
  const int d = c.S.dim;
  const int64_t nx = (int64_t)c.S.n_free * d, ne = c.S.n_elem;
  double *a = c.inst_acc + 2 * c.n_inst;
  cudaMemsetAsync(a, 0, 2 * (size_t)c.n_inst * sizeof(double), c.stream);
  launch_inst_sumsq(c, c.rx, nx, d, c.rank_inst, a);
  launch_inst_sumsq(c, c.rp, ne, 1, c.elem_inst, a);
  launch_inst_sumsq(c, c.rl, nx, d, c.rank_inst, a);
  launch_inst_sumsq(c, c.bx, nx, d, c.rank_inst, a + c.n_inst);
  launch_inst_sumsq(c, c.bp, ne, 1, c.elem_inst, a + c.n_inst);
  launch_inst_sumsq(c, c.bl, nx, d, c.rank_inst, a + c.n_inst);
}

}  // namespace sgn

extern "C" {

sgn_status sgn_batch_setup(int32_t n, const sgn_mesh *meshes, const sgn_objective *objectives,
                           const sgn_setup_opts *opts, sgn_t *out) {
  if (!out) return SGN_EINVAL;
  *out = nullptr;
  if (n <= 0 || !meshes) {
    sgn::set_error(nullptr, "sgn_batch_setup: need n >= 1 meshes");
    return SGN_EINVAL;
  }
  const int d = meshes[0].dim;
  int64_t nn = 0, ne = 0, nt = 0;
  for (int i = 0; i < n; ++i) {
    const sgn_mesh &m = meshes[i];
    if (m.dim != d || m.E0 != meshes[0].E0 || m.nu != meshes[0].nu) {
      sgn::set_error(nullptr, "sgn_batch_setup: every instance needs the same dim, E0 and nu (instance " +
                                  std::to_string(i) + ")");
      return SGN_EINVAL;
    }
    if (m.n_nodes <= 0 || m.n_elem <= 0 || !m.X_h || !m.conn_h || !m.fixed_h) {
      sgn::set_error(nullptr, "sgn_batch_setup: empty or incomplete mesh (instance " + std::to_string(i) + ")");
      return SGN_EINVAL;
    }
    if (objectives) {
      const sgn_objective &o = objectives[i];
      if (o.alpha != objectives[0].alpha || o.n_track < 0 || (o.n_track > 0 && (!o.track_dof_h || !o.target_h ||
                                                                                   !o.weight_h))) {
        sgn::set_error(nullptr, "sgn_batch_setup: objectives need the same alpha and complete arrays (instance " +
                                    std::to_string(i) + ")");
        return SGN_EINVAL;
      }
      nt += o.n_track;
    }
    nn += m.n_nodes;
    ne += m.n_elem;
  }
  if (nn > INT32_MAX / 4 || ne > INT32_MAX / 16) {
    sgn::set_error(nullptr, "sgn_batch_setup: the joined mesh is too large");
    return SGN_EINVAL;
  }
  std::vector<double> X;
  std::vector<int32_t> conn;
  std::vector<uint8_t> fixed;
  std::vector<int64_t> node_off(1, 0), elem_off(1, 0);
  std::vector<int64_t> track;
  std::vector<double> target, weight;
  try {
    X.reserve((size_t)nn * d); conn.reserve((size_t)ne * (d + 1)); fixed.reserve((size_t)nn);
    track.reserve((size_t)nt); target.reserve((size_t)nt); weight.reserve((size_t)nt);
    for (int i = 0; i < n; ++i) {
      const sgn_mesh &m = meshes[i];
      const int64_t off = node_off.back();
      X.insert(X.end(), m.X_h, m.X_h + (int64_t)m.n_nodes * d);
      for (int64_t k = 0; k < (int64_t)m.n_elem * (d + 1); ++k) {
        const int32_t v = m.conn_h[k];
        if (v < 0 || v >= m.n_nodes) {
          sgn::set_error(nullptr, "sgn_batch_setup: element node id out of range (instance " + std::to_string(i) +
                                      ")");
          return SGN_EINVAL;
        }
        conn.push_back((int32_t)(v + off));
      }
      fixed.insert(fixed.end(), m.fixed_h, m.fixed_h + m.n_nodes);
      if (objectives) {
        const sgn_objective &o = objectives[i];
        for (int t = 0; t < o.n_track; ++t) {
          const int64_t g = o.track_dof_h[t];
          if (g < 0 || g >= (int64_t)m.n_nodes * d) {
            sgn::set_error(nullptr, "sgn_batch_setup: tracked DOF out of range (instance " + std::to_string(i) + ")");
            return SGN_EINVAL;
          }
          track.push_back(g + off * d);
          target.push_back(o.target_h[t]);
          weight.push_back(o.weight_h[t]);
        }
      }
      node_off.push_back(off + m.n_nodes);
      elem_off.push_back(elem_off.back() + m.n_elem);
    }
  } catch (const std::bad_alloc &) {
    return SGN_ENOMEM;
  }
  sgn_mesh joined{d, (int32_t)nn, (int32_t)ne, X.data(), conn.data(), fixed.data(), meshes[0].E0, meshes[0].nu};
  sgn_t h = nullptr;
  sgn_status s = sgn_setup(&joined, opts, &h);
  if (s != SGN_OK) return s;
  h->n_inst = n;
  h->inst_node_off = std::move(node_off);
  h->inst_elem_off = std::move(elem_off);
  // instance of every free rank and every element (for per-instance norms)
  h->h_rank_inst.assign(h->S.n_free, 0);
  h->h_elem_inst.assign(h->S.n_elem, 0);
  for (int i = 0; i < n; ++i) {
    for (int64_t v = h->inst_node_off[i]; v < h->inst_node_off[i + 1]; ++v) {
      const int r = h->S.node_rank[v];
      if (r >= 0) h->h_rank_inst[r] = i;
    }
    for (int64_t e = h->inst_elem_off[i]; e < h->inst_elem_off[i + 1]; ++e) h->h_elem_inst[e] = i;
  }
  if (objectives) {
    h->pending_obj = true;
    h->pobj_track = std::move(track);
    h->pobj_target = std::move(target);
    h->pobj_weight = std::move(weight);
    h->pobj_alpha = objectives[0].alpha;
  }
  *out = h;
  return SGN_OK;
}

sgn_status sgn_batch_info(sgn_t h, int32_t *n, int64_t *node_off_h, int64_t *elem_off_h) {
  if (!h || !n) return SGN_EINVAL;
  *n = h->n_inst;
  if (h->n_inst <= 0) return SGN_OK;
  for (int i = 0; i <= h->n_inst; ++i) {
    if (node_off_h) node_off_h[i] = h->inst_node_off[i];
    if (elem_off_h) elem_off_h[i] = h->inst_elem_off[i];
  }
  return SGN_OK;
}

sgn_status sgn_batch_residuals(sgn_t h, int32_t kind, double *res_h) {
  if (!h || !res_h || (kind != SGN_BATCH_EQUILIBRIUM && kind != SGN_BATCH_KKT)) return SGN_EINVAL;
  if (h->n_inst <= 0 || !h->bound) return SGN_ESTATE;
  if ((kind == SGN_BATCH_EQUILIBRIUM && !h->inst_have_eq) || (kind == SGN_BATCH_KKT && !h->inst_have_kkt)) {
    sgn::set_error(h, "sgn_batch_residuals: no equilibrium / solve recorded yet");
    return SGN_ESTATE;
  }
  const int n = h->n_inst;
  std::vector<double> a(2 * (size_t)n);
  const double *src = h->inst_acc + (kind == SGN_BATCH_KKT ? 2 * n : 0);
  cudaError_t e = cudaMemcpyAsync(a.data(), src, a.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    sgn::set_error(h, std::string("sgn_batch_residuals: ") + cudaGetErrorString(e));
    return SGN_ECUDA;
  }
  for (int i = 0; i < n; ++i) res_h[i] = a[n + i] > 0 ? std::sqrt(a[i] / a[n + i]) : std::sqrt(a[i]);
  return SGN_OK;
}

}  // extern "C"
