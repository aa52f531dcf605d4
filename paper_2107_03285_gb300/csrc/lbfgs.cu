// L-BFGS initialised with the Sparse Gauss-Newton inverse Hessian (Sec. 4,
// "Combination with L-BFGS"): every search direction is the two-loop
// recursion over the most recent (s, y) pairs with H_0^{-1} applied by one
// solve of Eq. sparseSystemGN (right-hand side [0; -q; 0] gives dp =
// -H_GN^{-1} q), reusing the saddle-point factor of the current iterate.
// The optimisation loop around it (equilibrium, objective, adjoint gradient,
// backtracking line search) runs on the library's own calls; all vector
// arithmetic is done by kernels on the handle's stream.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace sgn {
namespace {

constexpr int TPB = 256;

// per-block partial sums of w (x - t)^2 over the free DOFs (rank-DOF layout,
// positions gathered from the node-major x) and of p^2 over the elements
template <int D>
__global__ void k_objective_partials(int n_free, int ne, const int32_t *__restrict__ rank_node,
                                     const double *__restrict__ x, const double *__restrict__ wA,
                                     const double *__restrict__ tgt, const double *__restrict__ p,
                                     double *__restrict__ partial) {
  __shared__ double sh[2][TPB];
  double a = 0.0, b = 0.0;
  const int64_t n = (int64_t)n_free * D;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n || i < ne;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < n) {
      const int r = (int)(i / D), c = (int)(i - (int64_t)r * D);
      const double w = wA[i];
      if (w != 0.0) {
        const double e = x[(int64_t)rank_node[r] * D + c] - tgt[i];
        a = fma(w * e, e, a);
      }
    }
    if (i < ne) b = fma(p[i], p[i], b);
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sh[0][0];
    partial[2 * blockIdx.x + 1] = sh[1][0];
  }
}

// y = a x + b z
__global__ void k_lincomb(int64_t n, double a, const double *__restrict__ x, double b, const double *__restrict__ z,
                          double *__restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * z[i];
}

void lincomb(Ctx &c, int64_t n, double a, const double *x, double b, const double *z, double *y) {
  k_lincomb<<<(unsigned)((n + TPB - 1) / TPB), TPB, 0, c.stream>>>(n, a, x, b, z, y);
  c.count();
}

}  // namespace

double objective_value(Ctx &c, const double *x, const double *p) {
  const int nb = c.n_partial / 2;
  if (c.S.dim == 2)
    k_objective_partials<2><<<nb, TPB, 0, c.stream>>>(c.S.n_free, c.S.n_elem, c.ds.rank_node, x, c.wA, c.tgt, p,
                                                       c.partial);
  else
    k_objective_partials<3><<<nb, TPB, 0, c.stream>>>(c.S.n_free, c.S.n_elem, c.ds.rank_node, x, c.wA, c.tgt, p,
                                                       c.partial);
  c.count();
  std::vector<double> h(2 * (size_t)nb);
  cudaMemcpyAsync(h.data(), c.partial, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream);
  cudaStreamSynchronize(c.stream);
  double a = 0.0, b = 0.0;
  for (int i = 0; i < nb; ++i) { a += h[2 * i]; b += h[2 * i + 1]; }
  return 0.5 * a + c.f_const + 0.5 * c.alpha * b;
}

// d = -H_k g by the two-loop recursion over the pairs (S[order[i]],
// Y[order[i]]), oldest first, with H_0^{-1} from the current saddle-point
// factor; q, r: n_p scratch
sgn_status lbfgs_two_loop(Ctx &c, int m, const double *S, const double *Y, const int *order, const double *g,
                          double *d, double *q, double *r) {
  const int64_t np = c.S.n_elem;
  cudaMemcpyAsync(q, g, np * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
  std::vector<double> rho(m), alpha(m);
  for (int i = m - 1; i >= 0; --i) {
    const double *s = S + (size_t)order[i] * np, *y = Y + (size_t)order[i] * np;
    rho[i] = 1.0 / device_dot(c, y, s, np);
    alpha[i] = rho[i] * device_dot(c, s, q, np);
    launch_axpy(c, q, y, -alpha[i], np);
  }
  // r = H_GN^{-1} q: the solve of Eq. sparseSystemGN with the paper's
  // right-hand side [0; -q; 0] returns dp = -H_GN^{-1} q
  sgn_solve_report rep;
  sgn_status st = sgn_solve(static_cast<sgn_ctx *>(&c), SGN_RHS_PAPER, q, nullptr, r, nullptr, nullptr, &rep);
  if (st != SGN_OK) return st;
  // r currently holds -H_0^{-1} q
  for (int i = 0; i < m; ++i) {
    const double *s = S + (size_t)order[i] * np, *y = Y + (size_t)order[i] * np;
    const double beta = -rho[i] * device_dot(c, y, r, np);  // rho y.(H_0^{-1} q ...), r negated
    launch_axpy(c, r, s, -(alpha[i] - beta), np);
  }
  // d = -H_k g = r (r is kept negated throughout)
  cudaMemcpyAsync(d, r, np * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
  return SGN_OK;
}

}  // namespace sgn

using namespace sgn;

extern "C" {

sgn_status sgn_objective_value(sgn_t h, const double *x_d, const double *p_d, double *f_h) {
  if (!h || !x_d || !p_d || !f_h) return SGN_EINVAL;
  if (!h->bound || !h->have_objective) return SGN_ESTATE;
  *f_h = objective_value(*h, x_d, p_d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_error(h, std::string("sgn_objective_value: ") + cudaGetErrorString(e)); return SGN_ECUDA; }
  return SGN_OK;
}

sgn_status sgn_lbfgs_direction(sgn_t h, int32_t m, const double *s_d, const double *y_d, const double *g_d,
                               double *d_d) {
  if (!h || m < 0 || (m > 0 && (!s_d || !y_d)) || !g_d || !d_d) return SGN_EINVAL;
  if (!h->bound) return SGN_ESTATE;
  if (!h->active || !h->active->factored) {
    set_error(h, "sgn_lbfgs_direction: the saddle-point matrix of the current iterate is not factored");
    return SGN_ESTATE;
  }
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  return lbfgs_two_loop(*h, m, s_d, y_d, order.data(), g_d, d_d, h->lbq, h->lbr);
}

sgn_status sgn_lbfgs_work_bytes(sgn_t h, int32_t m, size_t *bytes) {
  if (!h || !bytes || m < 0) return SGN_EINVAL;
  // m + 1 (s, y) slots (the newest candidate always has a free one), g, g
  // at the trial point, d, the trial p, scratch, and the trial positions
  *bytes = ((size_t)(2 * (m + 1) + 5) * h->S.n_elem + (size_t)h->S.n_nodes * h->S.dim) * sizeof(double);
  return SGN_OK;
}

sgn_status sgn_optimize_lbfgs(sgn_t h, const double *fext_d, double *p_d, double *x_d, void *work_d,
                              size_t work_bytes, const sgn_lbfgs_opts *opts, sgn_lbfgs_report *rep) {
  if (!h || !fext_d || !p_d || !x_d || !work_d || !opts || opts->m < 0 || opts->max_iter < 0) return SGN_EINVAL;
  if (!h->bound || !h->have_objective) return SGN_ESTATE;
  Ctx &c = *h;
  Store &sst = opts->precision == SGN_MIXED ? c.kkt32 : c.kkt64;
  if (!sst.enabled || !c.kf.enabled) {
    set_error(h, "sgn_optimize_lbfgs: needs the saddle-point store of its precision and SGN_STORE_KFACT");
    return SGN_ESTATE;
  }
  size_t need = 0;
  sgn_lbfgs_work_bytes(h, opts->m, &need);
  if (work_bytes < need || ((uintptr_t)work_d & 7)) return SGN_EINVAL;
  auto t_start = std::chrono::steady_clock::now();
  const int m = opts->m;
  const int64_t np = c.S.n_elem, nn = (int64_t)c.S.n_nodes * c.S.dim;
  double *Sbuf = static_cast<double *>(work_d), *Ybuf = Sbuf + (size_t)(m + 1) * np;
  double *g = Ybuf + (size_t)(m + 1) * np, *gt = g + np, *d = gt + np, *pt = d + np, *tmp = pt + np, *xt = tmp + np;
  sgn_newton_opts nopt{};
  nopt.precision = opts->eq_precision;
  sgn_newton_report nrep;
  const double armijo = opts->armijo > 0 ? opts->armijo : 1e-4;
  const int max_ls = opts->max_halvings > 0 ? opts->max_halvings : 30;
  sgn_lbfgs_report R{};
  int eq_iters = 0;
  // f, g at the start: equilibrium (from x_d), objective, adjoint gradient
  sgn_status st = sgn_equilibrium(h, p_d, fext_d, x_d, &nopt, &nrep);
  if (st != SGN_OK) return st;
  eq_iters += nrep.iters;
  double f = objective_value(c, x_d, p_d);
  auto gradient_at = [&](const double *x, const double *p, double *gout) -> sgn_status {
    sgn_status s2 = sgn_assemble(h, x, p);
    if (s2 == SGN_OK) s2 = sgn_factor_k(h);
    if (s2 == SGN_OK) s2 = sgn_gradient(h, gout);
    return s2;
  };
  st = gradient_at(x_d, p_d, g);
  if (st != SGN_OK) return st;
  double gn = std::sqrt(device_dot(c, g, g, np));
  std::vector<int> ring;  // slots of the stored pairs, oldest first
  R.f[0] = f;
  R.gnorm[0] = gn;
  int it = 0;
  for (; it < opts->max_iter; ++it) {
    if (opts->tol_g > 0 && gn <= opts->tol_g) { R.converged = 1; break; }
    // the Gauss-Newton factor of the current iterate (assembled by gradient_at)
    st = sgn_factor(h, (sgn_precision)opts->precision, nullptr);
    if (st != SGN_OK) return st;
    st = lbfgs_two_loop(c, (int)ring.size(), Sbuf, Ybuf, ring.data(), g, d, c.lbq, c.lbr);
    if (st != SGN_OK && st != SGN_EREFINE) return st;
    double slope = device_dot(c, g, d, np);
    if (!(slope < 0.0)) {  // not a descent direction: steepest descent
      lincomb(c, np, -1.0, g, 0.0, g, d);
      slope = -gn * gn;
      R.restarts++;
    }
    // backtracking line search on f(x(p), p), each trial from the last equilibrium
    double t = 1.0, ft = 0.0;
    bool acc = false;
    for (int ls = 0; ls < max_ls; ++ls) {
      lincomb(c, np, 1.0, p_d, t, d, pt);
      cudaMemcpyAsync(xt, x_d, nn * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
      st = sgn_equilibrium(h, pt, fext_d, xt, &nopt, &nrep);
      eq_iters += nrep.iters;
      R.trials++;
      if (st == SGN_OK) {
        ft = objective_value(c, xt, pt);
        if (ft <= f + armijo * t * slope) { acc = true; break; }
      } else if (st != SGN_ENEWTON && st != SGN_EINVERTED) {
        return st;
      }
      t *= 0.5;
    }
    if (!acc) break;  // no decrease along d: stop at the current iterate
    // gradient at the new iterate, then the pair (s, y)
    st = gradient_at(xt, pt, gt);
    if (st != SGN_OK) return st;
    if (m > 0) {
      // the candidate goes to a slot no stored pair uses (there are m + 1)
      int slot = 0;
      while (std::find(ring.begin(), ring.end(), slot) != ring.end()) ++slot;
      double *s = Sbuf + (size_t)slot * np, *y = Ybuf + (size_t)slot * np;
      lincomb(c, np, 1.0, pt, -1.0, p_d, s);
      lincomb(c, np, 1.0, gt, -1.0, g, y);
      const double sy = device_dot(c, s, y, np), ss = device_dot(c, s, s, np), yy = device_dot(c, y, y, np);
      if (sy > 1e-12 * std::sqrt(ss * yy)) {  // curvature condition: keep the pair
        if (ring.size() == (size_t)m) ring.erase(ring.begin());  // drop the oldest
        ring.push_back(slot);
      }
    }
    cudaMemcpyAsync(p_d, pt, np * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
    cudaMemcpyAsync(x_d, xt, nn * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
    cudaMemcpyAsync(g, gt, np * sizeof(double), cudaMemcpyDeviceToDevice, c.stream);
    f = ft;
    gn = std::sqrt(device_dot(c, g, g, np));
    if (it + 1 < 64) {
      R.f[it + 1] = f;
      R.gnorm[it + 1] = gn;
      R.step[it] = t;
    }
  }
  R.iters = it;
  R.equilibrium_iters = eq_iters;
  R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) { set_error(h, std::string("sgn_optimize_lbfgs: ") + cudaGetErrorString(e)); return SGN_ECUDA; }
  if (rep) *rep = R;
  return SGN_OK;
}

}  // extern "C"
