// Element evaluation, no-atomic assembly into the fixed pattern, right-hand
// sides, p elimination and FP64 residuals of the saddle-point system.
//
// Element model (the paper names linear simplices with a neo-Hookean material,
// Sec. 5 "Inverse Elastic Design"): Psi(F) = mu/2 (tr F^T F - d) - mu ln J +
// lambda/2 (ln J)^2 with E_e = E0 exp(p_e).  With F = sum_a x_a B_a^T and
// g_a = F^{-T} B_a the element blocks are, per node pair (a, b):
//   force      c_a     = vol (mu F B_a + (lambda ln J - mu) g_a)
//   Hessian    K_ab    = vol (mu (B_a.B_b) I + lambda g_a g_b^T + (mu - lambda ln J) g_b g_a^T)
//   dc/dp_e    column  = the element force (Psi is linear in E = E0 e^p),
// so each element only needs (vol mu, vol lambda, vol (mu - lambda ln J), g_a)
// and its force vector; the slot kernel rebuilds each K_ab from those.
#include <cmath>

#include "common.cuh"

namespace sgn {

namespace {

constexpr int TPB = 256;

inline int nblk(int64_t n, int t = TPB) { return (int)((n + t - 1) / t); }

template <int D>
__device__ __forceinline__ double det_inv(const double F[D][D], double Fi[D][D]) {
  if constexpr (D == 2) {
    double det = F[0][0] * F[1][1] - F[0][1] * F[1][0];
    double r = 1.0 / det;
    Fi[0][0] = F[1][1] * r; Fi[0][1] = -F[0][1] * r;
    Fi[1][0] = -F[1][0] * r; Fi[1][1] = F[0][0] * r;
    return det;
  } else {
    double c00 = F[1][1] * F[2][2] - F[1][2] * F[2][1];
    double c01 = F[1][2] * F[2][0] - F[1][0] * F[2][2];
    double c02 = F[1][0] * F[2][1] - F[1][1] * F[2][0];
    double det = F[0][0] * c00 + F[0][1] * c01 + F[0][2] * c02;
    double r = 1.0 / det;
    Fi[0][0] = c00 * r;
    Fi[1][0] = c01 * r;
    Fi[2][0] = c02 * r;
    Fi[0][1] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) * r;
    Fi[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) * r;
    Fi[2][1] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) * r;
    Fi[0][2] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) * r;
    Fi[1][2] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) * r;
    Fi[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) * r;
    return det;
  }
}

// F = I + sum_a u_a B_a^T with u_a = v_a - xs X_a: v holds positions (xs = 1)
// or displacements (xs = 0).  Summing displacements instead of positions
// (F = sum_a x_a B_a^T) keeps the round-off of F at eps |u| |B| rather than
// eps |x| |B|, independent of where the body sits.
template <int D>
__device__ __forceinline__ void load_F(int e, int ne, const int32_t *__restrict__ elem_node,
                                       const double *__restrict__ elem_B, const double *__restrict__ v,
                                       const double *__restrict__ X, double xs, double B[D + 1][D],
                                       double F[D][D]) {
  double ua[D + 1][D];
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    int n = __ldg(elem_node + (int64_t)a * ne + e);
#pragma unroll
    for (int i = 0; i < D; ++i) ua[a][i] = fma(-xs, __ldg(X + (int64_t)n * D + i), __ldg(v + (int64_t)n * D + i));
#pragma unroll
    for (int j = 0; j < D; ++j) B[a][j] = __ldg(elem_B + (int64_t)(a * D + j) * ne + e);
  }
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      double s = i == j ? 1.0 : 0.0;
#pragma unroll
      for (int a = 0; a <= D; ++a) s = fma(ua[a][i], B[a][j], s);
      F[i][j] = s;
    }
}

// one thread per element: element state + force (= column of dc/dp)
template <int D>
__global__ void __launch_bounds__(TPB) k_elem_state(int ne, const int32_t *__restrict__ elem_node,
                                                    const double *__restrict__ elem_B,
                                                    const double *__restrict__ elem_vol,
                                                    const double *__restrict__ x, const double *__restrict__ X,
                                                    double xs, const double *__restrict__ p,
                                                    double E0, double nu, double *__restrict__ st,
                                                    double *__restrict__ cpv, int *status) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double B[D + 1][D], F[D][D], Fi[D][D];
  load_F<D>(e, ne, elem_node, elem_B, x, X, xs, B, F);
  double J = det_inv<D>(F, Fi);
  if (!(J > 0.0)) {
    atomicOr(status, DEV_INVERTED);
    J = 1.0;
  }
  double lnJ = log(J);
  double E = E0 * exp(__ldg(p + e));
  double mu = E / (2.0 * (1.0 + nu));
  double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double vol = __ldg(elem_vol + e);
  st[e] = vol * mu;
  st[(int64_t)ne + e] = vol * lam;
  st[2 * (int64_t)ne + e] = vol * (mu - lam * lnJ);
  double cf = lam * lnJ - mu;
  bool bad = false;
#pragma unroll
  for (int a = 0; a <= D; ++a)
#pragma unroll
    for (int i = 0; i < D; ++i) {
      double g = 0.0, fb = 0.0;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        g = fma(Fi[j][i], B[a][j], g);
        fb = fma(F[i][j], B[a][j], fb);
      }
      double c = vol * (mu * fb + cf * g);
      bad |= !isfinite(c);
      st[(int64_t)(3 + a * D + i) * ne + e] = g;
      cpv[(int64_t)(a * D + i) * ne + e] = c;
    }
  if (bad) atomicOr(status, DEV_NONFINITE);
}

// one thread per upper block slot (r <= c): gathers every element
// contribution of the slot (no atomics), writes the block to (r, c) and its
// transpose to (c, r).  G = dc/dp C^{-1} dc/dp^T (the Schur complement left
// by eliminating p first) has the same block pattern.
template <int D>
__global__ void __launch_bounds__(TPB) k_slot_gather(int n_up, int ne, const int32_t *__restrict__ up_slot,
                                                     const int32_t *__restrict__ up_slot_t,
                                                     const int32_t *__restrict__ up_ptr,
                                                     const int32_t *__restrict__ up_contrib,
                                                     const double *__restrict__ elem_B,
                                                     const double *__restrict__ st,
                                                     const double *__restrict__ cpv, double inv_alpha,
                                                     double *__restrict__ Kv, double *__restrict__ Gv) {
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n_up) return;
  double Kb[D][D], Gb[D][D];
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int k = 0; k < D; ++k) { Kb[i][k] = 0.0; Gb[i][k] = 0.0; }
  int t0 = __ldg(up_ptr + u), t1 = __ldg(up_ptr + u + 1);
  for (int t = t0; t < t1; ++t) {
    int pk = __ldg(up_contrib + t);
    int e = pk >> 4, a = (pk >> 2) & 3, b = pk & 3;
    double s1 = __ldg(st + e), s2 = __ldg(st + (int64_t)ne + e), s3 = __ldg(st + 2 * (int64_t)ne + e);
    double Ba[D], Bb[D], ga[D], gb[D];
    double bab = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      Ba[j] = __ldg(elem_B + (int64_t)(a * D + j) * ne + e);
      Bb[j] = __ldg(elem_B + (int64_t)(b * D + j) * ne + e);
      ga[j] = __ldg(st + (int64_t)(3 + a * D + j) * ne + e);
      gb[j] = __ldg(st + (int64_t)(3 + b * D + j) * ne + e);
      bab = fma(Ba[j], Bb[j], bab);
    }
    double sb = s1 * bab;
#pragma unroll
    for (int i = 0; i < D; ++i) {
#pragma unroll
      for (int k = 0; k < D; ++k) Kb[i][k] = fma(s2, ga[i] * gb[k], fma(s3, gb[i] * ga[k], Kb[i][k]));
      Kb[i][i] += sb;
    }
    if (Gv) {
      double ca[D], cb[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        ca[j] = __ldg(cpv + (int64_t)(a * D + j) * ne + e);
        cb[j] = __ldg(cpv + (int64_t)(b * D + j) * ne + e) * inv_alpha;
      }
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int k = 0; k < D; ++k) Gb[i][k] = fma(ca[i], cb[k], Gb[i][k]);
    }
  }
  int s = __ldg(up_slot + u), sT = __ldg(up_slot_t + u);
#pragma unroll
  for (int i = 0; i < D; ++i)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      Kv[(int64_t)s * D * D + i * D + k] = Kb[i][k];
      if (sT != s) Kv[(int64_t)sT * D * D + k * D + i] = Kb[i][k];
      if (Gv) {
        Gv[(int64_t)s * D * D + i * D + k] = Gb[i][k];
        if (sT != s) Gv[(int64_t)sT * D * D + k * D + i] = Gb[i][k];
      }
    }
}

// df/dx = w (x - target) on tracked DOFs, df/dp = alpha p; keeps x (rank-DOF)
template <int D>
__global__ void k_objective(int n_free, const int32_t *__restrict__ rank_node, const double *__restrict__ x,
                            const double *__restrict__ wA, const double *__restrict__ tgt,
                            double *__restrict__ fx, double *__restrict__ xr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_free * D) return;
  int r = i / D, a = i - r * D;
  double xv = x[(int64_t)rank_node[r] * D + a];
  xr[i] = xv;
  fx[i] = wA[i] * (xv - tgt[i]);
}

__global__ void k_scale(int64_t n, const double *__restrict__ p, double a, double *__restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * p[i];
}

// reduced right-hand side of the (x, lambda) system after eliminating p:
//   [b_x ; b_l - dc/dp C^{-1} b_p], interleaved per DOF (x, lambda)
template <int D>
__global__ void k_reduce_rhs(int n_free, int ne, const int32_t *__restrict__ inc_ptr,
                             const int32_t *__restrict__ inc, const double *__restrict__ cpv,
                             const double *__restrict__ bx, const double *__restrict__ bp,
                             const double *__restrict__ bl, double inv_alpha, double *__restrict__ red) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_free) return;
  double acc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) acc[a] = bl ? bl[(int64_t)r * D + a] : 0.0;
  if (bp) {
    for (int t = inc_ptr[r]; t < inc_ptr[r + 1]; ++t) {
      int pk = inc[t];
      int e = pk >> 2, loc = pk & 3;
      double s = bp[e] * inv_alpha;
#pragma unroll
      for (int a = 0; a < D; ++a) acc[a] -= cpv[(int64_t)(loc * D + a) * ne + e] * s;
    }
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    red[(int64_t)r * 2 * D + 2 * a] = bx ? bx[(int64_t)r * D + a] : 0.0;
    red[(int64_t)r * 2 * D + 2 * a + 1] = acc[a];
  }
}

template <int D>
__global__ void k_recover_xl(int n_free, const double *__restrict__ red, double *__restrict__ zx,
                             double *__restrict__ zl) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_free * D) return;
  zx[i] = red[2 * (int64_t)i];
  zl[i] = red[2 * (int64_t)i + 1];
}

// dp = C^{-1} (b_p - dc/dp^T dl) per element; also the gradient form
// g = f_p + dc/dp^T lam when scale = 1, sign = +1
template <int D>
__global__ void k_elem_dot(int ne, const int32_t *__restrict__ elem_rank, const double *__restrict__ cpv,
                           const double *__restrict__ v, const double *__restrict__ base, double sign,
                           double scale, double *__restrict__ out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double s = 0.0;
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    int r = elem_rank[(int64_t)a * ne + e];
    if (r < 0) continue;
#pragma unroll
    for (int i = 0; i < D; ++i) s = fma(cpv[(int64_t)(a * D + i) * ne + e], v[(int64_t)r * D + i], s);
  }
  out[e] = scale * ((base ? base[e] : 0.0) + sign * s);
}

// FP64 residual rows of x and lambda: r_x = b_x - A z_x - K z_l,
// r_l = b_l - K z_x - dc/dp z_p   (one thread per free node)
template <int D>
__global__ void k_residual_nodes(int n_free, int ne, const int32_t *__restrict__ bsr_ptr,
                                 const int32_t *__restrict__ bsr_col, const double *__restrict__ Kv,
                                 const int32_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc,
                                 const double *__restrict__ cpv, const double *__restrict__ wA,
                                 const double *__restrict__ bx, const double *__restrict__ bl,
                                 const double *__restrict__ zx, const double *__restrict__ zp,
                                 const double *__restrict__ zl, double *__restrict__ rx,
                                 double *__restrict__ rl, double eps_x, double eps_l) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_free) return;
  double ax[D], al[D];
  // the x and lambda diagonals carry eps_x and -eps_l when the regularized
  // matrix of an inertia-corrected factorization is solved (else both 0)
#pragma unroll
  for (int a = 0; a < D; ++a) {
    ax[a] = bx[(int64_t)r * D + a] - (wA[(int64_t)r * D + a] + eps_x) * zx[(int64_t)r * D + a];
    al[a] = fma(eps_l, zl[(int64_t)r * D + a], bl[(int64_t)r * D + a]);
  }
  for (int k = bsr_ptr[r]; k < bsr_ptr[r + 1]; ++k) {
    int c = bsr_col[k];
    const double *Kb = Kv + (int64_t)k * D * D;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int b = 0; b < D; ++b) {
        double kv = Kb[a * D + b];
        ax[a] = fma(-kv, zl[(int64_t)c * D + b], ax[a]);
        al[a] = fma(-kv, zx[(int64_t)c * D + b], al[a]);
      }
  }
  for (int t = inc_ptr[r]; t < inc_ptr[r + 1]; ++t) {
    int pk = inc[t];
    int e = pk >> 2, loc = pk & 3;
    double zpe = zp[e];
#pragma unroll
    for (int a = 0; a < D; ++a) al[a] = fma(-cpv[(int64_t)(loc * D + a) * ne + e], zpe, al[a]);
  }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    rx[(int64_t)r * D + a] = ax[a];
    rl[(int64_t)r * D + a] = al[a];
  }
}

// r = b - K z (one thread per free node)
template <int D>
__global__ void k_residual_k(int n_free, const int32_t *__restrict__ bsr_ptr, const int32_t *__restrict__ bsr_col,
                             const double *__restrict__ Kv, const double *__restrict__ b,
                             const double *__restrict__ z, double *__restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_free) return;
  double acc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) acc[a] = b[(int64_t)i * D + a];
  for (int k = bsr_ptr[i]; k < bsr_ptr[i + 1]; ++k) {
    const int c = bsr_col[k];
    const double *Kb = Kv + (int64_t)k * D * D;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
      for (int bb = 0; bb < D; ++bb) acc[a] = fma(-Kb[a * D + bb], z[(int64_t)c * D + bb], acc[a]);
  }
#pragma unroll
  for (int a = 0; a < D; ++a) r[(int64_t)i * D + a] = acc[a];
}

template <int D>
__global__ void k_residual_p(int ne, const int32_t *__restrict__ elem_rank, const double *__restrict__ cpv,
                             double alpha, const double *__restrict__ bp, const double *__restrict__ zp,
                             const double *__restrict__ zl, double *__restrict__ rp) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double s = bp[e] - alpha * zp[e];
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    int r = elem_rank[(int64_t)a * ne + e];
    if (r < 0) continue;
#pragma unroll
    for (int i = 0; i < D; ++i) s = fma(-cpv[(int64_t)(a * D + i) * ne + e], zl[(int64_t)r * D + i], s);
  }
  rp[e] = s;
}

__global__ void k_sumsq3(const double *__restrict__ a, int64_t na, const double *__restrict__ b, int64_t nb,
                         const double *__restrict__ c, int64_t nc, double *__restrict__ partial) {
  __shared__ double sh[TPB];
  double s = 0.0;
  int64_t n = na + nb + nc;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = i < na ? a[i] : (i < na + nb ? b[i - na] : c[i - na - nb]);
    s = fma(v, v, s);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_dot(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                      double *__restrict__ partial) {
  __shared__ double sh[TPB];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s = fma(a[i], b[i], s);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_axpy(double *__restrict__ y, const double *__restrict__ x, double a, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(a, x[i], y[i]);
}

template <int D>
__global__ void k_to_nodes(int n_nodes, const int32_t *__restrict__ node_rank, const double *__restrict__ vr,
                           double *__restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes * D) return;
  int n = i / D, a = i - n * D;
  int r = node_rank[n];
  out[i] = r >= 0 ? vr[(int64_t)r * D + a] : 0.0;
}

template <int D>
__global__ void k_from_nodes(int n_free, const int32_t *__restrict__ rank_node, const double *__restrict__ nodes,
                             double *__restrict__ vr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_free * D) return;
  int r = i / D, a = i - r * D;
  vr[i] = nodes[(int64_t)rank_node[r] * D + a];
}

template <int D>
__global__ void k_internal_force(int n_free, int ne, const int32_t *__restrict__ inc_ptr,
                                 const int32_t *__restrict__ inc, const double *__restrict__ cpv,
                                 double *__restrict__ fr) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_free) return;
  double acc[D];
#pragma unroll
  for (int a = 0; a < D; ++a) acc[a] = 0.0;
  for (int t = inc_ptr[r]; t < inc_ptr[r + 1]; ++t) {
    int pk = inc[t];
    int e = pk >> 2, loc = pk & 3;
#pragma unroll
    for (int a = 0; a < D; ++a) acc[a] += cpv[(int64_t)(loc * D + a) * ne + e];
  }
#pragma unroll
  for (int a = 0; a < D; ++a) fr[(int64_t)r * D + a] = acc[a];
}

// per-block partial sums of vol Psi; +inf if any element of the block is inverted
template <int D>
__global__ void __launch_bounds__(TPB) k_energy(int ne, const int32_t *__restrict__ elem_node,
                                                const double *__restrict__ elem_B,
                                                const double *__restrict__ elem_vol,
                                                const double *__restrict__ x, const double *__restrict__ X, double xs,
                                                const double *__restrict__ p, double E0, double nu,
                                                double *__restrict__ partial) {
  __shared__ double sh[TPB];
  double s = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
    double B[D + 1][D], F[D][D], Fi[D][D];
    load_F<D>(e, ne, elem_node, elem_B, x, X, xs, B, F);
    double J = det_inv<D>(F, Fi);
    if (!(J > 0.0)) { s = INFINITY; continue; }
    double lnJ = log(J);
    double E = E0 * exp(p[e]);
    double mu = E / (2.0 * (1.0 + nu));
    double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    double I1 = 0.0;
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
      for (int j = 0; j < D; ++j) I1 = fma(F[i][j], F[i][j], I1);
    s += elem_vol[e] * (0.5 * mu * (I1 - D) - mu * lnJ + 0.5 * lam * lnJ * lnJ);
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = TPB / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// out = v + s X over all node coordinates (s = -1: displacements of
// positions v; s = +1: positions of displacements v)
__global__ void k_shift_rest(int64_t n, const double *__restrict__ v, const double *__restrict__ X, double s,
                             double *__restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = fma(s, X[i], v[i]);
}

template <int D>
__global__ void k_positions(int n_free, const int32_t *__restrict__ rank_node, const double *__restrict__ x0,
                            const double *__restrict__ dxr, double t, double *__restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_free * D) return;
  int r = i / D, a = i - r * D;
  int64_t g = (int64_t)rank_node[r] * D + a;
  x[g] = x0[g] + t * dxr[i];
}

}  // namespace

#define SGN_DISPATCH_D(c, KERNEL, GRID, BLOCK, SMEM, ...)                          \
  do {                                                                            \
    if ((c).S.dim == 2) KERNEL<2><<<GRID, BLOCK, SMEM, (c).stream>>>(__VA_ARGS__); \
    else KERNEL<3><<<GRID, BLOCK, SMEM, (c).stream>>>(__VA_ARGS__);               \
    (c).count();                                                                  \
  } while (0)

void launch_elem_state(Ctx &c, const double *x, const double *p) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_elem_state, nblk(d.n_elem), TPB, 0, d.n_elem, d.elem_node, d.elem_B, d.elem_vol, x, d.X,
                 1.0, p, c.E0, c.nu, c.st, c.cpv, c.status);
}

void launch_elem_state_disp(Ctx &c, const double *u, const double *p) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_elem_state, nblk(d.n_elem), TPB, 0, d.n_elem, d.elem_node, d.elem_B, d.elem_vol, u, d.X,
                 0.0, p, c.E0, c.nu, c.st, c.cpv, c.status);
}

// same two kernels with the element state in caller-chosen scratch memory
void launch_elem_state_into(Ctx &c, const double *x, const double *p, double *st) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_elem_state, nblk(d.n_elem), TPB, 0, d.n_elem, d.elem_node, d.elem_B, d.elem_vol, x, d.X,
                 1.0, p, c.E0, c.nu, st, c.cpv, c.status);
}

void launch_slot_gather_from(Ctx &c, const double *st) {
  const DevSym &d = c.ds;
  int n_up = (int)c.S.up_slot.size();
  SGN_DISPATCH_D(c, k_slot_gather, nblk(n_up), TPB, 0, n_up, d.n_elem, d.up_slot, d.up_slot_t, d.up_ptr,
                 d.up_contrib, d.elem_B, st, c.cpv, 1.0 / c.alpha, c.Kv, c.Gv);
}

void launch_slot_gather(Ctx &c, bool with_G) {
  const DevSym &d = c.ds;
  int n_up = (int)c.S.up_slot.size();
  SGN_DISPATCH_D(c, k_slot_gather, nblk(n_up), TPB, 0, n_up, d.n_elem, d.up_slot, d.up_slot_t, d.up_ptr,
                 d.up_contrib, d.elem_B, c.st, c.cpv, with_G ? 1.0 / c.alpha : 0.0, c.Kv,
                 with_G ? c.Gv : nullptr);
}

void launch_objective_terms(Ctx &c, const double *x, const double *p) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_objective, nblk((int64_t)d.n_free * d.dim), TPB, 0, d.n_free, d.rank_node, x, c.wA,
                 c.tgt, c.fx, c.xr);
  k_scale<<<nblk(d.n_elem), TPB, 0, c.stream>>>(d.n_elem, p, c.alpha, c.fp);
  c.count();
}

void launch_reduce_rhs(Ctx &c, const double *bx, const double *bp, const double *bl, double *red, int) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_reduce_rhs, nblk(d.n_free), TPB, 0, d.n_free, d.n_elem, d.inc_ptr, d.inc, c.cpv, bx, bp, bl,
                 1.0 / c.alpha, red);
}

void launch_recover(Ctx &c, const double *red, const double *bp, double *zx, double *zp, double *zl) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_recover_xl, nblk((int64_t)d.n_free * d.dim), TPB, 0, d.n_free, red, zx, zl);
  SGN_DISPATCH_D(c, k_elem_dot, nblk(d.n_elem), TPB, 0, d.n_elem, d.elem_rank, c.cpv, zl, bp, -1.0,
                 1.0 / c.alpha, zp);
}

void launch_residual(Ctx &c, const double *bx, const double *bp, const double *bl, const double *zx,
                     const double *zp, const double *zl, double *rx, double *rp, double *rl) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_residual_nodes, nblk(d.n_free), TPB, 0, d.n_free, d.n_elem, d.bsr_ptr, d.bsr_col, c.Kv,
                 d.inc_ptr, d.inc, c.cpv, c.wA, bx, bl, zx, zp, zl, rx, rl, c.res_eps_x, c.res_eps_l);
  SGN_DISPATCH_D(c, k_residual_p, nblk(d.n_elem), TPB, 0, d.n_elem, d.elem_rank, c.cpv, c.alpha, bp, zp, zl, rp);
}

void launch_residual_k(Ctx &c, const double *b, const double *z, double *r) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_residual_k, nblk(d.n_free), TPB, 0, d.n_free, d.bsr_ptr, d.bsr_col, c.Kv, b, z, r);
}

double device_sumsq3(Ctx &c, const double *a, int64_t na, const double *b, int64_t nb, const double *c2,
                     int64_t nc) {
  int blocks = c.n_partial;
  k_sumsq3<<<blocks, TPB, 0, c.stream>>>(a, na, b, nb, c2, nc, c.partial);
  c.count();
  std::vector<double> h(blocks);
  cudaMemcpyAsync(h.data(), c.partial, sizeof(double) * blocks, cudaMemcpyDeviceToHost, c.stream);
  cudaStreamSynchronize(c.stream);
  double s = 0.0;
  for (double v : h) s += v;
  return s;
}

void launch_sumsq3(Ctx &c, const double *a, int64_t na, const double *b, int64_t nb, const double *c2, int64_t nc,
                   double *partial_out) {
  k_sumsq3<<<c.n_partial, TPB, 0, c.stream>>>(a, na, b, nb, c2, nc, partial_out);
  c.count();
}

double device_dot(Ctx &c, const double *a, const double *b, int64_t n) {
  int blocks = c.n_partial;
  k_dot<<<blocks, TPB, 0, c.stream>>>(a, b, n, c.partial);
  c.count();
  std::vector<double> h(blocks);
  cudaMemcpyAsync(h.data(), c.partial, sizeof(double) * blocks, cudaMemcpyDeviceToHost, c.stream);
  cudaStreamSynchronize(c.stream);
  double s = 0.0;
  for (double v : h) s += v;
  return s;
}

void launch_axpy(Ctx &c, double *y, const double *x, double a, int64_t n) {
  k_axpy<<<nblk(n), TPB, 0, c.stream>>>(y, x, a, n);
  c.count();
}

void launch_to_nodes_plain(Ctx &c, const double *vr, double *out) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_to_nodes, nblk((int64_t)d.n_nodes * d.dim), TPB, 0, d.n_nodes, d.node_rank, vr, out);
}

void launch_to_nodes(Ctx &c, const double *vr, double *out, double) { launch_to_nodes_plain(c, vr, out); }

void launch_from_nodes(Ctx &c, const double *nodes, double *vr) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_from_nodes, nblk((int64_t)d.n_free * d.dim), TPB, 0, d.n_free, d.rank_node, nodes, vr);
}

void launch_internal_force(Ctx &c, double *fr) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_internal_force, nblk(d.n_free), TPB, 0, d.n_free, d.n_elem, d.inc_ptr, d.inc, c.cpv, fr);
}

int energy_blocks(Ctx &c) { return c.n_partial; }

void launch_energy_partials(Ctx &c, const double *x, const double *p, double *partials, int nblocks, bool disp) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_energy, nblocks, TPB, 0, d.n_elem, d.elem_node, d.elem_B, d.elem_vol, x, d.X,
                 disp ? 0.0 : 1.0, p, c.E0, c.nu, partials);
}

void launch_positions_update(Ctx &c, const double *x0, const double *dxr, double t, double *x) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_positions, nblk((int64_t)d.n_free * d.dim), TPB, 0, d.n_free, d.rank_node, x0, dxr, t, x);
}

void launch_shift_rest(Ctx &c, const double *v, double s, double *out) {
  const int64_t n = (int64_t)c.ds.n_nodes * c.ds.dim;
  k_shift_rest<<<nblk(n), TPB, 0, c.stream>>>(n, v, c.ds.X, s, out);
  c.count();
}

void launch_gradient_finish(Ctx &c, const double *lam_r, double *g) {
  const DevSym &d = c.ds;
  SGN_DISPATCH_D(c, k_elem_dot, nblk(d.n_elem), TPB, 0, d.n_elem, d.elem_rank, c.cpv, lam_r, c.fp, 1.0, 1.0, g);
}

}  // namespace sgn
