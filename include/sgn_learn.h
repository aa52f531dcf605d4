/*
 * sgn_learn.h -- learned warm start of the equilibrium solve (libsgn.so).
 *
 * The paper recomputes the equilibrium x(p) by Newton's method after every
 * parameter update (Sec. 5, "Computing Equilibrium States").  This module
 * predicts the starting point of that Newton solve from the design:
 *
 *   design      theta in R^n_rbf,  p_e = sum_k theta_k exp(-|X_e - c_k|^2 / (2 w^2))
 *               (X_e the element centroid, c_k the RBF centres, w the width)
 *   basis       u_bar + U c: mean and leading left singular vectors of the
 *               centred matrix of equilibrium displacement snapshots (randomised
 *               SVD: GPU GEMMs, a Cholesky-QR and a small symmetric eigensolve)
 *   network     c(theta) = MLP(theta): n_rbf -> hidden -> hidden -> n_modes,
 *               exact GELU after the hidden layers, BF16 operands with FP32
 *               accumulation, FP32 master weights trained by AdamW on the GPU
 *   warm start  x0 = X + u_bar + U c(theta); Newton starts from x0 unless the
 *               previous iterate has the smaller equilibrium residual.
 *
 * Conventions as in sgn.h: *_h host, *_d device (borrowed) pointers; calls
 * are stream-ordered on the parent handle's stream; the caller provides the
 * module's device buffer (sgn_learn_device_bytes / sgn_learn_bind).
 * Snapshot and basis vectors are node-major [n_nodes][dim] displacements
 * (u = x - X; zero at fixed nodes); the basis is column-major
 * [n_modes][n_nodes*dim].
 */
#ifndef SGN_LEARN_H
#define SGN_LEARN_H

#include "sgn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgn_learn_ctx *sgn_learn_t;

typedef struct {
  int32_t n_rbf;             /* design size (64) */
  const double *centers_h;   /* [n_rbf][dim] RBF centres */
  double width;              /* RBF width (0.15) */
  int32_t n_modes;           /* basis size (128) */
  int32_t hidden;            /* hidden width (512) */
  int32_t max_snap;          /* largest snapshot count passed to basis / train */
  int32_t batch;             /* training mini-batch (<= max_snap) */
} sgn_learn_opts;

/* Host-only creation on a bound sgn_t (kept by reference, must outlive L). */
sgn_status sgn_learn_create(sgn_t h, const sgn_learn_opts *opts, sgn_learn_t *out);
sgn_status sgn_learn_device_bytes(sgn_learn_t L, size_t *bytes);
/* Carves dev_buf (256-byte aligned) and builds the RBF matrix on the device. */
sgn_status sgn_learn_bind(sgn_learn_t L, void *dev_buf, size_t bytes);
void sgn_learn_destroy(sgn_learn_t L);

/* p_d[n_elem] = Phi theta_d[n_rbf] (the RBF design map). */
sgn_status sgn_rbf_params(sgn_learn_t L, const double *theta_d, double *p_d);

/* Displacement basis from snaps_d ([n_snap][n_nodes*dim], one snapshot per
 * row): mean, the n_modes leading left singular vectors of the centred
 * snapshots (randomised SVD with 32 oversampling columns and one power
 * iteration; seed drives its Gaussian test matrix) and sigma_h[n_modes]
 * (may be NULL).  Synchronises. */
sgn_status sgn_learn_basis(sgn_learn_t L, const double *snaps_d, int32_t n_snap, uint64_t seed, double *sigma_h);

/* Trains the MLP on (theta, snapshot) pairs: targets are the basis
 * coefficients of the centred snapshots, normalised per mode; inputs are
 * theta scaled by their RMS.  steps AdamW steps (b1 0.9, b2 0.999, eps 1e-8)
 * on mini-batches drawn (seeded) without replacement per epoch.
 * final_loss_h (may be NULL): mean normalised squared error of the last
 * mini-batch.  Synchronises. */
sgn_status sgn_learn_train(sgn_learn_t L, const double *thetas_d, const double *snaps_d, int32_t n_snap,
                           int32_t steps, float lr, float weight_decay, uint64_t seed, float *final_loss_h);

/* x0_d[n_nodes][dim] = X + u_bar + U c(theta_d). */
sgn_status sgn_learn_predict(sgn_learn_t L, const double *theta_d, double *x0_d);

/* Equilibrium at p = Phi theta (sgn_equilibrium) started from the learned
 * warm start or, when its residual ||c|| is larger, from x_prev_d (may be
 * NULL: the rest shape).  *used_warm_start (may be NULL) tells which.  x_d
 * receives the equilibrium.  Synchronises. */
sgn_status sgn_equilibrium_warm(sgn_learn_t L, const double *theta_d, const double *fext_d, const double *x_prev_d,
                                double *x_d, const sgn_newton_opts *opts, sgn_newton_report *report,
                                int32_t *used_warm_start);

/* ---- inspection and tests ------------------------------------------------ */
int64_t sgn_learn_param_count(sgn_learn_t L);
/* Copies the FP32 master parameters out (set = 0) or in (set = 1); layout
 * W1 [hidden][n_rbf], b1, W2 [hidden][hidden], b2, W3 [n_modes][hidden], b3. */
sgn_status sgn_learn_params(sgn_learn_t L, float *params_h, int32_t set);
/* Forward + backward of L = 1/(2n) sum ||MLP(x) - t||^2 on a host batch
 * x_h [n][n_rbf], t_h [n][n_modes] (n <= batch): loss and parameter
 * gradients (layout as sgn_learn_params), BF16 compute. */
sgn_status sgn_learn_grads(sgn_learn_t L, const float *x_h, const float *t_h, int32_t n, float *loss_h,
                           float *grads_h);
/* One AdamW step (b1 0.9, b2 0.999, eps 1e-8, decoupled weight decay) with
 * the given host gradients (layout as sgn_learn_params) on the master
 * parameters; the step count continues from the last step.  Synchronises. */
sgn_status sgn_learn_apply(sgn_learn_t L, const float *grads_h, float lr, float weight_decay);
/* mean_h [n_nodes*dim] and basis_h [n_modes][n_nodes*dim] (either may be NULL). */
sgn_status sgn_learn_basis_get(sgn_learn_t L, double *mean_h, double *basis_h);

#ifdef __cplusplus
}
#endif
#endif /* SGN_LEARN_H */
