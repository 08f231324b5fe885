/*
 * lbm_mlp.h - learned warm start of the lattice Boltzmann library (lbm.h).
 *
 * The paper has no learned component; it starts every run from rest.  This
 * part adds a small multilayer perceptron that proposes the initial density
 * and velocity of a tube from its parameters, trained on flow fields that
 * the method itself (lbm_step) has converged, so that a run starts near its
 * steady state instead of from rest.  The zero-velocity start
 * (lbm_init_fields with NULL arrays) stays the fallback.
 *
 * Network: n_layers >= 1 linear layers, widths n_in -> width -> ... -> width
 * -> n_out, tanh between layers and none after the last:
 *     z_l = h_l W_l^T + b_l,  h_0 = x,  h_{l+1} = tanh(z_l),  y = z_{L-1}.
 * Mixed precision: x, W_l, the hidden activations h_l and the back-propagated
 * errors are stored as bfloat16 (round to nearest even); every product is
 * accumulated in FP32 on the tensor cores; biases, outputs, gradients and the
 * optimiser state are FP32.  Loss: mean squared error over the n x n_out
 * outputs.  Optimiser: Adam (Kingma & Ba, 2015) on an FP32 master copy of the
 * parameters, re-rounded to bfloat16 after every step.
 *
 * Parameter vector (FP32): W_0 (row-major [rows_0][cols_0]), b_0, W_1, b_1,
 * ..., with (rows_l, cols_l) = (width, n_in), (width, width), ...,
 * (n_out, width); a one-layer network has W_0 [n_out][n_in].
 *
 * Conventions are those of lbm.h: LBM_* status codes, caller-owned arrays,
 * device memory from the caller's allocator, all work ordered on one stream.
 */
#ifndef LBM_MLP_H
#define LBM_MLP_H

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_mlp lbm_mlp;

/* Largest n_in, width and n_out accepted by lbm_mlp_create. */
enum { LBM_MLP_MAX_IN = 16, LBM_MLP_MAX_WIDTH = 1024, LBM_MLP_MAX_OUT = 16 };

/* Adam step size and decay rates (beta1, beta2 in [0, 1)), and eps > 0. */
typedef struct lbm_adam {
  double lr, beta1, beta2, eps;
} lbm_adam;

/* lbm_mlp_create - a network with zero parameters.  max_batch >= 1 rows per
 * training step (forward passes of more rows run in chunks of max_batch);
 * the activation buffers (about 2 (n_in + 2 width (n_layers + 1)) bytes per
 * row) are allocated here.  alloc may be NULL (cudaMalloc); cuda_stream NULL
 * is the legacy default stream.  LBM_EINVAL for sizes outside the limits. */
int lbm_mlp_create(int32_t n_in, int32_t width, int32_t n_layers, int32_t n_out,
                   int64_t max_batch, const lbm_allocator *alloc, void *cuda_stream,
                   lbm_mlp **out);

/* lbm_mlp_param_count - length of the parameter vector. */
int lbm_mlp_param_count(const lbm_mlp *net, int64_t *count);

/* lbm_mlp_set_params / lbm_mlp_get_params - copy the FP32 parameter vector in
 * or out (src/dst_is_device: device pointer, else host; host copies wait).
 * set_params also resets the optimiser state and its step counter. */
int lbm_mlp_set_params(lbm_mlp *net, const float *theta, int32_t src_is_device);
int lbm_mlp_get_params(lbm_mlp *net, float *theta, int32_t dst_is_device);

/* lbm_mlp_forward - y [n][n_out] = network(x [n][n_in]); device pointers,
 * asynchronous on the network's stream; n >= 0. */
int lbm_mlp_forward(lbm_mlp *net, const float *x, int64_t n, float *y);

/* lbm_mlp_loss_grad - loss (host, waits) and its gradient with respect to the
 * parameter vector for targets t [n][n_out], without changing the network.
 * x, t: device; grad [param_count] FP32 on the device or the host
 * (dst_is_device), may be NULL; 1 <= n <= max_batch. */
int lbm_mlp_loss_grad(lbm_mlp *net, const float *x, const float *t, int64_t n, double *loss,
                      float *grad, int32_t dst_is_device);

/* lbm_mlp_train_step - forward pass, loss, back-propagation and one Adam step
 * on the batch (x, t) (device, 1 <= n <= max_batch).  loss (host) may be
 * NULL: the call then returns without waiting; else it waits and stores the
 * batch loss before the update. */
int lbm_mlp_train_step(lbm_mlp *net, const float *x, const float *t, int64_t n,
                       const lbm_adam *opt, double *loss);

/* lbm_mlp_sync - wait for the network's stream. */
int lbm_mlp_sync(lbm_mlp *net);
const char *lbm_mlp_last_error(const lbm_mlp *net);
void lbm_mlp_destroy(lbm_mlp *net);

/* Frame of a straight tube on the lattice, and the features of its sites.
 *   centre, axis  a point of the tube axis and the unit flow direction, in
 *                 voxel coordinates;
 *   z0, length    axial coordinate (along axis, from centre) of the inlet
 *                 plane, and the tube length;
 *   radius        rest radius;
 *   global        n_global run-level features (already normalised; the
 *                 tube's size, stiffness, inflow and relaxation time);
 *   rho_scale, u_scale  output scales: rho = 1 + rho_scale y_0,
 *                 (u_r, u_z) = u_scale (y_1, y_2).
 * Site features: x = (global..., xi, eta) with xi = (s - z0)/length,
 * eta = r/radius, where s is the axial coordinate and r the distance from the
 * axis of the site; n_in = n_global + 2. */
enum { LBM_WARM_MAX_GLOBAL = 14 };
typedef struct lbm_warm_frame {
  double centre[3];
  double axis[3];
  double z0, length, radius;
  double rho_scale, u_scale;
  int32_t n_global;
  float global[LBM_WARM_MAX_GLOBAL];
} lbm_warm_frame;

/* lbm_warm_features - per-site features x [n_sites][n_global + 2] and, if t
 * is not NULL, training targets t [n_sites][3] = ((rho - 1)/rho_scale,
 * u.e_r/u_scale, u.axis/u_scale) of the context's current fields (e_r the
 * outward radial unit vector, 0 on the axis).  Device pointers, written on
 * the context's stream. */
int lbm_warm_features(lbm_ctx *ctx, const lbm_warm_frame *frame, float *x, float *t);

/* lbm_warm_start - the learned start: features of every site, the network's
 * (rho, u_r, u_z), and f = f^eq(rho, u) at every site (as lbm_init_fields);
 * resets the step counter.  The network needs n_in = n_global + 2 and
 * n_out = 3 and must live on the context's device; the call runs on the
 * context's stream, after the work queued on the network's stream, and
 * waits. */
int lbm_warm_start(lbm_ctx *ctx, lbm_mlp *net, const lbm_warm_frame *frame);

#ifdef __cplusplus
}
#endif

#endif /* LBM_MLP_H */
