/*
 * gmmsp_cnn.h - C ABI of the learned initialiser.
 *
 * Algorithm 1, step 1 of the paper (Sec. III-C) starts every Gaussian at
 * the centre pixel of its grid cell with Sigma_s = diag(v^2, v^2) and
 * Sigma_c = lambda^2 I.  The network here replaces that start: from the
 * CIELAB image it predicts, for every superpixel k, the offset of its fitted
 * mean from that start and the logarithms of its fitted covariance diagonal,
 * so that a few EM iterations (Sec. III-B, unchanged) reach the likelihood
 * that many iterations reach from the paper's start.  This network is not part
 * of the paper.
 *
 * Network (spacing v = 3 f; 32 channels; BF16 weights and activations, FP32
 * accumulation on the tensor cores):
 *   x0: the 3 x 3 pixel patches of each cell (27 values: L/50 - 1, a/50, b/50
 *       of 9 pixels, 5 zeros), f x f patches per cell;
 *   h1 = ReLU(W1 x0 + b1), h2 = ReLU(W2 h1 + b2)       (1 x 1 layers);
 *   c0 = mean of h2 over the cell's patches             (the n_x x n_y grid),
 *        channels 29-31 replaced by the scaled colour of the cell's start
 *        pixel (x_c, y_c) below, so that the cell layers see z_c;
 *   c_l = ReLU(conv3x3(c_{l-1}) + b), l = 1..3          (zero padding);
 *   out = conv3x3(c3) + b6, 16 channels of which 10 are used.
 * Outputs per superpixel k with start point (x_c, y_c) = (k_x v + v/2,
 * k_y v + v/2) and colour z_c there:
 *   0, 1  (mu_x - x_c) / v, (mu_y - y_c) / v
 *   2-4   (mu_L - L_c) / 10, (mu_a - a_c) / 10, (mu_b - b_c) / 10
 *   5, 6  ln(Sigma_s,xx / v^2), ln(Sigma_s,yy / v^2)
 *   7-9   ln(Sigma_c,LL / lambda^2), ln(Sigma_c,aa / lambda^2), ln(Sigma_c,bb / lambda^2)
 * theta_0 is the inverse map: mean clipped to the superpixel's window
 * (Eq. Ik), axis-aligned covariances whose diagonal is floored at eps_s,
 * eps_c (Eq. mlams, mlamc).
 *
 * Parameters: one flat float32 vector of gmmsp_net_param_count() values,
 * in the order W1, b1, W2, b2, W3, b3, W4, b4, W5, b5, W6, b6, with
 * W[cout][tap * 32 + cin] (tap = 3 dy + dx for the 3 x 3 layers, 0 for the
 * 1 x 1 layers), 32 output channels except W6 (16).
 *
 * Images: B CIELAB images of one size W x H, stored as three float32 planes
 * (L, a, b) of W H values each, image after image (the layout of
 * gmmsp_batch_lab).  Only the n_x v x n_y v pixels covered by whole cells
 * are read.
 *
 * Conventions as in gmmsp.h: *_dev device memory owned by the caller,
 * work queued on the network's stream, status codes, no aborts.  A network
 * is not thread-safe.  Device-side waits on the tensor-core barriers are
 * bounded; a wait that runs out sets an error word that gmmsp_net_check
 * (and every call that synchronises) reports as GMMSP_E_TIMEOUT.
 */
#ifndef GMMSP_CNN_H
#define GMMSP_CNN_H

#include "gmmsp.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GMMSP_NET_OUTPUTS 10     /* used outputs per superpixel */
#define GMMSP_NET_CHANNELS 16    /* floats per superpixel in gmmsp_net_forward's output */

typedef struct gmmsp_net_s *gmmsp_net;

/* Number of float32 parameters of the network. */
long long gmmsp_net_param_count(void);

/* A network for spacing v (a multiple of 3, 3 <= v <= 33), parameters zero.
 * stream: the CUDA stream (cudaStream_t, NULL = legacy default) of every call. */
gmmsp_status gmmsp_net_create(gmmsp_net *out, int spacing, void *stream);

/* Parameters in / out (host, count = gmmsp_net_param_count()); set resets the
 * Adam state.  Both synchronise. */
gmmsp_status gmmsp_net_set_weights(gmmsp_net n, const float *host, long long count);
gmmsp_status gmmsp_net_get_weights(gmmsp_net n, float *host, long long count);

/* Optimiser state in / out (host): the Adam first and second moments
 * (count = gmmsp_net_param_count() floats each) and the step count, so that
 * a checkpoint resumes training where it stopped (set after set_weights,
 * which clears the state).  v must be >= 0 and everything finite
 * (GMMSP_E_INVALID otherwise).  Both synchronise. */
gmmsp_status gmmsp_net_get_adam(gmmsp_net n, float *m_host, float *v_host, long long count, long long *step);
gmmsp_status gmmsp_net_set_adam(gmmsp_net n, const float *m_host, const float *v_host, long long count,
                                long long step);

/* Forward pass over B images: out_dev receives B n_y n_x x GMMSP_NET_CHANNELS
 * float32 (superpixel-major, k = k_y n_x + k_x within an image).  The first
 * call for a larger batch allocates workspace. */
gmmsp_status gmmsp_net_forward(gmmsp_net n, const float *lab_dev, int B, int W, int H, float *out_dev);

/* Loss and gradient.  target_dev: B K x GMMSP_NET_OUTPUTS float32 (see
 * gmmsp_batch_targets).  Loss = mean over the B K x 10 used outputs of the
 * squared difference.  The gradient goes to the network's gradient buffer
 * and, when grad_host is not NULL, to the host (param_count floats); when
 * grad_host or loss_host is given the call synchronises. */
gmmsp_status gmmsp_net_grad(gmmsp_net n, const float *lab_dev, int B, int W, int H, const float *target_dev,
                            float *grad_host, double *loss_host);

/* One Adam step (Kingma and Ba 2015) with the gradient of the last
 * gmmsp_net_grad. */
gmmsp_status gmmsp_net_adam(gmmsp_net n, float lr, float beta1, float beta2, float eps);

/* gmmsp_net_grad + gmmsp_net_adam(lr, 0.9, 0.999, 1e-8); loss_host (may be
 * NULL) receives the loss before the step, and then the call synchronises. */
gmmsp_status gmmsp_net_train_step(gmmsp_net n, const float *lab_dev, int B, int W, int H,
                                  const float *target_dev, float lr, double *loss_host);

/* Hidden activation c_layer (layer 0..3: the pooled grid c0 and the 3 x 3
 * layers c1..c3) of the last forward pass (gmmsp_net_forward, gmmsp_net_grad
 * or a learned start), converted to float32: count = B K x 32 values,
 * superpixel-major.  Synchronises.  For tests and diagnostics. */
gmmsp_status gmmsp_net_get_activation(gmmsp_net n, int layer, float *host, long long count);

/* Synchronises the stream; GMMSP_E_TIMEOUT if a device wait ran out since
 * the network was created. */
gmmsp_status gmmsp_net_check(gmmsp_net n);

/* Self-test of the bounded device-side waits used by the network kernels:
 * one block allocates tensor memory, waits on an mbarrier that nothing
 * arrives on for max_tries polls (1 .. 2^20), frees the tensor memory and
 * reports.  Returns GMMSP_E_TIMEOUT when the wait gave up, which is the
 * expected outcome.  The context stays usable.  Synchronises the stream
 * (cudaStream_t, NULL = legacy default). */
gmmsp_status gmmsp_tc_wait_selftest(int max_tries, void *stream);

const char *gmmsp_net_last_error(gmmsp_net n);
void gmmsp_net_destroy(gmmsp_net n);

/* ---- use with the EM contexts ----
 * gmmsp_init_from_net: replaces theta of a single-image context by the
 *   network's theta_0 for the context's current image (after gmmsp_init or
 *   gmmsp_reinit); the spacing must match.  Then gmmsp_em_iters /
 *   gmmsp_labels as usual.  The context must use GMMSP_COLOUR_FULL
 *   (GMMSP_E_INVALID otherwise, the context stays usable).
 * gmmsp_batch_set_init_net: every later gmmsp_batch_segment on b starts from
 *   the network's theta_0 instead of Sec. III-C (n = NULL restores it).  All
 *   images of b must have one size and b the network's spacing and the full
 *   colour model.  The network must outlive its use by b.
 * gmmsp_batch_lab: device pointer to b's CIELAB planes (valid until b is
 *   destroyed; filled by gmmsp_batch_segment).
 * gmmsp_batch_targets: training targets (B K x 10 float32, layout of the
 *   network outputs) from b's current theta, e.g. after many EM iterations.
 *   All images of b must have one size; the full colour model only. */
gmmsp_status gmmsp_init_from_net(gmmsp_ctx c, gmmsp_net n);

/* gmmsp_set_init: replaces theta of a single-image context by theta_0 built
 * from a caller's per-superpixel predictions in the network's output
 * parametrisation (device float32, K x 5 each, superpixel k = k_y n_x + k_x):
 *   dmu_dev     mean offsets from the cell's centre pixel (x_c, y_c, z_c):
 *               (dx, dy) in units of the spacing v, (dL, da, db) in units
 *               of 10 CIELAB;
 *   logeig_dev  logs of the covariance diagonals, Sigma_s in units of v^2
 *               (2 values), Sigma_c in units of lambda_c^2 (3 values),
 *               clipped to [-10, 10];
 * the spatial mean is clipped to the superpixel's window (Eq. Ik) and the
 * eigenvalues are floored at eps_s, eps_c (Eq. mlams, mlamc).  Not for the
 * grayscale model (GMMSP_E_INVALID).  A non-finite result is reported as
 * GMMSP_E_NUMERIC at the next synchronising call. */
gmmsp_status gmmsp_set_init(gmmsp_ctx c, const float *dmu_dev, const float *logeig_dev);
gmmsp_status gmmsp_batch_set_init_net(gmmsp_batch b, gmmsp_net n);
gmmsp_status gmmsp_batch_lab(gmmsp_batch b, const float **lab_dev);
gmmsp_status gmmsp_batch_targets(gmmsp_batch b, float *target_dev);

#ifdef __cplusplus
}
#endif

#endif /* GMMSP_CNN_H */
