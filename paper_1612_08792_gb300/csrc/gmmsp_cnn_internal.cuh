// Library-internal entry points of the learned initialiser, used by the
// single-image context and the batch context.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/gmmsp.h"
#include "../../include/gmmsp_cnn.h"
#include "gmmsp_internal.cuh"

namespace gmmsp {

// Checks that the network fits B images of geometry g (same spacing) and
// reserves its inference workspace.  Must not be called during stream capture.
gmmsp_status net_reserve(gmmsp_net n, int B, const Geom& g, std::string* why);

// Changes whenever the network's workspace moves (captured graphs must be
// re-captured then).
long long net_generation(gmmsp_net n);

// Enqueues the network on B CIELAB images (planes of W H floats, image after
// image) and writes theta_0 and the packed coefficients of all B K
// superpixels.  A non-finite theta_0 counts into counters[CNT_NONFINITE].
// With rgb non-null (a device batch table of B RGB8 images, all of geometry
// g, CIELAB planes at lab + 3 pix_off) the network's first kernel also does
// the sRGB -> CIELAB conversion of every pixel inside the n_x v x n_y v
// cell region and writes it to lab; the pixels outside it are left to the
// caller (launch_prepare_batch with skip_cells).
cudaError_t net_enqueue_init(gmmsp_net n, float* lab, const BatchImage* rgb, int B, const Geom& g,
                             double lambda_c, double eps_s, double eps_c, double* theta, float* gp,
                             unsigned long long* counters, cudaStream_t s);

// theta_0 and the packed coefficients of B K superpixels from the network's
// output parametrisation given as two device arrays: superpixel i's 5 mean
// offsets at dmu + i ds and 5 log-eigenvalues at logeig + i ls.
cudaError_t launch_init_from_outputs(const float* dmu, int ds, const float* logeig, int ls, const float* lab, int B,
                                     const Geom& g, double lambda_c, double eps_s, double eps_c, double* theta,
                                     float* gp, unsigned long long* counters, cudaStream_t s);

// Training targets (GMMSP_NET_OUTPUTS floats per superpixel) from fitted
// parameters theta of B images of geometry g.
cudaError_t launch_targets(const double* theta, const float* lab, int B, const Geom& g, double lambda_c,
                           float* target, cudaStream_t s);

}  // namespace gmmsp
