/*
 * gmmsp.h - C ABI of the GB300 (sm_103a) GMM superpixel library.
 *
 * The library computes the superpixels of Ban, Liu and Cao, "Superpixel
 * Segmentation Using Gaussian Mixture Model" (arXiv 1612.08792): one Gaussian
 * per grid seed over the 5-D pixel vector z = (x, y, L, a, b) with a block
 * diagonal covariance (Sec. III-C, Eq. BlockSigma), fitted by EM (Sec. III-B)
 * where each pixel only sees the Gaussians of its neighbouring seeds
 * (Eq. Ik), with the eigenvalue floor of Eq. (mlams)/(mlamc), and a label per
 * pixel by maximum posterior (Eq. obtLi).  Algorithm 1, steps 1-7, is split
 * over gmmsp_init (step 1), gmmsp_em_iters (steps 2-6) and gmmsp_labels
 * (step 7).  The connectivity post-processing (step 8) is not part of it.
 *
 * Conventions for every call:
 *   - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *     memory must stay valid until the work queued on the context's stream
 *     has finished.  Pointers named *_host are ordinary host memory.
 *   - Work is queued on the CUDA stream given to gmmsp_init and returns
 *     without waiting, except where a call says it synchronises.
 *   - A call returns a gmmsp_status and never aborts the process.  Invalid
 *     arguments are reported before any work is queued.  A CUDA error, or a
 *     non-finite input found on the device, puts the context into an error
 *     state: that call and every later call on it return GMMSP_E_STATE or
 *     the original code; gmmsp_last_error() describes the cause.
 *   - Contexts are not thread-safe; use one context per host thread.
 *   - Superpixel k sits at grid cell (k_x, k_y) = (k mod n_x, k / n_x)
 *     (Eq. kxy).  Per-superpixel arrays are indexed by k.
 */
#ifndef GMMSP_H
#define GMMSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmmsp_ctx_s *gmmsp_ctx;   /* opaque, owned by the library */

typedef enum {
    GMMSP_OK = 0,
    GMMSP_E_INVALID = 1,   /* bad argument; nothing was queued            */
    GMMSP_E_CUDA = 2,      /* a CUDA call failed                          */
    GMMSP_E_NOMEM = 3,     /* device allocation failed                    */
    GMMSP_E_NUMERIC = 4,   /* non-finite input or parameters              */
    GMMSP_E_TIMEOUT = 5,   /* a bounded device-side wait ran out          */
    GMMSP_E_STATE = 6      /* context is in an error state / wrong state  */
} gmmsp_status;

/* Image formats accepted by gmmsp_init / gmmsp_reinit. */
enum {
    GMMSP_RGB8 = 0,   /* H rows of W x (R,G,B) uint8 sRGB, row pitch in bytes   */
    GMMSP_LAB32 = 1,  /* H rows of W x (L,a,b) float32 CIELAB, row pitch in bytes */
    GMMSP_GRAY8 = 2   /* H rows of W uint8 grey levels (sRGB-encoded luminance),
                         row pitch in bytes; only with GMMSP_COLOUR_GRAY       */
};

/* Colour covariance model (Sec. III-A, III-C). */
enum {
    GMMSP_COLOUR_FULL = 0,  /* Sigma_c a full 3x3 over (L, a, b), Eq. (BlockSigma)  */
    GMMSP_COLOUR_SPLIT = 1, /* Sigma_c = diag(sigma_l^2, Sigma_(a,b)), Eq. (BlockSigma1):
                               no L-(a, b) covariance, a cheaper E- and M-step     */
    GMMSP_COLOUR_GRAY = 2   /* grayscale: the colour is the scalar CIE L* (of the L
                               channel of a colour input, or of a grey level), so
                               z = (x, y, L) and Sigma_c = sigma^2                  */
};

/* Arithmetic of the EM loop. */
enum {
    GMMSP_PREC_MIXED = 0, /* FP32 E-step and per-cell partial sums; the
                             superpixel sums formed FP64-accurate (FP32 pairs,
                             error-free TwoSum), FP64 update, floor, inversion */
    GMMSP_PREC_FP32 = 1   /* everything in FP32, raw (unshifted) moments    */
};

typedef struct {
    int spacing;        /* v_x = v_y; if > 0 it wins over K (Eq. nxyK)          */
    int K;              /* requested superpixel count; v = floor(sqrt(WH/K))
                           (Eq. vxy).  The effective K = n_x n_y is reported by
                           gmmsp_get_grid.                                     */
    float eps_s;        /* spatial eigenvalue floor, px^2 (Sec. III-C: 2)       */
    float eps_c;        /* colour eigenvalue floor, CIELAB^2 (Sec. IV-A: 8)     */
    float lambda_c;     /* initial colour standard deviation; Sigma_c,0 =
                           lambda_c^2 I (Sec. III-C; Sec. IV-A uses 8)          */
    int input_format;   /* GMMSP_RGB8, GMMSP_LAB32 or GMMSP_GRAY8              */
    int precision;      /* GMMSP_PREC_MIXED or GMMSP_PREC_FP32 (FULL model only) */
    int colour_model;   /* GMMSP_COLOUR_FULL, _SPLIT or _GRAY.  The split and
                           grayscale models are mixed precision only, and the
                           learned initialiser, the training targets and the
                           allocation-free entry point take the full model
                           only (GMMSP_E_INVALID otherwise).  Parameters come
                           out in the full layout: the split model's L-a, L-b
                           covariances are 0; grayscale has mu's a, b and
                           every Sigma_c entry but LL at 0.                    */
} gmmsp_params;

/* Fills p with the paper's settings: spacing 0, K 0 (the caller sets one of
 * them), eps_s 2, eps_c 8, lambda_c 8, RGB8, mixed precision, full colour
 * covariance. */
void gmmsp_default_params(gmmsp_params *p);

/*
 * Creates a context for W x H images and runs Algorithm 1, step 1 on
 * image_dev: converts the image to CIELAB (Sec. IV) and sets theta_0
 * (Sec. III-C: mu_k = z at the centre pixel of cell k, Sigma_s =
 * diag(v^2, v^2), Sigma_c = lambda_c^2 I).
 *   image_dev    device pointer to the first row (see GMMSP_RGB8/LAB32);
 *   pitch_bytes  distance between rows in bytes, >= 3 W (RGB8), 12 W (LAB32)
 *                or W (GRAY8);
 *   stream       cudaStream_t to queue work on (NULL = legacy default stream).
 * Allocates the context's device buffers (O(W H) bytes for the CIELAB image,
 * O(K) for theta and the per-cell partial sums).  Errors: GMMSP_E_INVALID
 * when W, H < 1, when neither spacing nor K is positive, when the grid is
 * empty (n_x or n_y = 0), when eps or lambda_c is not positive, for an
 * unknown format or colour model, or an unsupported combination of them
 * (see gmmsp_params); GMMSP_E_NOMEM; GMMSP_E_CUDA.  On error *out is NULL.
 */
gmmsp_status gmmsp_init(gmmsp_ctx *out, const void *image_dev, int width, int height,
                        int pitch_bytes, const gmmsp_params *p, void *stream);

/* Algorithm 1, step 1 again for a new image of the same size and format,
 * without allocating.  Clears an earlier error state. */
gmmsp_status gmmsp_reinit(gmmsp_ctx c, const void *image_dev, int pitch_bytes);

/*
 * Runs `iters` rounds of Algorithm 1, steps 4-6 on the current theta: each
 * round is an E-step over every pixel (Eq. Rik, each pixel over its <= 9
 * candidate Gaussians of Eq. Ik) fused with the per-cell partial sums of the
 * M-step, then the mean and block covariance update (Eq. UpdateMu,
 * UpdateSigS, UpdateSigC) with the eigenvalue floor (Eq. mlams, mlamc).
 * The first E-step of a round on theta_t also gives L(theta_t) (the
 * log-likelihood following Eq. ftheta, natural log, with the
 * (2 pi)^(-5/2) constant).
 *   loglik_host  NULL, or `iters` doubles receiving L(theta_t) of each round;
 *                when non-NULL the call synchronises the stream.
 * iters = 0 does nothing.  Errors: GMMSP_E_INVALID (iters < 0),
 * GMMSP_E_CUDA, GMMSP_E_STATE.
 */
gmmsp_status gmmsp_em_iters(gmmsp_ctx c, int iters, double *loglik_host);

/*
 * Algorithm 1, step 7 (with the E-step of step 6 on the current theta):
 * labels_dev[y W + x] = argmax over the pixel's candidates k of the
 * posterior (Eq. obtLi); ties go to the smaller k.
 *   labels_dev   device int32 array of W H entries, written;
 *   loglik_host  NULL or one double receiving L(theta) of this E-step;
 *                when non-NULL the call synchronises the stream.
 */
gmmsp_status gmmsp_labels(gmmsp_ctx c, int32_t *labels_dev, double *loglik_host);

/*
 * Whole pipeline in one call, Algorithm 1 steps 1-7: gmmsp_reinit(image),
 * gmmsp_em_iters(iters), gmmsp_labels.  The kernel sequence is captured into
 * a CUDA graph on the first call for a given (iters, image, labels) and
 * replayed afterwards, so repeated calls cost one graph launch.
 *   loglik_host  NULL, or iters + 1 doubles: L(theta_0) .. L(theta_iters);
 *                when non-NULL the call synchronises the stream.
 */
gmmsp_status gmmsp_segment(gmmsp_ctx c, const void *image_dev, int pitch_bytes, int iters,
                           int32_t *labels_dev, double *loglik_host);

/*
 * Copies the context's CIELAB image (the pixel colours c_i of z_i, Sec. III-A,
 * after the conversion of Sec. IV) to the host as W H x (L, a, b) float32
 * (synchronises).  Errors: GMMSP_E_INVALID for NULL.
 */
gmmsp_status gmmsp_get_lab(gmmsp_ctx c, float *lab_host);

/* Grid of Eq. (vxy)/(nxyK): spacing v, n_x, n_y, K = n_x n_y.  Any pointer may be NULL. */
gmmsp_status gmmsp_get_grid(gmmsp_ctx c, int *v, int *nx, int *ny, int *K);

/*
 * Copies theta to the host (synchronises): mu_host K x 5 (x, y, L, a, b),
 * cov_s_host K x 3 (xx, xy, yy), cov_c_host K x 6 (LL, La, Lb, aa, ab, bb),
 * the floored covariances of Eq. (eigdecrs)/(eigdecrc).  Any may be NULL.
 */
gmmsp_status gmmsp_get_params(gmmsp_ctx c, double *mu_host, double *cov_s_host, double *cov_c_host);

/*
 * Replaces theta (same layout as gmmsp_get_params), e.g. to resume EM from a
 * saved state or to start from another initialisation.  Covariances must be
 * symmetric positive definite; they are used as given (no floor).  Errors:
 * GMMSP_E_INVALID for a NULL pointer, GMMSP_E_NUMERIC for a non-finite value
 * or a covariance that is not positive definite.  Synchronises.
 */
gmmsp_status gmmsp_set_params(gmmsp_ctx c, const double *mu_host, const double *cov_s_host,
                              const double *cov_c_host);

/*
 * Counters since the last init/reinit (synchronises): dead = superpixels
 * kept unchanged because their total posterior weight was below 1e-8;
 * raised_s / raised_c = eigenvalues lifted to eps_s / eps_c by the floor.
 * Any pointer may be NULL.
 */
gmmsp_status gmmsp_get_stats(gmmsp_ctx c, long long *dead, long long *raised_s, long long *raised_c);

/*
 * Kernel timing (no counterpart in the paper: a measurement aid).  Launches
 * one kernel of the pipeline `reps` times on the context's stream, each
 * launch between two CUDA events, and returns the mean launch time in
 * milliseconds (synchronises).  `which` is
 *   GMMSP_KERNEL_EM_PASS  (0)  the fused E-step + M-step partial pass on
 *                              the current theta (rewrites the partial sums);
 *   GMMSP_KERNEL_LABELS   (1)  the label pass (writes labels_dev);
 *   GMMSP_KERNEL_FINALIZE (2)  the FP64 M-step finalize on the current partial
 *                              sums; theta is saved before the first launch
 *                              and restored before each one (outside the
 *                              timed interval), so the call leaves theta as
 *                              it found it.  Allocates a K-sized scratch copy.
 * If flush_dev is non-NULL, flush_bytes of it are overwritten before every
 * launch (outside the timed interval) so each launch starts with a cold L2.
 */
enum { GMMSP_KERNEL_EM_PASS = 0, GMMSP_KERNEL_LABELS = 1, GMMSP_KERNEL_FINALIZE = 2 };
gmmsp_status gmmsp_profile_kernel(gmmsp_ctx c, int which, int reps, int32_t *labels_dev,
                                  void *flush_dev, unsigned long long flush_bytes, double *avg_ms);

/*
 * Launch shape of the fused E + M-partial pass (no counterpart in the paper):
 * the number of warps that share one v x v cell, 1, 2 or 4.  More warps per
 * cell give small images more parallelism; one warp per cell has the least
 * reduction work for large images.  gmmsp_init picks a default from the
 * cell count.  Changing it drops a captured gmmsp_segment graph.
 */
gmmsp_status gmmsp_set_launch(gmmsp_ctx c, int warps_per_cell);
gmmsp_status gmmsp_get_launch(gmmsp_ctx c, int *warps_per_cell);

/*
 * Autotuner: times the E + M-partial pass on the current theta for each
 * launch shape (1, 2, 4 warps per cell; `reps` timed launches each after
 * one warm-up), keeps the fastest and returns it in *best (may be NULL);
 * times_ms (NULL or 3 doubles) receives the mean time of each shape.
 * Synchronises.
 */
gmmsp_status gmmsp_autotune(gmmsp_ctx c, int reps, int *best, double *times_ms);

/*
 * Batches: many images of uneven sizes segmented together, Algorithm 1,
 * steps 1-7, for every image, with one kernel launch per step for the whole
 * batch (persistent blocks walk the batch's cells / superpixels), the step
 * sequence captured into one CUDA graph on the first call (per iteration
 * count) and replayed afterwards.  The paper segments one image at a time;
 * batching is this library's way of filling the GPU with small images.
 *
 * gmmsp_batch_create: n images with sizes widths[i] x heights[i] (host
 *   arrays), shared parameters p (spacing or K per image as for gmmsp_init,
 *   format, precision), work queued on `stream`.  Allocates one device block
 *   for all images' CIELAB planes, parameters and partial sums.  Errors as
 *   for gmmsp_init.
 * gmmsp_batch_segment: images_dev[i] (device rows, pitches[i] bytes each) in,
 *   labels_dev[i] (device int32 W H) out; host arrays of n pointers / pitches.
 *   loglik_host NULL or n doubles: L(theta_iters) of each image (the label
 *   pass' log-likelihood); when non-NULL the call synchronises.  The image
 *   table is copied to the device on every call, so the pointers may change
 *   between calls without a new capture.
 * gmmsp_batch_get_params: theta of image i (layout of gmmsp_get_params);
 *   synchronises.
 * gmmsp_batch_autotune: times the batch E + M-partial pass at 3, 4, 5, 6 and
 *   7 blocks per SM (`reps` launches each, on the given images; 3-5: a
 *   persistent grid of that many blocks per SM; 6, 7: one cell per warp with
 *   the registers capped for that occupancy), keeps the fastest, then times
 *   the two finalize kernels and keeps the faster; times_ms NULL or 5
 *   doubles (E + M pass, in candidate order).  The first pass of a segment
 *   (its covariance blocks are diagonal after either start, Sec. III-C or the
 *   learned one) gets a choice of its own: the diagonal kernels at 6 and 7
 *   are timed too, and the fastest of them and the 3-5 times is kept.
 *   Synchronises.
 * gmmsp_batch_set_launch: blocks per SM of the E + M pass (1..16; >= 6
 *   selects the one-cell-per-warp kernel); the first pass keeps its own
 *   choice where the autotuner or gmmsp_batch_set_first_pass made one.
 * gmmsp_batch_set_first_pass: blocks per SM of a segment's first E + M pass
 *   (1..16, or 0: the same as the other passes; the default).
 * gmmsp_batch_get_first_pass: the first pass's blocks per SM in effect and,
 *   in times_ms (NULL or 2 doubles), the autotuned times of its diagonal
 *   kernels at 6 and 7 (ms; 0 before gmmsp_batch_autotune).
 * gmmsp_batch_info: totals over the batch (any pointer may be NULL).
 */
typedef struct gmmsp_batch_s *gmmsp_batch;
gmmsp_status gmmsp_batch_create(gmmsp_batch *out, int n, const int *widths, const int *heights,
                                const gmmsp_params *p, void *stream);
gmmsp_status gmmsp_batch_segment(gmmsp_batch b, const void *const *images_dev, const int *pitches,
                                 int iters, int32_t *const *labels_dev, double *loglik_host);
gmmsp_status gmmsp_batch_get_params(gmmsp_batch b, int i, double *mu_host, double *cov_s_host,
                                    double *cov_c_host);
gmmsp_status gmmsp_batch_autotune(gmmsp_batch b, const void *const *images_dev, const int *pitches,
                                  int32_t *const *labels_dev, int reps, int *best, double *times_ms);
gmmsp_status gmmsp_batch_set_launch(gmmsp_batch b, int blocks_per_sm);
gmmsp_status gmmsp_batch_set_first_pass(gmmsp_batch b, int blocks_per_sm);
gmmsp_status gmmsp_batch_get_first_pass(gmmsp_batch b, int *blocks_per_sm, double *times_ms);
/* One E + M pass from the start, for checking the first-pass kernels (Algorithm
 * 1 steps 1-3: the conversion and theta_0 as a segment begins, Sec. III-C or
 * the network; then the E-step, Eq. Rik, and the M-step partial sums of Eq.
 * UpdateMu / UpdateSigS / UpdateSigC per cell), at blocks_per_sm (1..16, as
 * gmmsp_batch_set_launch) with diagonal 1 (the kernel that leaves the zero
 * off-diagonal covariance terms of theta_0 out) or 0 (the general kernel).
 * Copies the per-cell partials to partials_host: total_cells rows of 136 FP32
 * values (9 candidate slots x 15 statistics, then the cell's log-likelihood;
 * mixed precision: statistics about the previous mean, log2 units; FP32
 * precision: raw moments, nats), *n_floats of them.  With partials_host
 * NULL only *n_floats is set.  Images, pitches and labels as
 * gmmsp_batch_segment (labels are not written).  Synchronises the batch's
 * stream.  Errors: GMMSP_E_INVALID for a NULL handle, both outputs NULL or an
 * argument out of range; GMMSP_E_CUDA on a CUDA error. */
gmmsp_status gmmsp_batch_first_pass_partials(gmmsp_batch b, const void *const *images_dev, const int *pitches,
                                             int32_t *const *labels_dev, int blocks_per_sm, int diagonal,
                                             float *partials_host, long long *n_floats);
/* Launch choices of b: blocks per SM of the E + M pass, whether the finalize
 * runs 16 lanes per superpixel (1) or one thread per superpixel (0), and the
 * two finalize times the autotuner measured (ms; 0 before gmmsp_batch_autotune).
 * Any pointer may be NULL. */
gmmsp_status gmmsp_batch_get_tuning(gmmsp_batch b, int *blocks_per_sm, int *finalize16, double *finalize_ms);
/* Sets both launch choices, e.g. from a tuning cache (blocks_per_sm 1..16,
 * finalize16 0 or 1; finalize16 has an effect only where the 16-lane
 * finalize applies: mixed precision, full colour model).  The first E + M
 * pass follows blocks_per_sm again until gmmsp_batch_set_first_pass. */
gmmsp_status gmmsp_batch_set_tuning(gmmsp_batch b, int blocks_per_sm, int finalize16);
gmmsp_status gmmsp_batch_info(gmmsp_batch b, long long *total_pixels, int *total_k, int *total_cells);
/* Copies image i's CIELAB colours (Sec. III-A, after the conversion of Sec.
 * IV) as the last gmmsp_batch_segment left them on the device to the host as
 * W H x (L, a, b) float32 (synchronises the batch's stream).
 * Errors: GMMSP_E_INVALID for NULL or i outside [0, n). */
gmmsp_status gmmsp_batch_get_lab(gmmsp_batch b, int i, float *lab_host);
const char *gmmsp_batch_last_error(gmmsp_batch b);
void gmmsp_batch_destroy(gmmsp_batch b);

/*
 * Bounds-check status (no counterpart in the paper: a stand-in for a memory
 * checker, which is not run on this hardware).  A library built with the
 * compile flag GMMSP_CHECK_BOUNDS (paper_1612_08792_gb300/build.py,
 * build(checked=True): _build/libgmmsp_checked.so) tests the index of every
 * global-memory access of the EM kernels against its buffer -- candidate
 * coefficients, pixel reads, per-cell partial sums, superpixel parameters,
 * labels and their values, the batch table lookups, the CIELAB writes of the
 * learned start's converting first kernel -- skips an access that
 * falls outside and records the first such event of each kernel translation
 * unit.  The ordinary build compiles the checks away.
 *   checked          receives 1 if this library was built with the checks,
 *                    else 0;
 *   first_violation  receives 0 if nothing was recorded since the last call,
 *                    else (1 << 63) | site << 40 | (index mod 2^40), site one
 *                    of the GMMSP_BND_* values.
 * A checked library synchronises the device, reads and clears the status
 * words; an unchecked one touches no device.  Either pointer may be NULL.
 * Errors: GMMSP_E_CUDA.
 */
#define GMMSP_BND_GP 1         /* a candidate's packed coefficients: superpixel in [0, K) */
#define GMMSP_BND_PIXEL_X 2    /* a pixel read: x in [0, W)                                */
#define GMMSP_BND_PIXEL_Y 3    /* a pixel read or write: y in [0, H) (or the pixel index) */
#define GMMSP_BND_PARTIAL_W 4  /* a cell's partial sums written: cell in [0, cells)        */
#define GMMSP_BND_PARTIAL_R 5  /* partial sums read by the finalize: cell in [0, cells)    */
#define GMMSP_BND_THETA 6      /* a superpixel's parameters written: k in [0, K)           */
#define GMMSP_BND_LABEL 7      /* a label written: pixel in [0, W H)                       */
#define GMMSP_BND_LABEL_K 8    /* a label's value: k in [0, K)                             */
#define GMMSP_BND_CELL_LL 9    /* a cell's log-likelihood written: cell in [0, cells)      */
#define GMMSP_BND_IMAGE 10     /* a batch item's image: in [0, n)                          */
#define GMMSP_BND_ITEM 11      /* a batch item in its image: cell or superpixel in range   */
gmmsp_status gmmsp_bounds_status(int *checked, unsigned long long *first_violation);

/*
 * Allocation-free segmentation (the paper has no counterpart; this serves
 * callers that cannot allocate device memory where they run: code inside a
 * memory pool or a caching allocator that owns all device memory, code that
 * must not trigger the device synchronisation that cudaMalloc/cudaFree can
 * cause, and plug-ins that are only handed their input and output buffers).
 *
 * Runs the same steps as gmmsp_init (GMMSP_LAB32) + gmmsp_em_iters(iters) +
 * gmmsp_labels on a CIELAB image, with the same kernels, and allocates
 * nothing: its working memory (theta, the packed E-step coefficients, the
 * per-cell partial sums, counters) is one fixed __device__ array of
 * GMMSP_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads
 * the library holds until the process exits.
 *   lab_dev      device rows of W x (L, a, b) float32, 4-byte aligned;
 *   pitch_bytes  row pitch, >= 12 W, a multiple of 4;
 *   p            spacing or K, eps_s, eps_c, lambda_c as for gmmsp_init
 *                (finite and > 0; input_format is ignored; precision must be
 *                MIXED and colour_model FULL);
 *   labels_dev   device int32[W H], written (argmax posterior, Eq. obtLi);
 *   stream       cudaStream_t to queue on; the call does not synchronise;
 *   err          NULL, or err_len bytes receiving a message on failure.
 * Non-finite input is not detected here (the context and batch paths report
 * it as GMMSP_E_NUMERIC; this call never synchronises to read a counter):
 * the parameters of the superpixels it reaches become NaN, and the labels of
 * their pixels are then unspecified, though each still names one of its
 * pixel's candidate superpixels (Eq. Ik).
 * Limits: the cell grid ceil(W/v) x ceil(H/v) may hold at most
 * GMMSP_NOALLOC_MAX_CELLS cells (e.g. 481x321 at v >= 8, 1920x1080 at
 * v >= 30); larger grids return GMMSP_E_INVALID with the sizes in err.
 * Every call shares the one array, which keeps the previous call's
 * contents (the call clears what must start at zero): calls that overlap on
 * the GPU (different streams, devices' work still in flight on another
 * stream) race and must be serialised by the caller.  On each device the
 * first call looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.
 */
#define GMMSP_NOALLOC_MAX_CELLS 4096
#define GMMSP_NOALLOC_SCRATCH_BYTES ((5u << 20) + (64u << 10))
gmmsp_status gmmsp_segment_lab_noalloc(const float *lab_dev, int width, int height, int pitch_bytes,
                                       const gmmsp_params *p, int iters, int32_t *labels_dev,
                                       void *stream, char *err, int err_len);

/*
 * In-pipeline kernel timing (no counterpart in the paper: a measurement aid).
 * gmmsp_set_timing(c, 1) makes every later call record a CUDA event between
 * its steps (inside a gmmsp_segment graph they become event nodes; changing
 * the setting drops a captured graph).  gmmsp_get_timing synchronises and
 * returns, for the last call that queued work, the milliseconds between
 * consecutive events: for gmmsp_segment with T iterations the 2T + 2 values
 * are [conversion + theta_0, E+M pass 0, finalize 0, ..., E+M pass T-1,
 * finalize T-1, label pass]; gmmsp_em_iters gives the 2T pass/finalize
 * values; gmmsp_labels one.  *n receives the count, at most cap are written.
 */
gmmsp_status gmmsp_set_timing(gmmsp_ctx c, int enable);
gmmsp_status gmmsp_get_timing(gmmsp_ctx c, double *ms, int cap, int *n);

/* Text of the last error on c (never NULL; "" when there is none). */
const char *gmmsp_last_error(gmmsp_ctx c);

/* Name of a status code. */
const char *gmmsp_status_string(gmmsp_status s);

/* Frees the context and its device buffers (synchronises its stream). NULL is ignored. */
void gmmsp_destroy(gmmsp_ctx c);

#ifdef __cplusplus
}
#endif

#endif /* GMMSP_H */
