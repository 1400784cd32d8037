/*
 * gmmsp_metrics.h - accuracy of a superpixel segmentation against a ground
 * truth, the three metrics of Sec. IV of the paper (N pixels, superpixel
 * pixel sets s_k, ground-truth segments s_g):
 *   BR   boundary recall: the fraction of ground-truth boundary pixels with a
 *        superpixel boundary pixel within Chebyshev distance `radius` (the
 *        paper: two pixels).  A boundary pixel is a pixel with a 4-neighbour
 *        of another label (both sides of an edge count).
 *   UE   Eq. (ue): (1/N) sum over pairs (k, g) with |s_k & s_g| > eps |s_k| of
 *        |s_k|, minus 1 (the paper: eps = 0.05).
 *   ASA  Eq. (asa): (1/N) sum_k max_g |s_k & s_g|.
 * All three come from integer counts, so the results are exact; the counts
 * are returned too.
 */
#ifndef GMMSP_METRICS_H
#define GMMSP_METRICS_H

#include <stdint.h>

#include "gmmsp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double br, ue, asa;
    long long br_recovered, br_total;   /* BR = br_recovered / br_total (1 when there is no boundary) */
    long long ue_sum;                   /* UE = ue_sum / N - 1 */
    long long asa_sum;                  /* ASA = asa_sum / N */
} gmmsp_seg_metrics;

/* labels_dev: W H int32 superpixel labels in [0, K); gt_dev: W H int32
 * ground-truth segment ids in [0, G) (both device memory, row-major, owned by
 * the caller).  K G must not exceed 2^31 (a dense K x G overlap table is
 * counted on the device).  Allocates its scratch, works on `stream`
 * (cudaStream_t, NULL = legacy default) and synchronises.  Returns
 * GMMSP_E_INVALID for bad arguments or for a label or id out of range (found
 * on the device), GMMSP_E_NOMEM / GMMSP_E_CUDA on CUDA failures. */
gmmsp_status gmmsp_segmentation_metrics(const int32_t *labels_dev, const int32_t *gt_dev, int W, int H, int K,
                                        int G, int radius, double eps, gmmsp_seg_metrics *out_host,
                                        void *stream);

/* The same for n images in one call (four kernel launches for all of them,
 * one allocation, one synchronisation): image i is labels_dev[i], gt_dev[i]
 * of W[i] x H[i] pixels with K[i] superpixels and G[i] segments, and its
 * metrics go to out_host[i] (n entries).  Returns GMMSP_E_INVALID for bad
 * arguments, or when a label or id of any image is out of range (out_host is
 * filled for all images then). */
gmmsp_status gmmsp_segmentation_metrics_many(int n, const int32_t *const *labels_dev, const int32_t *const *gt_dev,
                                             const int *W, const int *H, const int *K, const int *G, int radius,
                                             double eps, gmmsp_seg_metrics *out_host, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GMMSP_METRICS_H */
