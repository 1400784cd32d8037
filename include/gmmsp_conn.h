/*
 * gmmsp_conn.h - connectivity post-processing of a label map (Algorithm 1,
 * step 8; Sec. III-D of the paper).
 *
 * The paper sorts the isolated superpixels by size and merges, one after the
 * other, those smaller than a quarter of the desired superpixel size into the
 * neighbouring superpixel nearest in colour; a merge adds the source's size
 * to the destination's.  Readings:
 *   - an isolated superpixel is a 4-connected component of one label; the
 *     desired size is N / K, so a component c is small when 4 K |c| < N;
 *   - components are taken in order of (size, smallest pixel index), fixed
 *     before the merging; at its turn a component is merged only if it is
 *     still small (merges into it count) and has a neighbour;
 *   - its neighbours are the current groups of the components 4-adjacent to
 *     its group; the nearest is the one whose founding component's mean
 *     colour is closest (squared CIELAB distance; ties to the smaller index);
 *     a component's mean colour is sum(round(2^20 z)) / |c| (integer sums);
 *   - every pixel takes the label of its group's founding component.
 * The result equals the sequential pass over the whole image (the GPU runs
 * it independently per cluster of adjacent small components).
 */
#ifndef GMMSP_CONN_H
#define GMMSP_CONN_H

#include <stdint.h>

#include "gmmsp.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    long long components;   /* 4-connected components of the input */
    long long small;        /* of them below the size threshold */
    long long merged;       /* merges made */
} gmmsp_conn_stats;

/* labels_dev: W H int32 labels (device, row-major), rewritten in place;
 * lab_planes_dev: the image's CIELAB as three float32 planes (L, a, b) of
 * W H values (device; e.g. gmmsp_get_lab's layout transposed, or a batch's
 * planes); K: the number of superpixels the labels come from (the desired
 * size is W H / K).  Allocates its scratch (about 90 bytes per pixel), works
 * on `stream` (cudaStream_t, NULL = legacy default) and synchronises.
 * stats_host may be NULL.  GMMSP_E_TIMEOUT if a bounded device-side loop ran
 * out (the labels are then unspecified). */
gmmsp_status gmmsp_enforce_connectivity(int32_t *labels_dev, const float *lab_planes_dev, int W, int H, int K,
                                        gmmsp_conn_stats *stats_host, void *stream);

/* The same on a context's current labels (after gmmsp_labels or
 * gmmsp_segment into labels_dev), with the context's CIELAB image and K. */
gmmsp_status gmmsp_connectivity(gmmsp_ctx c, int32_t *labels_dev, gmmsp_conn_stats *stats_host);

/* The same on every image of a batch (labels_dev[i] as given to
 * gmmsp_batch_segment), with the batch's CIELAB planes; stats_host (may be
 * NULL) receives the totals over the images.  Synchronises. */
gmmsp_status gmmsp_batch_connectivity(gmmsp_batch b, int32_t *const *labels_dev, gmmsp_conn_stats *stats_host);

#ifdef __cplusplus
}
#endif

#endif /* GMMSP_CONN_H */
