"""Accuracy metrics of Sec. IV (boundary recall, Eq. ue, Eq. asa), plain numpy.

TEST INFRASTRUCTURE ONLY: used by ``tests/`` and ``bench.py``'s CPU legs,
never by the product library, and sharing no code with it.

Definitions (N pixels, superpixel pixel sets s_k, ground-truth segments s_g):
  * boundary pixel of a label map: a pixel with a 4-neighbour of another
    label (both sides of an edge are boundary pixels);
  * BR: the fraction of ground-truth boundary pixels that have a superpixel
    boundary pixel within Chebyshev distance `radius` (2 in the paper);
  * UE = (1/N) sum over pairs (k, g) with |s_k & s_g| > eps |s_k| of |s_k|,
    minus 1 (Eq. ue, eps = 0.05);
  * ASA = (1/N) sum_k max_g |s_k & s_g| (Eq. asa).
Each is computed from its definition: the overlap table by counting pixel
pairs, the boundary test by comparing every pixel with its neighbours, the
recall by scanning the window of every ground-truth boundary pixel.

Pinned by tests/test_oracle_metrics.py: hand-computed values on small label
maps, identities (labels equal to the ground truth: BR = 1, UE = 0, ASA = 1;
one superpixel: ASA = largest segment / N), and brute force over pixel pairs.
"""
from __future__ import annotations

import numpy as np


def boundary_map(labels) -> np.ndarray:
    """True where a pixel has a 4-neighbour with another label."""
    L = np.asarray(labels)
    b = np.zeros(L.shape, dtype=bool)
    d = L[:, 1:] != L[:, :-1]           # horizontal neighbours
    b[:, 1:] |= d
    b[:, :-1] |= d
    d = L[1:, :] != L[:-1, :]           # vertical neighbours
    b[1:, :] |= d
    b[:-1, :] |= d
    return b


def overlap_table(labels, gt):
    """|s_k & s_g| for every (superpixel, segment) pair that occurs: dict (k, g) -> count."""
    L = np.asarray(labels).ravel().astype(np.int64)
    G = np.asarray(gt).ravel().astype(np.int64)
    pairs, counts = np.unique(np.stack([L, G], 1), axis=0, return_counts=True)
    return {(int(k), int(g)): int(c) for (k, g), c in zip(pairs, counts)}


def boundary_recall(labels, gt, radius: int = 2):
    """(BR, recovered, total) over the ground-truth boundary pixels."""
    sb = boundary_map(labels)
    gb = boundary_map(gt)
    H, W = sb.shape
    ys, xs = np.nonzero(gb)
    rec = 0
    for y, x in zip(ys, xs):
        y0, y1 = max(0, y - radius), min(H, y + radius + 1)
        x0, x1 = max(0, x - radius), min(W, x + radius + 1)
        rec += bool(sb[y0:y1, x0:x1].any())
    total = len(ys)
    return (rec / total if total else 1.0), rec, total


def undersegmentation_error(labels, gt, eps: float = 0.05):
    """(UE, sum of |s_k| over the qualifying pairs)."""
    tab = overlap_table(labels, gt)
    size = {}
    for (k, _), c in tab.items():
        size[k] = size.get(k, 0) + c
    acc = sum(size[k] for (k, _), c in tab.items() if c > eps * size[k])
    N = np.asarray(labels).size
    return acc / N - 1.0, acc


def achievable_segmentation_accuracy(labels, gt):
    """(ASA, sum over k of the largest overlap)."""
    tab = overlap_table(labels, gt)
    best = {}
    for (k, _), c in tab.items():
        best[k] = max(best.get(k, 0), c)
    acc = sum(best.values())
    return acc / np.asarray(labels).size, acc


def all_metrics(labels, gt, radius: int = 2, eps: float = 0.05):
    br, rec, tot = boundary_recall(labels, gt, radius)
    ue, ue_acc = undersegmentation_error(labels, gt, eps)
    asa, asa_acc = achievable_segmentation_accuracy(labels, gt)
    return dict(br=br, ue=ue, asa=asa, br_recovered=rec, br_total=tot, ue_sum=ue_acc, asa_sum=asa_acc)
