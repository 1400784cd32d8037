"""Pins of the accuracy-metric oracle (oracle/metrics.py)."""
import numpy as np
import pytest

from oracle import metrics as om


def test_boundary_map_hand_computed():
    L = np.array([[0, 0, 1],
                  [0, 0, 1],
                  [2, 2, 2]])
    expect = np.array([[0, 1, 1],
                       [1, 1, 1],
                       [1, 1, 1]], dtype=bool)
    np.testing.assert_array_equal(om.boundary_map(L), expect)
    assert not om.boundary_map(np.zeros((4, 5))).any()


def test_hand_computed_metrics():
    # 4 x 4 image; ground truth: left half 0, right half 1.
    gt = np.array([[0, 0, 1, 1]] * 4)
    # superpixels: k=0 covers columns 0-2 of rows 0-1 (leaks 2 pixels into g=1),
    # k=1 the rest of rows 0-1, k=2 rows 2-3.
    L = np.array([[0, 0, 0, 1],
                  [0, 0, 0, 1],
                  [2, 2, 2, 2],
                  [2, 2, 2, 2]])
    N = 16
    # overlaps: (0,0)=4 (0,1)=2 (1,1)=2 (2,0)=4 (2,1)=4; sizes 6, 2, 8
    # ASA = (4 + 2 + 4) / 16
    asa, acc = om.achievable_segmentation_accuracy(L, gt)
    assert acc == 10 and asa == pytest.approx(10 / 16)
    # UE with eps = 0.05: every pair qualifies (2 > 0.3, 4 > 0.4) -> 6 + 6 + 2 + 8 + 8 = 30
    ue, acc = om.undersegmentation_error(L, gt, 0.05)
    assert acc == 30 and ue == pytest.approx(30 / N - 1)
    # eps = 0.4: (0,1): 2 > 2.4? no; (2,0): 4 > 3.2 yes -> 6 + 2 + 8 + 8 = 24
    assert om.undersegmentation_error(L, gt, 0.4)[1] == 24
    # BR: the gt boundary pixels are columns 1 and 2 (8 pixels); superpixel boundary pixels are
    # columns 2-3 of rows 0-1 and rows 1-2 entirely; radius 0: gt boundary pixels that are also
    # superpixel boundary pixels: column 2 rows 0-1, columns 1-2 rows 1-2 -> (0,2),(1,1),(1,2),(2,1),(2,2)
    br0, rec, tot = om.boundary_recall(L, gt, radius=0)
    assert tot == 8 and rec == 5
    br2, rec, tot = om.boundary_recall(L, gt, radius=2)
    assert rec == 8 and br2 == 1.0


def test_identities():
    rng = np.random.default_rng(0)
    gt = rng.integers(0, 5, (20, 30))
    m = om.all_metrics(gt, gt)
    assert m["br"] == 1.0 and m["ue"] == 0.0 and m["asa"] == 1.0
    # one superpixel over everything: ASA = largest segment / N, UE = (#segments with >5% ) - 1
    one = np.zeros_like(gt)
    sizes = np.bincount(gt.ravel())
    m = om.all_metrics(one, gt)
    assert m["asa"] == pytest.approx(sizes.max() / gt.size)
    assert m["ue"] == pytest.approx((sizes > 0.05 * gt.size).sum() - 1)
    assert m["br"] == 0.0


def test_brute_force_random_maps():
    rng = np.random.default_rng(1)
    L = rng.integers(0, 7, (12, 9))
    gt = rng.integers(0, 4, (12, 9))
    # overlap counts by brute force over pixels
    tab = {}
    for k, g in zip(L.ravel(), gt.ravel()):
        tab[(k, g)] = tab.get((k, g), 0) + 1
    assert tab == om.overlap_table(L, gt)
    # boundary recall by brute force over pixel pairs
    H, W = L.shape
    def bnd(M, y, x):
        return any(0 <= y + dy < H and 0 <= x + dx < W and M[y + dy, x + dx] != M[y, x]
                   for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)))
    rec = tot = 0
    for y in range(H):
        for x in range(W):
            if bnd(gt, y, x):
                tot += 1
                rec += any(bnd(L, yy, xx) for yy in range(max(0, y - 2), min(H, y + 3))
                           for xx in range(max(0, x - 2), min(W, x + 3)))
    _, r, t = om.boundary_recall(L, gt, 2)
    assert (r, t) == (rec, tot)
