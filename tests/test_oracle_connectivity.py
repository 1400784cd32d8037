"""Pins of the connectivity post-processing oracle (oracle/connectivity.py)."""
import numpy as np
import pytest

from oracle import connectivity as oc


def test_components_match_scipy():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    L = rng.integers(0, 4, (23, 31))
    comp = oc.components(L)
    # same partition as scipy's 4-connected labelling of each label value
    for v in range(4):
        lab, n = ndimage.label(L == v)
        for c in range(1, n + 1):
            ids = np.unique(comp[lab == c])
            assert len(ids) == 1                        # one component ...
            assert (comp == ids[0]).sum() == (lab == c).sum()   # ... and all of it
            assert ids[0] == np.flatnonzero((lab == c).ravel())[0]  # id = smallest pixel index


def test_island_goes_to_the_nearer_colour():
    # two big superpixels (left red-ish, right blue-ish); a 2-pixel island of label 5
    # inside the right one but touching the left: it goes to the nearer colour.
    H, W = 10, 10
    L = np.zeros((H, W), dtype=np.int64)
    L[:, 5:] = 1
    L[4, 5:7] = 5
    lab = np.zeros((H, W, 3), dtype=np.float32)
    lab[:, :5] = (50, 40, 0)
    lab[:, 5:] = (50, -40, 0)
    lab[4, 5:7] = (50, 30, 0)                    # nearer to the left colour
    out, st = oc.enforce_connectivity(L, lab, K=2)
    assert st["components"] == 3 and st["small"] == 1 and st["merged"] == 1
    assert (out[4, 5:7] == 0).all()
    np.testing.assert_array_equal(np.delete(out.ravel(), [45, 46]), np.delete(L.ravel(), [45, 46]))
    lab[4, 5:7] = (50, -30, 0)                   # now nearer to the right colour
    out, _ = oc.enforce_connectivity(L, lab, K=2)
    assert (out[4, 5:7] == 1).all()


def test_size_updating_and_chain_order():
    # a row of 1-pixel components 2, 3 inside a big superpixel 0; 2 (index 21) is
    # processed before 3 (index 22): 2 merges into 3 (nearer colour) and 3, now of
    # size 2 and still small, merges into 0 -> both become 0.
    H, W = 8, 8
    L = np.zeros((H, W), dtype=np.int64)
    L[2, 5] = 2
    L[2, 6] = 3
    lab = np.zeros((H, W, 3), dtype=np.float32)
    lab[...] = (20, 0, 0)
    lab[2, 5] = (80, 0, 0)
    lab[2, 6] = (79, 0, 0)
    out, st = oc.enforce_connectivity(L, lab, K=4)       # threshold: 4 K |c| < 64 -> |c| < 4
    assert st["merged"] == 2
    assert (out == 0).all()
    # with K = 32 the threshold is |c| < 0.5: nothing is small
    out, st = oc.enforce_connectivity(L, lab, K=32)
    assert st["small"] == 0 and (out == L).all()


def test_invariants_on_noisy_labels():
    rng = np.random.default_rng(3)
    H, W, K = 40, 50, 20
    base = (np.arange(W)[None, :] // 10) + 5 * (np.arange(H)[:, None] // 8)
    L = base.copy()
    noise = rng.random((H, W)) < 0.08
    L[noise] = rng.integers(0, 25, noise.sum())
    lab = rng.normal(50, 10, (H, W, 3)).astype(np.float32)
    out, st = oc.enforce_connectivity(L, lab, K)
    N = H * W
    assert st["merged"] > 0
    # every component of the output that is below the threshold has no neighbour
    comp = oc.components(out)
    ids, sizes = np.unique(comp, return_counts=True)
    for i, sz in zip(ids, sizes):
        if 4 * K * sz < N:
            mask = comp == i
            nb = np.zeros_like(mask)
            nb[:, 1:] |= mask[:, :-1]; nb[:, :-1] |= mask[:, 1:]
            nb[1:, :] |= mask[:-1, :]; nb[:-1, :] |= mask[1:, :]
            assert not (nb & ~mask).any(), "a small component with a neighbour survived"
    # large components of the input keep their pixels' labels
    comp_in = oc.components(L)
    ids, sizes = np.unique(comp_in, return_counts=True)
    large = ids[4 * K * sizes >= N]
    keep = np.isin(comp_in, large)
    np.testing.assert_array_equal(out[keep], L[keep])
