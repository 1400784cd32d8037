"""Connectivity post-processing (Algorithm 1, step 8) on the GPU against the oracle: exact."""
import numpy as np
import pytest

import oracle
from oracle import connectivity as oc
from synth import voronoi_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    torch.cuda.set_device(0)
    return gm


def gpu_conn(gm, labels, lab, K):
    import torch
    H, W = labels.shape
    lt = torch.from_numpy(np.ascontiguousarray(labels.astype(np.int32))).cuda()
    planes = torch.from_numpy(np.ascontiguousarray(np.asarray(lab, dtype=np.float32).transpose(2, 0, 1))).cuda()
    st = gm.gmmsp_enforce_connectivity(lt, planes, W, H, K)
    return lt.cpu().numpy(), st


def check(gm, labels, lab, K):
    ref, rst = oc.enforce_connectivity(labels, lab, K)
    out, st = gpu_conn(gm, labels, lab, K)
    assert st == rst, (st, rst)
    np.testing.assert_array_equal(out, ref)
    return st


def test_hand_cases(gm):
    H, W = 10, 10
    L = np.zeros((H, W), dtype=np.int64)
    L[:, 5:] = 1
    L[4, 5:7] = 5
    lab = np.zeros((H, W, 3), dtype=np.float32)
    lab[:, :5] = (50, 40, 0)
    lab[:, 5:] = (50, -40, 0)
    lab[4, 5:7] = (50, 30, 0)
    assert check(gm, L, lab, 2)["merged"] == 1
    L = np.zeros((8, 8), dtype=np.int64)
    L[2, 5], L[2, 6] = 2, 3
    lab = np.full((8, 8, 3), 20, dtype=np.float32)
    lab[2, 5], lab[2, 6] = (80, 0, 0), (79, 0, 0)
    assert check(gm, L, lab, 4)["merged"] == 2
    assert check(gm, L, lab, 32)["small"] == 0
    # a single label everywhere: one component, nothing to do
    assert check(gm, np.zeros((9, 7), dtype=np.int64), lab[:9, :7] if lab.shape[0] >= 9 else
                 np.zeros((9, 7, 3), dtype=np.float32), 3)["merged"] == 0


@pytest.mark.parametrize("seed,H,W,K,p", [(3, 40, 50, 20, 0.08), (4, 64, 64, 16, 0.3), (5, 97, 61, 40, 0.15),
                                          (6, 33, 200, 30, 0.5)])
def test_noisy_label_maps(gm, seed, H, W, K, p):
    rng = np.random.default_rng(seed)
    base = (np.arange(W)[None, :] * 7 // W) + 7 * (np.arange(H)[:, None] * 5 // H)
    L = base.copy()
    noise = rng.random((H, W)) < p
    L[noise] = rng.integers(0, 40, noise.sum())
    lab = rng.normal(50, 15, (H, W, 3)).astype(np.float32)
    lab[rng.random((H, W)) < 0.2] = 50.0            # exact colour ties
    check(gm, L, lab, K)


@pytest.mark.parametrize("T", [2, 10])
def test_em_output(gm, T):
    import torch
    W, H = 481, 321
    img = voronoi_image(W, H, 150, 8.0, 11)
    lab = oracle.rgb2lab(img).astype(np.float32)
    sp = gm.Superpixels(torch.from_numpy(lab).cuda(), spacing=15)
    sp.em_iters(T)
    labels = sp.labels()
    K = sp.grid.K
    ref, rst = oc.enforce_connectivity(labels.cpu().numpy(), lab, K)
    st = sp.connectivity(labels)            # the context's own CIELAB planes
    sp.close()
    assert st == rst and st["merged"] > 100
    np.testing.assert_array_equal(labels.cpu().numpy(), ref)


def test_batch_connectivity(gm):
    import torch
    sizes = [(320, 240), (481, 321), (97, 61)]
    imgs = [voronoi_image(W, H, max(4, W * H // 1000), 8.0, 20 + i) for i, (W, H) in enumerate(sizes)]
    bt = gm.SuperpixelsBatch([(H, W) for (W, H) in sizes], spacing=12)
    labels = bt.segment([torch.from_numpy(x).cuda() for x in imgs], iters=5)
    before = [x.cpu().numpy() for x in labels]
    st = bt.connectivity()
    total = {"components": 0, "small": 0, "merged": 0}
    for i, (W, H) in enumerate(sizes):
        lab = bt.get_lab(i)                 # the colours the device converted and merged on
        assert np.max(np.abs(lab - oracle.rgb2lab(imgs[i]))) < 1e-3
        ref, rst = oc.enforce_connectivity(before[i], lab, (W // 12) * (H // 12))
        np.testing.assert_array_equal(labels[i].cpu().numpy(), ref)
        for k in total:
            total[k] += rst[k]
    assert all(st[k] == total[k] for k in total), (st, total)
    bt.close()


def test_batch_connectivity_at_full_size(gm):
    """The conn256 workload at full size, as bench.py times it: the label maps of 256 held-out
    481x321 images (seeds 1,000,000 + i, 150 regions, sigma 8) after 10 plain-EM iterations at
    spacing 15, one batch call of Algorithm 1, step 8. Maps 0, 127 and 255 equal the oracle's
    on the device CIELAB; every map keeps its labels in [0, K)."""
    import torch
    from synth.voronoi_torch import voronoi_batch
    n, W, H, v = 256, 481, 321, 15
    K = (W // v) * (H // v)
    buf = voronoi_batch(W, H, 150, 8.0, range(1_000_000, 1_000_000 + n))
    bt = gm.SuperpixelsBatch([(H, W)] * n, spacing=v)
    bt.segment([buf[i] for i in range(n)], iters=10)
    torch.cuda.synchronize()
    sample = (0, 127, 255)
    before = {i: bt.labels[i].cpu().numpy() for i in sample}
    st = bt.connectivity()
    torch.cuda.synchronize()
    for i in sample:
        ref, _ = oc.enforce_connectivity(before[i], bt.get_lab(i), K)
        np.testing.assert_array_equal(bt.labels[i].cpu().numpy(), ref)
    after = torch.stack(bt.labels)
    assert bool(((after >= 0) & (after < K)).all())
    assert min(st.values()) >= 0
    bt.close()
