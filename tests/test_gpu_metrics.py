"""Accuracy metrics (BR, Eq. ue, Eq. asa) on the GPU against the metric oracle: exact."""
import numpy as np
import pytest

import oracle
from oracle import metrics as om
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


def gpu_metrics(gm, labels, gt, K, G, radius=2, eps=0.05):
    import torch
    lt = torch.from_numpy(np.ascontiguousarray(labels.astype(np.int32))).cuda()
    gtt = torch.from_numpy(np.ascontiguousarray(gt.astype(np.int32))).cuda()
    return gm.gmmsp_segmentation_metrics(lt, gtt, K, G, radius, eps)


def check_equal(m, ref):
    assert m["br_recovered"] == ref["br_recovered"] and m["br_total"] == ref["br_total"]
    assert m["ue_sum"] == ref["ue_sum"] and m["asa_sum"] == ref["asa_sum"]
    assert m["br"] == ref["br"] and m["ue"] == ref["ue"] and m["asa"] == ref["asa"]


@pytest.mark.parametrize("H,W,K,G,radius,eps", [(12, 9, 7, 4, 2, 0.05), (37, 23, 50, 6, 1, 0.05),
                                                (64, 80, 300, 12, 2, 0.2), (5, 5, 3, 2, 0, 0.05)])
def test_random_maps_exact(gm, H, W, K, G, radius, eps):
    rng = np.random.default_rng(H * W)
    labels = rng.integers(0, K, (H, W))
    gt = rng.integers(0, G, (H, W))
    check_equal(gpu_metrics(gm, labels, gt, K, G, radius, eps), om.all_metrics(labels, gt, radius, eps))


def test_em_segmentation_exact(gm):
    import torch
    W, H = 481, 321
    img, reg = voronoi_image(W, H, 150, 8.0, 7, return_regions=True)
    sp = gm.Superpixels(torch.from_numpy(img).cuda(), spacing=15)
    sp.em_iters(10)
    labels = sp.labels().cpu().numpy()
    K = sp.grid.K
    sp.close()
    ref = om.all_metrics(labels, reg, 2, 0.05)
    check_equal(gpu_metrics(gm, labels, reg, K, 150), ref)
    assert 0.5 < ref["br"] <= 1.0 and 0.0 <= ref["ue"] and 0.8 < ref["asa"] <= 1.0
    # identities
    m = gpu_metrics(gm, reg, reg, 150, 150)
    assert m["br"] == 1.0 and m["ue"] == 0.0 and m["asa"] == 1.0


def test_out_of_range_is_rejected(gm):
    labels = np.zeros((8, 8), dtype=np.int32)
    labels[3, 3] = 9
    with pytest.raises(gm.GmmspError):
        gpu_metrics(gm, labels, np.zeros((8, 8), dtype=np.int32), 5, 1)


def test_many_equals_oracle_per_image(gm):
    """The batched call over images of different sizes, label counts and segment counts."""
    import torch
    rng = np.random.default_rng(5)
    cases = [(12, 9, 7, 4), (37, 23, 50, 6), (64, 80, 300, 12), (5, 5, 3, 2), (40, 33, 20, 20)]
    labels, gts, refs = [], [], []
    for H, W, K, G in cases:
        lab = rng.integers(0, K, (H, W))
        gt = rng.integers(0, G, (H, W))
        labels.append(torch.from_numpy(lab.astype(np.int32)).cuda())
        gts.append(torch.from_numpy(gt.astype(np.int32)).cuda())
        refs.append(om.all_metrics(lab, gt, 2, 0.05))
    out = gm.gmmsp_segmentation_metrics_many(labels, gts, [c[2] for c in cases], [c[3] for c in cases])
    for m, ref in zip(out, refs):
        check_equal(m, ref)
    # one image out of range fails the call
    bad = labels[1].clone()
    bad[0, 0] = 10_000
    with pytest.raises(gm.GmmspError):
        gm.gmmsp_segmentation_metrics_many([labels[0], bad], gts[:2], [cases[0][2], cases[1][2]],
                                           [cases[0][3], cases[1][3]])


def test_many_at_full_size(gm):
    """The metrics256 workload at full size, as bench.py times it: BR, UE (Eq. ue) and ASA (Eq.
    asa) of the label maps of 256 held-out 481x321 images (seeds 1,000,000 + i) after 10
    plain-EM iterations at spacing 15, against the generator's 150 regions, in one batched call.
    Maps 0, 127 and 255 equal the oracle's exactly."""
    import torch
    from synth.voronoi_torch import voronoi_batch
    n, W, H, v, G = 256, 481, 321, 15, 150
    K = (W // v) * (H // v)
    regs = torch.empty((n, H, W), dtype=torch.int32, device="cuda")
    buf = voronoi_batch(W, H, G, 8.0, range(1_000_000, 1_000_000 + n), regions_out=regs)
    bt = gm.SuperpixelsBatch([(H, W)] * n, spacing=v)
    labels = bt.segment([buf[i] for i in range(n)], iters=10)
    torch.cuda.synchronize()
    out = gm.gmmsp_segmentation_metrics_many(labels, [regs[i] for i in range(n)], K, G)
    assert len(out) == n
    for i in (0, 127, 255):
        check_equal(out[i], om.all_metrics(labels[i].cpu().numpy(), regs[i].cpu().numpy(), 2, 0.05))
    bt.close()
