"""Batched segmentation (gmmsp_batch_*) against the single-image path and the oracle."""
import numpy as np
import pytest

import oracle
from synth import voronoi_image
from synth.voronoi import batch_regions
from tests import parity

pytestmark = pytest.mark.gpu

SIZES = [(37, 23), (320, 240), (70, 52), (481, 321), (97, 61), (150, 110)]


@pytest.fixture(scope="module")
def gm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    torch.cuda.set_device(0)
    return gm


def make_labs(sizes, seed0=100):
    labs = []
    for i, (W, H) in enumerate(sizes):
        img = voronoi_image(W, H, batch_regions(W, H), 8.0, seed0 + i)
        labs.append(oracle.rgb2lab(img).astype(np.float32))
    return labs


def test_batch_matches_single_images_and_oracle(gm):
    import torch
    spacing, T = 8, 10
    labs = make_labs(SIZES)
    dev = [torch.from_numpy(x).cuda() for x in labs]
    bt = gm.SuperpixelsBatch([(H, W) for (W, H) in SIZES], spacing=spacing, lab_input=True)
    labels, ll = bt.segment(dev, iters=T, want_loglik=True)
    torch.cuda.synchronize()
    for i, (W, H) in enumerate(SIZES):
        sp = gm.Superpixels(dev[i], spacing=spacing)
        sp.set_launch(1)
        sp.em_iters(T)
        ref_labels, ref_ll = sp.labels(want_loglik=True)
        mu_s, cs_s, cc_s = sp.get_params()
        K = sp.grid.K
        sp.close()
        mu_b, cs_b, cc_b = bt.get_params(i, K)
        assert parity.mean_rel_err(mu_b, mu_s) < 1e-6
        assert parity.cov_rel_err(cc_b, cc_s) < 1e-6
        agree = (labels[i].cpu().numpy() == ref_labels.cpu().numpy()).mean()
        assert agree >= 0.9999, (i, agree)
        assert abs(ll[i] - ref_ll) <= 1e-6 * abs(ref_ll)
        if i in (0, 3):  # and against the oracle
            ref = oracle.em(labs[i].astype(np.float64), W, H, spacing=spacing, T=T)
            assert parity.mean_rel_err(mu_b, ref.theta.mu) <= parity.MEAN_TOL
            assert parity.cov_rel_err(cc_b, ref.theta.cc) <= parity.COV_TOL
            a, nd, worst = parity.label_report(labels[i].cpu().numpy(), ref.labels, ref.margin)
            assert a >= parity.LABEL_AGREE and worst < parity.MARGIN_TOL, (a, nd, worst)
    bt.close()


def test_batch_rgb_input_graph_replay_and_autotune(gm):
    import torch
    sizes = [(320, 240), (481, 321), (640, 480), (320, 240)]
    imgs = [torch.from_numpy(voronoi_image(W, H, batch_regions(W, H), 8.0, 7 + i)).cuda()
            for i, (W, H) in enumerate(sizes)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bt = gm.SuperpixelsBatch([(H, W) for (W, H) in sizes], spacing=15, stream=stream)
        best, times = bt.autotune(imgs, reps=2)
        assert best in times and all(t > 0 for t in times.values())
        first = [x.clone() for x in bt.segment(imgs, iters=10)]   # captures
        again, ll = bt.segment(imgs, iters=10, want_loglik=True)  # replays (new capture for ll)
        third = bt.segment(imgs, iters=10)                         # replays
        stream.synchronize()
    for a, b, c in zip(first, again, third):
        torch.testing.assert_close(a, b, rtol=0, atol=0)
        torch.testing.assert_close(a, c, rtol=0, atol=0)
    pix, K, cells = bt.info()
    assert pix == sum(W * H for W, H in sizes)
    assert np.all(np.isfinite(ll))
    # single-image RGB path on the third image
    sp = gm.Superpixels(imgs[2], spacing=15)
    sp.set_launch(1)
    sp.em_iters(10)
    ref = sp.labels().cpu().numpy()
    sp.close()
    assert (third[2].cpu().numpy() == ref).mean() >= 0.9999
    bt.close()


def test_batch_rejects_bad_arguments(gm):
    p = gm.gmmsp_default_params()
    p.spacing = 12
    with pytest.raises(gm.GmmspError):
        gm.gmmsp_batch_create([320, 5], [240, 5], p)  # second image smaller than the spacing


def test_tuning_cache_applies_stored_choices(gm, tmp_path):
    import torch
    from synth.voronoi_torch import voronoi_batch
    path = str(tmp_path / "tuning.json")
    buf = voronoi_batch(481, 321, 150, 8.0, [1, 2, 3, 4])
    imgs = [buf[i] for i in range(4)]
    a = gm.SuperpixelsBatch([(321, 481)] * 4, spacing=15)
    best, times = a.autotune(imgs, reps=1, cache=path)
    ref = [x.clone() for x in a.segment(imgs, iters=3)]
    tun = a.tuning()
    a.close()
    b = gm.SuperpixelsBatch([(321, 481)] * 4, spacing=15)
    b.set_launch(3 if best != 3 else 4)
    best2, times2 = b.autotune(imgs, reps=1, cache=path)      # served from the cache
    assert best2 == best and times2 == times
    assert b.tuning()["blocks_per_sm"] == tun["blocks_per_sm"]
    assert b.tuning()["finalize16"] == tun["finalize16"]
    assert b.tuning()["first_pass_blocks_per_sm"] == tun["first_pass_blocks_per_sm"]
    for x, y in zip(b.segment(imgs, iters=3), ref):
        assert (x.cpu().numpy() == y.cpu().numpy()).mean() >= 0.9999
    b.close()


@pytest.mark.parametrize("start,colour", [("plain", "full"), ("plain", "split"), ("plain", "gray"),
                                          ("learned", "full")])
def test_first_pass_diagonal_kernel_equals_general(gm, start, colour):
    """Both starts give axis-aligned covariances, so the first E + M pass runs a kernel that leaves
    the zero off-diagonal terms out. Its per-cell partials must equal the general kernel's (value
    for value), at both launch choices of the one-cell-per-warp kernel (Eq. Rik, UpdateMu,
    UpdateSigS/C)."""
    import torch
    from synth.voronoi_torch import voronoi_batch
    n, H, W = 6, 321, 481
    buf = voronoi_batch(W, H, 150, 8.0, list(range(40, 40 + n)))
    imgs = [buf[i] for i in range(n)]
    bt = gm.SuperpixelsBatch([(H, W)] * n, spacing=15, colour=colour)
    if start == "learned":
        from paper_1612_08792_gb300.learned_init import load_pretrained
        bt.set_init_net(load_pretrained(15))
    for bps in (6, 7):
        gen = bt.first_pass_partials(imgs, bps, diagonal=False)
        diag = bt.first_pass_partials(imgs, bps, diagonal=True)
        assert gen.shape == (bt.info()[2], 136) and np.isfinite(gen).all()
        assert gen[:, 0:135:15].sum() > 0  # posterior weights present
        assert np.array_equal(diag, gen), (bps, int((diag != gen).sum()))
    bt.close()
    torch.cuda.synchronize()


def test_batch256_at_full_size(gm):
    """The batch256 workload at full size, as bench.py times it: 256 sRGB images of the five sizes
    320x240 ... 1920x1080 (171 Mpx), spacing 15, 10 plain-EM iterations, the autotuner's launch
    choices. Every label map: each label is one of its pixel's 3 x 3 seeds (Eq. obtLi). The first
    image of each size: theta_10, labels and L against the oracle (Algorithm 1 steps 1-7) on the
    GPU's CIELAB."""
    import torch
    from synth.voronoi import batch_sizes
    sizes = batch_sizes(256)
    cache, imgs = {}, []
    for i, (Wi, Hi) in enumerate(sizes):  # the bench's images: 4 seeded images per size, reused
        key = (Wi, Hi, i % 4)
        if key not in cache:
            cache[key] = torch.from_numpy(voronoi_image(Wi, Hi, batch_regions(Wi, Hi), 8.0, seed=i % 4)).cuda()
        imgs.append(cache[key])
    v, T = 15, 10
    bt = gm.SuperpixelsBatch([(h, w) for (w, h) in sizes], spacing=v)
    bt.autotune(imgs, reps=2)
    labels, ll = bt.segment(imgs, iters=T, want_loglik=True)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(ll))
    for i, (Wi, Hi) in enumerate(sizes):
        nx, ny = Wi // v, Hi // v
        lab_i = labels[i].long()
        ys = torch.arange(Hi, device=lab_i.device).view(Hi, 1)
        xs = torch.arange(Wi, device=lab_i.device).view(1, Wi)
        ok = (lab_i >= 0) & (lab_i < nx * ny) & ((lab_i % nx - xs // v).abs() <= 1) & \
             ((lab_i // nx - ys // v).abs() <= 1)
        assert bool(ok.all()), (i, Wi, Hi)
    for size in sorted(set(sizes)):
        i = sizes.index(size)
        Wi, Hi = size
        ref = oracle.em(bt.get_lab(i).astype(np.float64), Wi, Hi, spacing=v, T=T)
        mu, cs, cc = bt.get_params(i, (Wi // v) * (Hi // v))
        assert parity.mean_rel_err(mu, ref.theta.mu) <= parity.MEAN_TOL
        assert parity.cov_rel_err(cs, ref.theta.cs) <= parity.COV_TOL
        assert parity.cov_rel_err(cc, ref.theta.cc) <= parity.COV_TOL
        a, nd, worst = parity.label_report(labels[i].cpu().numpy(), ref.labels, ref.margin)
        assert a >= parity.LABEL_AGREE and worst < parity.MARGIN_TOL, (size, a, nd, worst)
        assert abs(ll[i] - ref.loglik[-1]) <= parity.LL_RTOL * abs(ref.loglik[-1]), (size, ll[i], ref.loglik[-1])
    bt.close()
