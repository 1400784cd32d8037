"""CUDA path vs the FP64 oracle on the same seeded inputs, through the C ABI.

Both sides get the same FP32 CIELAB image (the oracle's FP64 conversion
rounded to FP32), so the EM comparison does not mix in colour-conversion
error; the on-device conversion is compared separately.
"""
import numpy as np
import pytest

import oracle
from synth import voronoi_image
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    torch.cuda.set_device(0)
    return gm


def lab_input(W, H, regions, sigma, seed):
    img = voronoi_image(W, H, regions, sigma, seed)
    return img, oracle.rgb2lab(img).astype(np.float32)


def run_gpu(gm, lab32, K=0, spacing=0, T=10, precision=0, wpc=None):
    import torch
    dev = torch.from_numpy(lab32).cuda()
    sp = gm.Superpixels(dev, K=K, spacing=spacing, precision=precision)
    if wpc is not None:
        sp.set_launch(wpc)
    ll = list(sp.em_iters(T, want_loglik=True)) if T > 0 else []
    labels, ll_last = sp.labels(want_loglik=True)
    mu, cs, cc = sp.get_params()
    stats = sp.stats()
    grid = sp.grid
    sp.close()
    return dict(labels=labels.cpu().numpy(), ll=np.array(ll + [ll_last]), mu=mu, cs=cs, cc=cc,
                stats=stats, grid=grid)


CASES = [
    # W, H, regions, sigma, seed, K, spacing, T
    (16, 16, 3, 8.0, 1, 0, 4, 3),
    (16, 16, 3, 8.0, 2, 0, 5, 3),
    (37, 23, 4, 8.0, 3, 0, 6, 5),       # remainders in x and y
    (70, 52, 6, 8.0, 4, 0, 8, 10),
    (97, 61, 8, 8.0, 5, 0, 7, 10),      # several tiles and ragged cells
    (320, 240, 40, 8.0, 0, 0, 12, 10),  # 320x240, spacing 12 (K = 520)
    (481, 321, 150, 8.0, 0, 1000, 0, 10),  # 481x321, K = 1000 -> v = 12, K = 1040
]


@pytest.mark.parametrize("wpc", [1, 2, 4])
@pytest.mark.parametrize("W,H,R,sigma,seed,K,sp,T", CASES)
def test_em_matches_oracle(gm, W, H, R, sigma, seed, K, sp, T, wpc):
    _, lab32 = lab_input(W, H, R, sigma, seed)
    ref = oracle.em(lab32.astype(np.float64), W, H, K=K, spacing=sp, T=T)
    got = run_gpu(gm, lab32, K=K, spacing=sp, T=T, wpc=wpc)
    assert (got["grid"].v, got["grid"].nx, got["grid"].ny, got["grid"].K) == \
        (ref.grid.v, ref.grid.nx, ref.grid.ny, ref.grid.K)
    np.testing.assert_allclose(got["ll"], ref.loglik, rtol=parity.LL_RTOL)
    assert parity.mean_rel_err(got["mu"], ref.theta.mu) <= parity.MEAN_TOL
    assert parity.cov_rel_err(got["cs"], ref.theta.cs) <= parity.COV_TOL
    assert parity.cov_rel_err(got["cc"], ref.theta.cc) <= parity.COV_TOL
    agree, ndiff, worst = parity.label_report(got["labels"], ref.labels, ref.margin)
    assert agree >= parity.LABEL_AGREE, (agree, ndiff, worst)
    assert worst < parity.MARGIN_TOL, (agree, ndiff, worst)
    assert got["stats"][0] == ref.dead
    # every label lies in the pixel's candidate set
    cand, ncand = oracle.candidates(ref.grid)
    lab = got["labels"].ravel()
    ok = ((cand == lab[:, None]) & (np.arange(9)[None, :] < ncand[:, None])).any(1)
    assert ok.all()


def test_initial_labels_and_loglik(gm):
    # T = 0: labels and L(theta_0) straight from the initialisation
    _, lab32 = lab_input(320, 240, 40, 8.0, 7)
    ref = oracle.em(lab32.astype(np.float64), 320, 240, spacing=12, T=0)
    got = run_gpu(gm, lab32, spacing=12, T=0)
    np.testing.assert_allclose(got["ll"], ref.loglik, rtol=parity.LL_RTOL)
    np.testing.assert_array_equal(got["mu"], ref.theta.mu)
    agree, ndiff, worst = parity.label_report(got["labels"], ref.labels, ref.margin)
    assert agree >= parity.LABEL_AGREE and worst < parity.MARGIN_TOL, (agree, ndiff, worst)


def test_label_pass_on_oracle_theta(gm):
    # The label kernel alone: give it the oracle's theta_T, compare with the
    # oracle's labels from the same theta.
    import torch
    W, H = 481, 321
    _, lab32 = lab_input(W, H, 150, 8.0, 11)
    ref = oracle.em(lab32.astype(np.float64), W, H, K=1000, T=10)
    dev = torch.from_numpy(lab32).cuda()
    sp = gm.Superpixels(dev, K=1000)
    sp.set_params(ref.theta.mu, ref.theta.cs, ref.theta.cc)
    labels, ll = sp.labels(want_loglik=True)
    sp.close()
    agree, ndiff, worst = parity.label_report(labels.cpu().numpy(), ref.labels, ref.margin)
    assert agree >= 0.9999 and worst < parity.MARGIN_TOL, (agree, ndiff, worst)
    np.testing.assert_allclose(ll, ref.loglik[-1], rtol=parity.LL_RTOL)


def test_rgb2lab_on_device(gm):
    import torch
    img = voronoi_image(123, 77, 9, 8.0, seed=5)
    ref = oracle.rgb2lab(img)
    sp = gm.Superpixels(torch.from_numpy(img).cuda(), spacing=8)
    lab = sp.get_lab()
    sp.close()
    assert np.max(np.abs(lab - ref)) < 1e-3
    allc = np.stack(np.meshgrid(np.arange(0, 256, 5), np.arange(0, 256, 5), np.arange(0, 256, 5)), -1)
    allc = allc.reshape(52, -1, 3).astype(np.uint8)
    sp = gm.Superpixels(torch.from_numpy(np.ascontiguousarray(allc)).cuda(), spacing=8)
    lab = sp.get_lab()
    sp.close()
    assert np.max(np.abs(lab - oracle.rgb2lab(allc))) < 1e-3


def test_rgb_input_end_to_end(gm):
    # RGB8 in, labels out, against the oracle on its own FP64 conversion.
    import torch
    W, H = 320, 240
    img = voronoi_image(W, H, 40, 8.0, seed=0)
    ref = oracle.em(oracle.rgb2lab(img), W, H, spacing=12, T=10)
    sp = gm.Superpixels(torch.from_numpy(img).cuda(), spacing=12)
    sp.em_iters(10)
    labels = sp.labels().cpu().numpy()
    mu, cs, cc = sp.get_params()
    sp.close()
    assert (labels == ref.labels).mean() >= parity.LABEL_AGREE
    assert parity.mean_rel_err(mu, ref.theta.mu) <= 1e-3


def test_segment_graph_equals_stepwise(gm):
    import torch
    W, H = 481, 321
    img = torch.from_numpy(voronoi_image(W, H, 150, 8.0, seed=2)).cuda()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a = gm.Superpixels(img, K=1000, stream=stream)
        a.em_iters(10)
        la, lla = a.labels(want_loglik=True)
        out = torch.empty((H, W), dtype=torch.int32, device="cuda")
        for _ in range(3):  # first call captures, later calls replay
            lb, llb = a.segment(img, iters=10, out=out, want_loglik=True)
        stream.synchronize()
    torch.testing.assert_close(la, lb, rtol=0, atol=0)
    assert llb[-1] == lla
    a.close()


def test_resume_equals_uninterrupted(gm):
    import torch
    _, lab32 = lab_input(320, 240, 40, 8.0, 3)
    dev = torch.from_numpy(lab32).cuda()
    a = gm.Superpixels(dev, spacing=12)
    a.em_iters(10)
    la = a.labels()
    mu_a = a.get_params()[0]
    b = gm.Superpixels(dev, spacing=12)
    b.em_iters(5)
    saved = b.get_params()
    c = gm.Superpixels(dev, spacing=12)
    c.set_params(*saved)
    c.em_iters(5)
    lc = c.labels()
    np.testing.assert_array_equal(mu_a, c.get_params()[0])
    torch.testing.assert_close(la, lc, rtol=0, atol=0)
    for s in (a, b, c):
        s.close()


def test_loglik_non_decreasing(gm):
    _, lab32 = lab_input(481, 321, 150, 8.0, 21)
    got = run_gpu(gm, lab32, K=1000, T=10)
    d = np.diff(got["ll"])
    assert np.all(d >= -1e-6 * np.abs(got["ll"][1:])), got["ll"]


def test_fp32_variant_error_is_reported(gm):
    # All-FP32 arithmetic with raw moments: it still runs and its error
    # against the oracle is larger than the mixed path's but bounded.
    W, H = 481, 321
    _, lab32 = lab_input(W, H, 150, 8.0, 0)
    ref = oracle.em(lab32.astype(np.float64), W, H, K=1000, T=10)
    mixed = run_gpu(gm, lab32, K=1000, T=10, precision=0)
    fp32 = run_gpu(gm, lab32, K=1000, T=10, precision=1)
    e_mixed = parity.cov_rel_err(mixed["cs"], ref.theta.cs)
    e_fp32 = parity.cov_rel_err(fp32["cs"], ref.theta.cs)
    assert e_mixed <= parity.COV_TOL
    assert e_fp32 < 0.5
    assert (fp32["labels"] == ref.labels).mean() > 0.95


def test_autotune_and_kernel_timing(gm):
    import torch
    W, H = 481, 321
    img = torch.from_numpy(voronoi_image(W, H, 150, 8.0, seed=4)).cuda()
    sp = gm.Superpixels(img, K=1000)
    sp.em_iters(2)
    before = sp.get_params()
    best, times = sp.autotune(reps=3)
    assert best in (1, 2, 4) and sp.get_launch() == best
    assert all(t > 0 for t in times.values())
    labels = torch.empty((H, W), dtype=torch.int32, device="cuda")
    for which in (gm.GMMSP_KERNEL_EM_PASS, gm.GMMSP_KERNEL_FINALIZE, gm.GMMSP_KERNEL_LABELS):
        assert sp.profile_kernel(which, reps=3, labels=labels) > 0
    after = sp.get_params()  # timing leaves theta as it was
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)
    sp.close()


def test_nonfinite_input_is_reported(gm):
    import torch
    lab = np.zeros((32, 32, 3), dtype=np.float32)
    lab[5, 7, 1] = np.nan
    sp = gm.Superpixels(torch.from_numpy(lab).cuda(), spacing=8)
    with pytest.raises(gm.GmmspError) as ei:
        sp.em_iters(2, want_loglik=True)
    assert ei.value.status == 4
    with pytest.raises(gm.GmmspError) as ei:
        sp.em_iters(1)
    assert ei.value.status == 6  # sticky until reinit
    sp.reinit(torch.zeros((32, 32, 3), dtype=torch.float32, device="cuda"))
    sp.em_iters(1, want_loglik=True)
    sp.close()


def test_allocation_failure_injection(gm, monkeypatch):
    import torch
    monkeypatch.setenv("GMMSP_FAIL_ALLOC", "1")
    with pytest.raises(gm.GmmspError) as ei:
        gm.Superpixels(torch.zeros((32, 32, 3), dtype=torch.uint8, device="cuda"), spacing=8)
    assert ei.value.status == 3


@pytest.mark.slow
def test_4k_matches_oracle(gm):
    # 3840x2160, K = 20000 -> v = 20, K = 20736: the full-size single-image workload.
    W, H = 3840, 2160
    _, lab32 = lab_input(W, H, 2000, 6.0, 0)
    ref = oracle.em(lab32.astype(np.float64), W, H, K=20000, T=10)
    got = run_gpu(gm, lab32, K=20000, T=10)
    np.testing.assert_allclose(got["ll"], ref.loglik, rtol=parity.LL_RTOL)
    assert parity.mean_rel_err(got["mu"], ref.theta.mu) <= parity.MEAN_TOL
    assert parity.cov_rel_err(got["cs"], ref.theta.cs) <= parity.COV_TOL
    assert parity.cov_rel_err(got["cc"], ref.theta.cc) <= parity.COV_TOL
    agree, ndiff, worst = parity.label_report(got["labels"], ref.labels, ref.margin)
    assert agree >= parity.LABEL_AGREE and worst < parity.MARGIN_TOL, (agree, ndiff, worst)


@pytest.mark.parametrize("colour", ["full", "split", "gray"])
@pytest.mark.parametrize("W,H,R,seed,K,sp", [(37, 23, 4, 3, 0, 6), (97, 61, 8, 5, 0, 7), (481, 321, 150, 7, 0, 15),
                                             (320, 240, 40, 8, 0, 12)])
def test_argmax_only_labels_equal_full_scan(gm, colour, W, H, R, seed, K, sp):
    """Without a log-likelihood the label pass skips candidates whose spatial bound
    cannot reach the best value; its labels must equal those of the full scan."""
    import torch
    _, lab32 = lab_input(W, H, R, 8.0, seed)
    ctx = gm.Superpixels(torch.from_numpy(lab32).cuda(), K=K, spacing=sp, colour=colour)
    for t in (0, 2, 5):
        if t:
            ctx.em_iters(t - (0 if t == 2 else 2))
        full, _ = ctx.labels(want_loglik=True)
        fast = ctx.labels()
        torch.testing.assert_close(fast, full, rtol=0, atol=0)
    ctx.close()
    # and in a batch of uneven sizes
    imgs = [torch.from_numpy(lab_input(w, h, max(4, w * h // 1000), 8.0, 40 + i)[1]).cuda()
            for i, (w, h) in enumerate([(W, H), (160, 120), (W, H)])]
    bt = gm.SuperpixelsBatch([(x.shape[0], x.shape[1]) for x in imgs], spacing=sp or 12, lab_input=True,
                             colour=colour)
    a = [x.clone() for x in bt.segment(imgs, iters=3)]
    b, _ = bt.segment(imgs, iters=3, want_loglik=True)
    for x, y in zip(a, b):
        torch.testing.assert_close(x, y, rtol=0, atol=0)
    bt.close()
