"""The split (Eq. BlockSigma1) and grayscale colour models on the GPU against the oracle.

Both sides take the same FP32 CIELAB input (grayscale reads its L channel
only); the grey-level conversion is compared separately.  Same parity bar as
the full model (tests/parity.py).
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


def lab32_of(W, H, regions, seed):
    return oracle.rgb2lab(voronoi_image(W, H, regions, 8.0, seed)).astype(np.float32)


def check_parity(got, ref, colour):
    np.testing.assert_allclose(got["ll"], ref.loglik, rtol=parity.LL_RTOL)
    assert parity.mean_rel_err(got["mu"], ref.theta.mu) <= parity.MEAN_TOL
    assert parity.cov_rel_err(got["cs"], ref.theta.cs) <= parity.COV_TOL
    assert parity.cov_rel_err(got["cc"], ref.theta.cc) <= parity.COV_TOL
    agree, ndiff, worst = parity.label_report(got["labels"], ref.labels, ref.margin)
    assert agree >= parity.LABEL_AGREE, (agree, ndiff, worst)
    assert worst < parity.MARGIN_TOL, (agree, ndiff, worst)
    # the entries a model does not have are exactly zero
    assert np.all(got["cc"][:, 1:3] == 0.0)
    if colour == "gray":
        assert np.all(got["mu"][:, 3:] == 0.0) and np.all(got["cc"][:, 3:] == 0.0)


def run_single(gm, lab32, colour, K=0, spacing=0, T=10, wpc=None):
    import torch
    sp = gm.Superpixels(torch.from_numpy(lab32).cuda(), K=K, spacing=spacing, colour=colour)
    if wpc is not None:
        sp.set_launch(wpc)
    ll = list(sp.em_iters(T, want_loglik=True)) if T > 0 else []
    labels, ll_last = sp.labels(want_loglik=True)
    mu, cs, cc = sp.get_params()
    dead = sp.stats()[0]
    sp.close()
    return dict(labels=labels.cpu().numpy(), ll=np.array(ll + [ll_last]), mu=mu, cs=cs, cc=cc, dead=dead)


CASES = [
    # W, H, regions, seed, K, spacing, T
    (16, 16, 3, 1, 0, 4, 3),
    (37, 23, 4, 3, 0, 6, 5),          # remainders in x and y
    (97, 61, 8, 5, 0, 7, 10),         # several tiles and ragged cells
    (320, 240, 40, 0, 0, 12, 10),     # 320x240 at spacing 12
    (481, 321, 150, 0, 1000, 0, 10),  # 481x321, K = 1000 -> v = 12, K = 1040
]


@pytest.mark.parametrize("colour", ["split", "gray"])
@pytest.mark.parametrize("W,H,R,seed,K,sp,T", CASES)
def test_single_image_matches_oracle(gm, colour, W, H, R, seed, K, sp, T):
    lab32 = lab32_of(W, H, R, seed)
    ref = oracle.em(lab32.astype(np.float64), W, H, K=K, spacing=sp, T=T, colour=colour)
    for wpc in (1, 4):
        got = run_single(gm, lab32, colour, K=K, spacing=sp, T=T, wpc=wpc)
        check_parity(got, ref, colour)
        assert got["dead"] == ref.dead


@pytest.mark.parametrize("colour", ["split", "gray"])
def test_batch_matches_oracle_and_replays(gm, colour):
    import torch
    sizes = [(320, 240), (481, 321), (97, 61)]
    labs = [lab32_of(W, H, max(4, W * H // 1000), 30 + i) for i, (W, H) in enumerate(sizes)]
    imgs = [torch.from_numpy(x).cuda() for x in labs]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bt = gm.SuperpixelsBatch([(H, W) for (W, H) in sizes], spacing=12, lab_input=True, colour=colour,
                                 stream=stream)
        bt.autotune(imgs, reps=1)
        labels, ll = bt.segment(imgs, iters=10, want_loglik=True)
        first = [x.clone() for x in labels]
        again = bt.segment(imgs, iters=10)                # graph replay
    stream.synchronize()
    for i, (W, H) in enumerate(sizes):
        torch.testing.assert_close(first[i], again[i], rtol=0, atol=0)
        ref = oracle.em(labs[i].astype(np.float64), W, H, spacing=12, T=10, colour=colour)
        K = ref.grid.K
        mu, cs, cc = bt.get_params(i, K)
        got = dict(labels=first[i].cpu().numpy(), ll=np.array([ll[i]]), mu=mu, cs=cs, cc=cc)
        ref.loglik = ref.loglik[-1:]
        check_parity(got, ref, colour)
    bt.close()


def test_models_agree_on_zero_ab_images(gm):
    # a = b = 0: the three models give the same labels and spatial parameters on the GPU too
    W, H = 320, 240
    lab32 = lab32_of(W, H, 40, 9)
    lab32[..., 1:] = 0.0
    runs = {c: run_single(gm, lab32, c, spacing=12, T=10) for c in ("full", "split", "gray")}
    for c in ("split", "gray"):
        assert (runs[c]["labels"] == runs["full"]["labels"]).mean() >= 0.9999
        assert parity.mean_rel_err(runs[c]["mu"][:, :3], runs["full"]["mu"][:, :3]) <= 1e-5
        assert parity.cov_rel_err(runs[c]["cs"], runs["full"]["cs"]) <= 1e-5
    N = W * H
    np.testing.assert_allclose(runs["gray"]["ll"][1:] - runs["full"]["ll"][1:], N * np.log(2 * np.pi * 8.0),
                               rtol=1e-5)


def test_gray_levels_conversion_and_end_to_end(gm):
    import torch
    W, H = 481, 321
    g8 = voronoi_image(W, H, 150, 8.0, 12)[..., 1].copy()          # one channel as grey levels
    ref_L = oracle.gray2l(g8)
    sp = gm.Superpixels(torch.from_numpy(g8).cuda(), spacing=15, colour="gray")
    lab = sp.get_lab()                                             # (H, W, 3) float32
    L = lab[..., 0]
    assert np.all(lab[..., 1:] == 0.0)                            # the a, b planes stay zero
    np.testing.assert_allclose(L, ref_L, rtol=0, atol=2e-4)
    sp.em_iters(10)
    labels = sp.labels().cpu().numpy()
    sp.close()
    # the oracle on the device's own L plane: the same EM input
    ref = oracle.em(np.stack([L, np.zeros_like(L), np.zeros_like(L)], -1).astype(np.float64), W, H,
                    spacing=15, T=10, colour="gray")
    agree, ndiff, worst = parity.label_report(labels, ref.labels, ref.margin)
    assert agree >= parity.LABEL_AGREE and worst < parity.MARGIN_TOL, (agree, ndiff, worst)
    # a batch of grey-level images gives the single context's labels
    bt = gm.SuperpixelsBatch([(H, W)] * 2, spacing=15, colour="gray", gray_input=True)
    out = bt.segment([torch.from_numpy(g8).cuda()] * 2, iters=10)
    for x in out:
        assert (x.cpu().numpy() == labels).mean() >= 0.9999
    bt.close()


def test_unsupported_combinations_raise(gm):
    import torch
    from paper_1612_08792_gb300.learned_init import InitNet, init_weights
    lab32 = torch.from_numpy(lab32_of(64, 48, 6, 1)).cuda()
    with pytest.raises(gm.GmmspError):
        gm.Superpixels(lab32, spacing=8, colour="split", precision=gm.GMMSP_PREC_FP32)
    g8 = torch.zeros((48, 64), dtype=torch.uint8, device="cuda")
    with pytest.raises(gm.GmmspError):
        gm.Superpixels(g8, spacing=8, colour="full")
    net = InitNet(15, weights=init_weights(1))
    sp = gm.Superpixels(torch.from_numpy(lab32_of(481, 321, 150, 2)).cuda(), spacing=15, colour="split")
    with pytest.raises(gm.GmmspError):
        sp.init_from_net(net)
    sp.em_iters(2)                       # the context stays usable
    sp.close()
    bt = gm.SuperpixelsBatch([(321, 481)], spacing=15, colour="gray")
    with pytest.raises(gm.GmmspError):
        bt.set_init_net(net)
    bt.close()
    net.close()
