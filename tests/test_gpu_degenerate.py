"""Degenerate cases of the method on the GPU against the oracle: a single superpixel, a
constant image (every colour covariance at the floor), one row or one column of
superpixels, a spacing equal to the image side, and superpixels with no weight."""
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


def run(gm, lab32, spacing, T, colour="full"):
    import torch
    sp = gm.Superpixels(torch.from_numpy(np.ascontiguousarray(lab32)).cuda(), spacing=spacing, colour=colour)
    ll = list(sp.em_iters(T, want_loglik=True)) if T else []
    labels, ll_last = sp.labels(want_loglik=True)
    mu, cs, cc = sp.get_params()
    dead = sp.stats()[0]
    grid = sp.grid
    sp.close()
    return dict(labels=labels.cpu().numpy(), ll=np.array(ll + [ll_last]), mu=mu, cs=cs, cc=cc, dead=dead, grid=grid)


def check(got, ref):
    np.testing.assert_allclose(got["ll"], ref.loglik, rtol=parity.LL_RTOL)
    assert parity.mean_rel_err(got["mu"], ref.theta.mu) <= parity.MEAN_TOL
    assert parity.cov_rel_err(got["cs"], ref.theta.cs) <= parity.COV_TOL
    assert parity.cov_rel_err(got["cc"], ref.theta.cc) <= parity.COV_TOL
    agree, ndiff, worst = parity.label_report(got["labels"], ref.labels, ref.margin)
    assert agree >= parity.LABEL_AGREE and worst < parity.MARGIN_TOL, (agree, ndiff, worst)
    assert got["dead"] == ref.dead


def lab_of(W, H, regions, seed):
    return oracle.rgb2lab(voronoi_image(W, H, regions, 8.0, seed)).astype(np.float32)


@pytest.mark.parametrize("W,H,v", [(16, 16, 16), (23, 17, 17), (5, 5, 5)])
def test_single_superpixel(gm, W, H, v):
    lab32 = lab_of(W, H, 3, 1)
    ref = oracle.em(lab32.astype(np.float64), W, H, spacing=v, T=3)
    got = run(gm, lab32, v, 3)
    assert got["grid"].K == 1 and np.all(got["labels"] == 0)
    check(got, ref)


@pytest.mark.parametrize("colour", ["full", "split", "gray"])
def test_constant_image_floors_colour(gm, colour):
    W, H, v = 36, 24, 6
    lab32 = np.empty((H, W, 3), dtype=np.float32)
    lab32[...] = (50.0, 10.0, -20.0)
    ref = oracle.em(lab32.astype(np.float64), W, H, spacing=v, T=4, colour=colour)
    got = run(gm, lab32, v, 4, colour)
    check(got, ref)
    C = parity.unpack(got["cc"])
    want = 8.0 * np.eye(3) if colour != "gray" else np.diag([8.0, 0.0, 0.0])
    np.testing.assert_allclose(C, np.broadcast_to(want, C.shape), atol=1e-6)


@pytest.mark.parametrize("W,H,v", [(200, 12, 12), (12, 150, 12), (61, 13, 6)])
def test_one_row_or_column_of_superpixels(gm, W, H, v):
    lab32 = lab_of(W, H, 8, 2)
    ref = oracle.em(lab32.astype(np.float64), W, H, spacing=v, T=5)
    got = run(gm, lab32, v, 5)
    assert min(got["grid"].nx, got["grid"].ny) <= 5
    check(got, ref)


def test_superpixel_without_weight_keeps_its_parameters(gm):
    """Two colour blocks and a start whose middle Gaussian sits in neither: it loses all
    weight and keeps theta (the reading for W < 1e-8), on both sides."""
    import torch
    W, H, v = 48, 16, 16
    lab32 = np.zeros((H, W, 3), dtype=np.float32)
    lab32[:, :24] = (20.0, 0.0, 0.0)
    lab32[:, 24:] = (90.0, 0.0, 0.0)
    g = oracle.grid(W, H, spacing=v)
    th = oracle.init_theta(lab32.astype(np.float64), g)
    th.mu[1, 2:] = (55.0, 80.0, -80.0)            # far from every pixel's colour
    th.cc[1] = (1.0, 0.0, 0.0, 1.0, 0.0, 1.0)       # and narrow
    ref = oracle.em(lab32.astype(np.float64), W, H, spacing=v, T=3, theta0=th)
    sp = gm.Superpixels(torch.from_numpy(lab32).cuda(), spacing=v)
    sp.set_params(th.mu, th.cs, th.cc)
    ll = list(sp.em_iters(3, want_loglik=True))
    labels, ll_last = sp.labels(want_loglik=True)
    mu, cs, cc = sp.get_params()
    dead = sp.stats()[0]
    sp.close()
    assert ref.dead > 0 and dead == ref.dead
    np.testing.assert_allclose(mu[1], th.mu[1], rtol=1e-6)
    check(dict(labels=labels.cpu().numpy(), ll=np.array(ll + [ll_last]), mu=mu, cs=cs, cc=cc, dead=dead), ref)


@pytest.mark.parametrize("W,H,v", [(320, 240, 80), (400, 130, 120), (257, 199, 64)])
def test_large_spacing(gm, W, H, v):
    """Cells of up to 120 x 120 pixels (with remainders): candidate means staged relative to
    the processed cell reach about 2 v, and a cell's pixel loop runs hundreds of batches."""
    lab32 = lab_of(W, H, 12, 3)
    ref = oracle.em(lab32.astype(np.float64), W, H, spacing=v, T=5)
    got = run(gm, lab32, v, 5)
    assert got["grid"].K == ref.grid.K
    check(got, ref)


@pytest.mark.parametrize("v", [8, 15])
def test_nan_pixels_keep_labels_in_candidate_sets(gm, v):
    """A NaN pixel in a corner cell (no density compares) and one in the remainder corner: every label
    still names one of its pixel's candidates (Eq. Ik, obtLi), on the context and allocation-free paths,
    and the context path reports the input as GMMSP_E_NUMERIC.  At v = 15 a corner cell has 225 =
    7 x 32 + 1 pixels, and its last pixel (14, 14), taken apart from the 32-pixel batches, is NaN too."""
    import torch
    W, H, T = 97, 61, 3                             # remainder strips 1 and 5 (v = 8), 7 and 1 (v = 15)
    lab = oracle.rgb2lab(voronoi_image(W, H, 12, 8.0, 17)).astype(np.float32)
    lab[0, 0] = np.nan
    lab[H - 1, W - 1, 1] = np.nan
    if v == 15:
        lab[14, 14] = np.nan
    g = oracle.grid(W, H, spacing=v)
    cand, _ = oracle.candidates(g)

    def in_candidates(labels):
        return bool(np.all(np.any(cand == labels.reshape(-1, 1), axis=1)))

    dev = torch.from_numpy(lab).cuda()
    p = gm.gmmsp_default_params()
    p.spacing = v
    out = torch.full((H, W), -1, dtype=torch.int32, device="cuda")
    gm.gmmsp_segment_lab_noalloc(dev, W, H, W * 12, p, T, out)
    torch.cuda.synchronize()
    assert in_candidates(out.cpu().numpy())
    sp = gm.Superpixels(dev, spacing=v)
    sp.em_iters(T)
    labels = sp.labels()
    torch.cuda.synchronize()
    assert in_candidates(labels.cpu().numpy())
    with pytest.raises(gm.GmmspError) as ei:
        sp.labels(want_loglik=True)
    assert ei.value.status == 4
    sp.close()
