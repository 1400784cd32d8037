"""The batch kernels that the bench's workloads run, against the FP64 oracle.

Every launch variant the batch autotuner can pick (3-5 blocks per SM: the
persistent E + M kernel; 6, 7: the one-cell-per-warp kernels with capped
registers; each with the one-thread and the 16-lane finalize) runs Algorithm 1,
steps 2-7 (Eq. Rik, UpdateMu, UpdateSigS/C, mlams/mlamc, obtLi) on the learned
start's workload (481 x 321 at spacing 15) and on uneven sizes of the batched
workload; every image's means, covariances, final log-likelihood and labels
are compared with the oracle at the parity bar.  The learned start is then
checked end to end: the GPU's theta_0 from the trained network, given to the
oracle, must give the GPU's theta_2, labels and L(theta_2).
"""
import numpy as np
import pytest

import oracle
from synth import voronoi_image
from synth.voronoi import batch_regions
from tests import parity

pytestmark = pytest.mark.gpu

V = 15
T = 10
SIZES = [(481, 321), (481, 321), (481, 321), (320, 240), (640, 480), (1280, 720), (97, 61), (37, 23)]
LEARN_W, LEARN_H, LEARN_B = 481, 321, 4


@pytest.fixture(scope="module")
def gm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    torch.cuda.set_device(0)
    return gm


def make_lab(W, H, seed):
    regions = 150 if (W, H) == (481, 321) else batch_regions(W, H)
    return oracle.rgb2lab(voronoi_image(W, H, regions, 8.0, seed)).astype(np.float32)


@pytest.fixture(scope="module")
def plain_case():
    labs = [make_lab(W, H, 2_000_000 + i) for i, (W, H) in enumerate(SIZES)]
    refs = [oracle.em(lab.astype(np.float64), W, H, spacing=V, T=T) for lab, (W, H) in zip(labs, SIZES)]
    return labs, refs


def check_image(mu, cs, cc, labels, ll, ref, what):
    em = parity.mean_rel_err(mu, ref.theta.mu)
    es = parity.cov_rel_err(cs, ref.theta.cs)
    ec = parity.cov_rel_err(cc, ref.theta.cc)
    assert em <= parity.MEAN_TOL and es <= parity.COV_TOL and ec <= parity.COV_TOL, (what, em, es, ec)
    agree, ndiff, worst = parity.label_report(labels, ref.labels, ref.margin)
    assert agree >= parity.LABEL_AGREE and worst < parity.MARGIN_TOL, (what, agree, ndiff, worst)
    assert abs(ll - ref.loglik[-1]) <= parity.LL_RTOL * abs(ref.loglik[-1]), (what, ll, ref.loglik[-1])


@pytest.mark.parametrize("fin16", [False, True])
@pytest.mark.parametrize("bps", [3, 4, 5, 6, 7])
def test_batch_launch_variants_match_oracle(gm, plain_case, bps, fin16):
    import torch
    labs, refs = plain_case
    dev = [torch.from_numpy(x).cuda() for x in labs]
    bt = gm.SuperpixelsBatch([(H, W) for (W, H) in SIZES], spacing=V, lab_input=True)
    gm.gmmsp_batch_set_tuning(bt.b, bps, fin16)
    assert bt.tuning()["blocks_per_sm"] == bps and bt.tuning()["finalize16"] == fin16
    labels, ll = bt.segment(dev, iters=T, want_loglik=True)
    torch.cuda.synchronize()
    for i, (W, H) in enumerate(SIZES):
        mu, cs, cc = bt.get_params(i, refs[i].grid.K)
        check_image(mu, cs, cc, labels[i].cpu().numpy(), ll[i], refs[i], (bps, fin16, i, W, H))
    bt.close()


@pytest.mark.parametrize("bps,first", [(7, 6), (6, 7), (7, 4), (4, 7)])
def test_batch_first_pass_launch_of_its_own(gm, plain_case, bps, first):
    """A segment's first E + M pass (diagonal blocks) at another launch choice than the rest."""
    import torch
    labs, refs = plain_case
    dev = [torch.from_numpy(x).cuda() for x in labs]
    bt = gm.SuperpixelsBatch([(H, W) for (W, H) in SIZES], spacing=V, lab_input=True)
    gm.gmmsp_batch_set_tuning(bt.b, bps, True)
    assert bt.tuning()["first_pass_blocks_per_sm"] == bps  # follows until set
    bt.set_launch(bps, first_pass=first)
    assert bt.tuning()["first_pass_blocks_per_sm"] == first and bt.tuning()["blocks_per_sm"] == bps
    labels, ll = bt.segment(dev, iters=T, want_loglik=True)
    torch.cuda.synchronize()
    for i, (W, H) in enumerate(SIZES):
        mu, cs, cc = bt.get_params(i, refs[i].grid.K)
        check_image(mu, cs, cc, labels[i].cpu().numpy(), ll[i], refs[i], (bps, first, i, W, H))
    bt.close()


@pytest.fixture(scope="module")
def learned_case(gm):
    """The trained network's theta_0 on the GPU for LEARN_B images of the learned start's workload."""
    import torch
    from paper_1612_08792_gb300.learned_init import load_pretrained
    labs = [make_lab(LEARN_W, LEARN_H, 3_000_000 + i) for i in range(LEARN_B)]
    dev = [torch.from_numpy(x).cuda() for x in labs]
    net = load_pretrained(V)
    bt = gm.SuperpixelsBatch([(LEARN_H, LEARN_W)] * LEARN_B, spacing=V, lab_input=True)
    bt.set_init_net(net)
    bt.segment(dev, iters=0)
    torch.cuda.synchronize()
    K = (LEARN_W // V) * (LEARN_H // V)
    theta0 = [oracle.Theta(*bt.get_params(i, K)) for i in range(LEARN_B)]
    net.check()
    bt.close()
    refs = [oracle.em(lab.astype(np.float64), LEARN_W, LEARN_H, spacing=V, T=2, theta0=th)
            for lab, th in zip(labs, theta0)]
    yield labs, dev, net, theta0, refs
    net.close()


@pytest.mark.parametrize("bps", [3, 5, 6, 7])
def test_learned_start_then_two_iterations_match_oracle(gm, learned_case, bps):
    import torch
    labs, dev, net, theta0, refs = learned_case
    bt = gm.SuperpixelsBatch([(LEARN_H, LEARN_W)] * LEARN_B, spacing=V, lab_input=True)
    bt.set_init_net(net)
    gm.gmmsp_batch_set_tuning(bt.b, bps, bps % 2 == 1)
    labels, ll = bt.segment(dev, iters=2, want_loglik=True)
    torch.cuda.synchronize()
    K = (LEARN_W // V) * (LEARN_H // V)
    for i in range(LEARN_B):
        # the oracle starts from exactly the GPU's theta_0 (the learned start is the only input)
        assert np.all(np.isfinite(theta0[i].mu)) and np.all(theta0[i].cs[:, 0] > 0)
        mu, cs, cc = bt.get_params(i, K)
        check_image(mu, cs, cc, labels[i].cpu().numpy(), ll[i], refs[i], ("learned", bps, i))
    bt.close()


def test_headline_step_at_full_size(gm):
    """The learned start + 2 iterations on the full headline batch, as bench.py times it: 256
    held-out 481x321 sRGB images (seeds 1,000,000 + i, 150 regions, sigma 8), spacing 15, RGB8
    input converted inside the network's first kernel, the autotuner's launch choices.
    Every label map of the batch: each label is the index of one of its pixel's 3 x 3 seeds
    (Eq. obtLi, the window of Eq. Ik). Images 0, 127 and 255: theta_2, the labels and L(theta_2)
    against the oracle (Algorithm 1 steps 2-7) started from the GPU's theta_0 on the GPU's CIELAB."""
    import torch
    from paper_1612_08792_gb300.learned_init import load_pretrained
    from synth.voronoi_torch import voronoi_batch
    n, W, H, v = 256, 481, 321, 15
    nx, ny = W // v, H // v
    K = nx * ny
    buf = voronoi_batch(W, H, 150, 8.0, range(1_000_000, 1_000_000 + n))
    imgs = [buf[i] for i in range(n)]
    net = load_pretrained(v)
    bt = gm.SuperpixelsBatch([(H, W)] * n, spacing=v)
    bt.autotune(imgs, reps=2)
    bt.set_init_net(net)
    sample = (0, 127, 255)
    bt.segment(imgs, iters=0)  # theta_0 and the CIELAB of the step's start
    torch.cuda.synchronize()
    theta0 = {i: oracle.Theta(*bt.get_params(i, K)) for i in sample}
    labs = {i: bt.get_lab(i) for i in sample}
    labels, ll = bt.segment(imgs, iters=2, want_loglik=True)
    torch.cuda.synchronize()
    net.check()

    lab_all = torch.stack(labels).long()
    ys = torch.arange(H, device=lab_all.device).view(1, H, 1)
    xs = torch.arange(W, device=lab_all.device).view(1, 1, W)
    kx, ky = lab_all % nx, lab_all // nx
    assert bool(((lab_all >= 0) & (lab_all < K)).all())
    assert bool(((kx - xs // v).abs() <= 1).all()) and bool(((ky - ys // v).abs() <= 1).all())
    assert np.all(np.isfinite(ll))

    for i in sample:
        ref = oracle.em(labs[i].astype(np.float64), W, H, spacing=v, T=2, theta0=theta0[i])
        mu, cs, cc = bt.get_params(i, K)
        check_image(mu, cs, cc, labels[i].cpu().numpy(), ll[i], ref, ("full size", i))
    bt.close()
    net.close()
