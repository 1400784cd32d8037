"""The learned initialiser on the GPU (gmmsp_net_*) against the FP64 network oracle."""
import numpy as np
import pytest

import oracle
from oracle import cnn as ocnn
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


def lab_planes(sizes_seeds, W, H):
    """(B, 3, H, W) float32 CIELAB planes of seeded synthetic images (oracle conversion)."""
    out = []
    for seed in sizes_seeds:
        img = voronoi_image(W, H, max(4, W * H // 1000), 8.0, seed)
        out.append(oracle.rgb2lab(img).astype(np.float32).transpose(2, 0, 1))
    return np.ascontiguousarray(np.stack(out))  # planes in memory order (the device copy keeps strides)


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-30))


def test_weights_round_trip_and_bad_arguments(gm):
    from paper_1612_08792_gb300.learned_init import InitNet, init_weights
    assert gm.gmmsp_net_param_count() == ocnn.param_count()
    w = init_weights(3)
    net = InitNet(15, weights=w)
    np.testing.assert_array_equal(net.get_weights(), w)
    with pytest.raises(gm.GmmspError):
        gm.gmmsp_net_set_weights(net.n, w[:-1])
    with pytest.raises(gm.GmmspError):
        gm.gmmsp_net_create(14)
    bad = w.copy()
    bad[7] = np.nan
    with pytest.raises(gm.GmmspError):
        gm.gmmsp_net_set_weights(net.n, bad)
    # a batch of mixed sizes cannot take a learned start; nor one of another spacing
    b1 = gm.SuperpixelsBatch([(321, 481), (240, 320)], spacing=15)
    with pytest.raises(gm.GmmspError):
        b1.set_init_net(net)
    b2 = gm.SuperpixelsBatch([(321, 481)], spacing=12)
    with pytest.raises(gm.GmmspError):
        b2.set_init_net(net)
    b1.close()
    b2.close()
    net.check()
    net.close()


@pytest.mark.parametrize("W,H,v,B", [(481, 321, 15, 2), (100, 70, 15, 3), (64, 50, 9, 2), (77, 61, 12, 1),
                                     (40, 40, 21, 2)])
def test_forward_matches_oracle(gm, W, H, v, B):
    import torch
    from paper_1612_08792_gb300.learned_init import InitNet, init_weights
    lab = lab_planes(range(20, 20 + B), W, H)
    w = init_weights(v)
    w[-16:] = np.linspace(-1, 1, 16)          # nonzero output biases
    net = InitNet(v, weights=w)
    dev = torch.from_numpy(lab).cuda()
    out = net.forward(dev.data_ptr(), B, W, H).cpu().numpy()
    net.check()
    ref, _ = ocnn.forward(w, lab, v, emulate_bf16=True)
    assert out.shape == ref.shape
    assert np.all(np.isfinite(out))
    # BF16 activations, FP32 accumulation: the only differences are rounding flips
    assert rel_l2(out, ref) < 2e-3, rel_l2(out, ref)
    assert np.max(np.abs(out - ref)) < 1e-2 * np.max(np.abs(ref))
    _, cache = ocnn.forward(w, lab, v, emulate_bf16=True)
    cells = out.shape[0] * out.shape[1] * out.shape[2]
    for l in range(4):
        act = gm.gmmsp_net_get_activation(net.n, l, cells).reshape(cache["c"][l].shape)
        assert rel_l2(act, cache["c"][l]) < 2e-3, (l, rel_l2(act, cache["c"][l]))
    # the exact FP64 network is within BF16 distance too
    exact, _ = ocnn.forward(w, lab, v)
    assert rel_l2(out, exact) < 3e-2
    net.close()


GRAD_CASES = [(481, 321, 15, 2), (100, 70, 15, 3), (64, 50, 9, 2), (77, 61, 12, 1), (40, 40, 21, 2)]
# Relative L2 error of each layer's weight and bias gradient against the BF16-emulating FP64
# oracle.  The device's backward pass stores the activation gradients in BF16 and accumulates
# in FP32, the oracle accumulates in FP64: the gradients differ by the BF16 rounding flips that
# the two accumulation orders cause.  Measured on a GB300 (largest per-layer value over weights
# and biases): 481x321 B=2 1.1e-3 (the case with the most positions, so the most flips),
# 100x70 B=3 1.3e-6, 64x50 v=9 2.7e-7, 77x61 v=12 2.3e-7, 40x40 v=21 4.7e-8; the loss within
# 1.1e-7 relative.  GRAD_TOL keeps a factor of about 4 over the largest.
GRAD_TOL = 5e-3
LOSS_RTOL = 1e-5


@pytest.mark.parametrize("W,H,v,B", GRAD_CASES)
def test_gradient_matches_oracle(gm, W, H, v, B):
    import json
    import os
    import torch
    from paper_1612_08792_gb300.learned_init import InitNet, init_weights
    lab = lab_planes(range(30, 30 + B), W, H)
    w = init_weights(11)
    net = InitNet(v, weights=w)
    K = (W // v) * (H // v)
    tgt = np.random.default_rng(12).normal(0, 1, (B, K, 10)).astype(np.float32)
    dev = torch.from_numpy(lab).cuda()        # held: a dropped temporary's memory could take the target
    loss, g = net.grad(dev, B, W, H, torch.from_numpy(tgt).cuda())
    out, cache = ocnn.forward(w, lab, v, emulate_bf16=True)
    ref_loss, g_out = ocnn.loss(out, tgt)
    ref = ocnn.backward(cache, g_out)
    assert loss == pytest.approx(ref_loss, rel=LOSS_RTOL)
    o = 0
    errs = []
    for taps, cout in ocnn.LAYERS:
        nw = cout * taps * 32
        gw, rw = g[o:o + nw], ref[o:o + nw]
        gb, rb = g[o + nw:o + nw + cout], ref[o + nw:o + nw + cout]
        errs.append((rel_l2(gw, rw), rel_l2(gb, rb)))
        o += nw + cout
    cos = float(np.dot(g, ref) / np.linalg.norm(g) / np.linalg.norm(ref))
    if os.environ.get("GMMSP_GRAD_OUT"):
        with open(os.environ["GMMSP_GRAD_OUT"], "a") as fh:
            fh.write(json.dumps({"case": [W, H, v, B], "layers_w_b": errs, "cos": cos,
                                 "loss_rel": abs(loss - ref_loss) / ref_loss}) + "\n")
    for l, (ew, eb) in enumerate(errs):
        assert ew < GRAD_TOL and eb < GRAD_TOL, (l, ew, eb)
    assert cos > 0.999, cos
    # unused input channels of the first layer get exactly zero gradient
    assert np.all(g[:1024].reshape(32, 32)[:, 27:] == 0)
    net.close()


def test_theta0_and_targets_match_oracle(gm):
    import torch
    from paper_1612_08792_gb300.learned_init import InitNet, init_weights
    W, H, v = 481, 321, 15
    lab = lab_planes([40, 41], W, H)
    w = init_weights(13)
    w[-16:] = 0.3 * np.random.default_rng(14).normal(size=16)
    net = InitNet(v, weights=w)
    # single context: theta_0 from the network against the oracle's map of the same outputs
    img0 = torch.from_numpy(np.ascontiguousarray(lab[0].transpose(1, 2, 0))).cuda()
    sp = gm.Superpixels(img0, spacing=v)
    sp.init_from_net(net)
    mu, cs, cc = sp.get_params()
    dev0 = torch.from_numpy(lab[:1]).cuda()
    out = net.forward(dev0, 1, W, H).cpu().numpy()[0]
    rmu, rcs, rcc = ocnn.theta0_from_outputs(out.reshape(-1, 16), lab[0], v)
    assert parity.mean_rel_err(mu, rmu) < 1e-9
    assert parity.cov_rel_err(cs, rcs) < 1e-9
    assert parity.cov_rel_err(cc, rcc) < 1e-9
    sp.close()
    # batch targets after a few EM iterations against the oracle's target map
    imgs = [torch.from_numpy(np.ascontiguousarray(lab[i].transpose(1, 2, 0))).cuda() for i in range(2)]
    bt = gm.SuperpixelsBatch([(H, W)] * 2, spacing=v, lab_input=True)
    bt.segment(imgs, iters=5)
    K = (W // v) * (H // v)
    t = torch.empty(2 * K * 10, dtype=torch.float32, device="cuda")
    bt.targets(t)
    t = t.cpu().numpy().reshape(2, K, 10)
    for i in range(2):
        mu_i, cs_i, cc_i = bt.get_params(i, K)
        ref = ocnn.targets(mu_i, cs_i, cc_i, lab[i], v)
        np.testing.assert_allclose(t[i], ref, rtol=1e-5, atol=1e-5)
    bt.close()
    net.close()


def test_learned_start_batch_equals_single_context(gm):
    import torch
    from paper_1612_08792_gb300.learned_init import InitNet, init_weights
    W, H, v = 481, 321, 15
    lab = lab_planes([50, 51, 52], W, H)
    w = init_weights(15)
    w[-16:] = 0.2 * np.random.default_rng(16).normal(size=16)
    net = InitNet(v, weights=w)
    imgs = [torch.from_numpy(np.ascontiguousarray(lab[i].transpose(1, 2, 0))).cuda() for i in range(3)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        bt = gm.SuperpixelsBatch([(H, W)] * 3, spacing=v, lab_input=True, stream=stream)
        bt.set_init_net(net)
        labels, ll = bt.segment(imgs, iters=2, want_loglik=True)   # captured graph
        again = [x.clone() for x in bt.segment(imgs, iters=2)]    # replay
    stream.synchronize()
    for i in range(3):
        torch.testing.assert_close(labels[i], again[i], rtol=0, atol=0)
        sp = gm.Superpixels(imgs[i], spacing=v)
        sp.set_launch(1)
        sp.init_from_net(net)
        sp.em_iters(2)
        ref, ref_ll = sp.labels(want_loglik=True)
        sp.close()
        assert (labels[i].cpu().numpy() == ref.cpu().numpy()).mean() >= 0.9999
        assert abs(ll[i] - ref_ll) <= 1e-6 * abs(ref_ll)
    bt.close()
    net.check()
    net.close()


def test_training_reduces_loss(gm):
    import torch
    from paper_1612_08792_gb300.learned_init import InitNet, init_weights, layer_slices
    from synth.voronoi_torch import voronoi_batch
    W, H, v, B = 481, 321, 15, 4
    K = (W // v) * (H // v)
    buf = voronoi_batch(W, H, 150, 8.0, [101, 102, 103, 104])
    bt = gm.SuperpixelsBatch([(H, W)] * B, spacing=v)
    bt.segment([buf[i] for i in range(B)], iters=20)
    tgt = torch.empty(B * K * 10, dtype=torch.float32, device="cuda")
    bt.targets(tgt)
    w = init_weights(17)
    b6 = layer_slices()[5][1]
    w[b6.start:b6.start + 10] = tgt.view(-1, 10).mean(0).cpu().numpy()
    net = InitNet(v, weights=w)
    losses = [net.train_step(bt.lab_ptr(), B, W, H, tgt, 3e-3) for _ in range(60)]
    assert np.all(np.isfinite(losses))
    # the output biases start at the target mean, so the first loss is the targets' variance
    assert losses[-1] < 0.8 * losses[0], (losses[0], losses[-1])
    assert np.mean(losses[-10:]) < np.mean(losses[:10])
    net.check()
    bt.close()
    net.close()


def test_pretrained_start_gain(gm):
    """Held-out images: the trained network's start + 2 EM iterations beats the
    paper's start + 2 iterations and is within 0.5 % of the paper's start + 10
    iterations in mean log-likelihood per pixel."""
    import os
    from paper_1612_08792_gb300.learned_init import InitNet, evaluate, pretrained_path
    path = pretrained_path(15)
    if not os.path.exists(path):
        pytest.skip("no trained weights in the package")
    net = InitNet.load(path)
    ev = evaluate(net, n_images=32, plain_iters=(2, 10), learned_iters=(2,))
    assert ev["learned2"] > ev["plain2"], ev
    assert abs(ev["learned2"] - ev["plain10"]) / abs(ev["plain10"]) <= 0.005, ev
    net.close()


def test_bounded_wait_gives_up_and_context_survives(gm):
    """A tensor-core wait on an mbarrier that nothing arrives on runs out after
    its bound, frees its tensor memory and reports GMMSP_E_TIMEOUT; the context
    then runs the network as before."""
    import torch
    from paper_1612_08792_gb300.learned_init import InitNet, init_weights
    assert gm.gmmsp_tc_wait_selftest(256) == gm.GMMSP_E_TIMEOUT
    assert gm.gmmsp_tc_wait_selftest(4096) == gm.GMMSP_E_TIMEOUT
    W, H, v = 64, 50, 9
    lab = lab_planes([60], W, H)
    w = init_weights(18)
    net = InitNet(v, weights=w)
    dev = torch.from_numpy(lab).cuda()
    out = net.forward(dev, 1, W, H).cpu().numpy()
    net.check()
    ref, _ = ocnn.forward(w, lab, v, emulate_bf16=True)
    assert rel_l2(out, ref) < 2e-3
    net.close()


def test_checkpoint_with_optimizer_resumes_exactly(gm, tmp_path):
    """Training k + k steps through a save/load with the Adam state equals 2k steps."""
    import torch
    from paper_1612_08792_gb300.learned_init import InitNet, init_weights
    W, H, v, B = 64, 50, 9, 2
    lab = torch.from_numpy(lab_planes([70, 71], W, H)).cuda()
    K = (W // v) * (H // v)
    tgt = torch.from_numpy(np.random.default_rng(72).normal(0, 1, (B * K, 10)).astype(np.float32)).cuda()
    w0 = init_weights(19)
    ref = InitNet(v, weights=w0)
    for _ in range(6):
        ref.train_step(lab.data_ptr(), B, W, H, tgt, 1e-3, want_loss=False)
    a = InitNet(v, weights=w0)
    for _ in range(3):
        a.train_step(lab.data_ptr(), B, W, H, tgt, 1e-3, want_loss=False)
    path = str(tmp_path / "ckpt.npz")
    a.save(path, optimizer=True)
    b = InitNet.load(path)
    m, v2, step = gm.gmmsp_net_get_adam(b.n)
    assert step == 3 and np.all(v2 >= 0)
    for _ in range(3):
        b.train_step(lab.data_ptr(), B, W, H, tgt, 1e-3, want_loss=False)
    np.testing.assert_array_equal(b.get_weights(), ref.get_weights())
    # without the optimiser state the resumed run differs (Adam restarts)
    a.save(path)
    c = InitNet.load(path)
    for _ in range(3):
        c.train_step(lab.data_ptr(), B, W, H, tgt, 1e-3, want_loss=False)
    assert not np.array_equal(c.get_weights(), ref.get_weights())
    with pytest.raises(gm.GmmspError):
        gm.gmmsp_net_set_adam(c.n, m, -np.ones_like(v2), 1)
    for net in (ref, a, b, c):
        net.close()


def test_set_init_from_arrays_matches_oracle(gm):
    """theta_0 from caller-provided predictions equals the oracle's map of the same values."""
    import torch
    W, H, v = 481, 321, 15
    lab = lab_planes([80], W, H)
    K = (W // v) * (H // v)
    rng = np.random.default_rng(81)
    out = np.zeros((K, 16), dtype=np.float32)
    out[:, :5] = rng.normal(0, 0.6, (K, 5))
    out[:, 5:10] = rng.normal(0, 1.5, (K, 5))
    out[::7, 5:10] = 30.0                       # clipped at 10
    out[::11, 7:10] = -20.0                     # floored at eps_c
    img0 = torch.from_numpy(np.ascontiguousarray(lab[0].transpose(1, 2, 0))).cuda()
    sp = gm.Superpixels(img0, spacing=v)
    sp.set_init(torch.from_numpy(np.ascontiguousarray(out[:, :5])).cuda(),
                torch.from_numpy(np.ascontiguousarray(out[:, 5:10])).cuda())
    mu, cs, cc = sp.get_params()
    rmu, rcs, rcc = ocnn.theta0_from_outputs(out, lab[0], v)
    assert parity.mean_rel_err(mu, rmu) < 1e-9
    assert parity.cov_rel_err(cs, rcs) < 1e-9
    assert parity.cov_rel_err(cc, rcc) < 1e-9
    sp.em_iters(2)                               # and EM runs from there
    labels, ll = sp.labels(want_loglik=True)
    assert np.isfinite(ll)
    with pytest.raises(ValueError):
        sp.set_init(torch.zeros((K - 1, 5), device="cuda"), torch.zeros((K - 1, 5), device="cuda"))
    sp.close()
    g8 = torch.from_numpy((lab[0, 0] * 2.55).clip(0, 255).astype(np.uint8)).cuda()
    sg = gm.Superpixels(g8, spacing=v, colour="gray")
    with pytest.raises(gm.GmmspError):
        sg.set_init(torch.zeros((K, 5), device="cuda"), torch.zeros((K, 5), device="cuda"))
    sg.close()
