"""Pins of the network oracle (oracle/cnn.py) against things other than itself."""
import numpy as np
import pytest

from oracle import cnn


def rand_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, cnn.param_count())


def rand_lab(B, H, W, seed):
    rng = np.random.default_rng(seed)
    lab = np.empty((B, 3, H, W))
    lab[:, 0] = rng.uniform(0, 100, (B, H, W))
    lab[:, 1:] = rng.uniform(-60, 60, (B, 2, H, W))
    return lab


def test_param_count_and_layout():
    # 2 x (32 x 32 + 32) + 3 x (32 x 288 + 32) + (16 x 288 + 16)
    assert cnn.param_count() == 2 * (1024 + 32) + 3 * (9216 + 32) + (4608 + 16) == 34480
    flat = np.arange(cnn.param_count(), dtype=np.float64)
    P = cnn.unpack(flat)
    assert P[0][0].shape == (32, 32) and P[5][0].shape == (16, 288)
    assert P[1][0][0, 0] == 1024 + 32          # W2 follows W1 and b1
    np.testing.assert_array_equal(cnn.pack(P), flat)


def test_conv3x3_matches_scipy_correlate2d():
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 7, 32))
    W = rng.normal(size=(3, 9 * 32))
    b = rng.normal(size=3)
    y = cnn.conv3x3(x, W, b)
    for n in range(2):
        for o in range(3):
            ref = np.full((5, 7), b[o])
            for c in range(32):
                kern = W[o, c::32].reshape(3, 3)   # taps t = 3 dy + dx for input channel c
                ref += scipy_signal.correlate2d(x[n, :, :, c], kern, mode="same", boundary="fill")
            np.testing.assert_allclose(y[n, :, :, o], ref, rtol=1e-12, atol=1e-12)


def test_patch_layout_brute_force():
    B, H, W, v = 2, 31, 40, 9     # f = 3; remainders 4 columns, 4 rows
    lab = rand_lab(B, H, W, 2)
    x0 = cnn.patches(lab, v)
    nx, ny = W // v, H // v
    f = v // 3
    assert x0.shape == (B, ny, nx, f, f, 32)
    rng = np.random.default_rng(3)
    for _ in range(200):
        n, ky, kx, qy, qx = (rng.integers(B), rng.integers(ny), rng.integers(nx), rng.integers(f),
                             rng.integers(f))
        dy, dx, col = rng.integers(3), rng.integers(3), rng.integers(3)
        px, py = kx * v + 3 * qx + dx, ky * v + 3 * qy + dy
        val = lab[n, col, py, px]
        expect = val * 0.02 - 1.0 if col == 0 else val * 0.02
        assert x0[n, ky, kx, qy, qx, (3 * dy + dx) * 3 + col] == pytest.approx(expect, abs=1e-13)
    assert np.all(x0[..., 27:] == 0)


def test_pool_is_block_mean():
    B, H, W, v = 1, 30, 45, 15
    lab = rand_lab(B, H, W, 4)
    flat = rand_params(5)
    out, cache = cnn.forward(flat, lab, v)
    h2, c0 = cache["h2"], cache["c"][0]
    ny, nx, f = H // v, W // v, v // 3
    ref = h2.reshape(B, ny, nx, f * f, 32).mean(axis=3)
    np.testing.assert_allclose(c0[..., :cnn.START_CH], ref[..., :cnn.START_CH], rtol=1e-13, atol=1e-13)
    # the last three channels are the scaled colour of the Sec. III-C start pixel (k_x v + v//2, ...)
    c = v // 2
    for ky in range(ny):
        for kx in range(nx):
            px = lab[0, :, ky * v + c, kx * v + c]
            want = [px[0] * cnn.IN_SCALE - 1.0, px[1] * cnn.IN_SCALE, px[2] * cnn.IN_SCALE]
            np.testing.assert_allclose(c0[0, ky, kx, cnn.START_CH:], want, rtol=1e-13, atol=1e-13)
    assert out.shape == (B, ny, nx, 16)


@pytest.mark.parametrize("v", [9, 15])
def test_backward_matches_finite_differences(v):
    B, H, W = 2, 2 * v + 4, 3 * v + 2
    lab = rand_lab(B, H, W, 6)
    flat = rand_params(7, 0.25)
    nx, ny = W // v, H // v
    target = np.random.default_rng(8).normal(size=(B, ny * nx, 10))

    def L(p):
        out, _ = cnn.forward(p, lab, v)
        return cnn.loss(out, target)[0]

    out, cache = cnn.forward(flat, lab, v)
    _, g_out = cnn.loss(out, target)
    g = cnn.backward(cache, g_out)
    rng = np.random.default_rng(9)
    offs = np.cumsum([0] + [cout * taps * 32 + cout for taps, cout in cnn.LAYERS])
    idx = []
    for l in range(6):
        idx += list(rng.integers(offs[l], offs[l + 1], 6))
        idx.append(offs[l + 1] - 1)       # a bias
    idx.append(5)                          # W1[0][5]: an input channel in use
    for i in idx:
        h = 1e-6
        p1, p2 = flat.copy(), flat.copy()
        p1[i] += h
        p2[i] -= h
        fd = (L(p1) - L(p2)) / (2 * h)
        assert fd == pytest.approx(g[i], rel=2e-6, abs=1e-9), i
    # padded input channels 27..31 carry no gradient
    W1g = g[:1024].reshape(32, 32)
    assert np.all(W1g[:, 27:] == 0)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(10)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 1000), rng.normal(0, 1e4, 1000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -0.0, 0.0, 65504.0]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(cnn.bf16(x), ref)
    # ties go to the even mantissa
    assert cnn.bf16(1.0 + 2 ** -8) == 1.0
    assert cnn.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6


def test_targets_and_theta0_are_inverse():
    rng = np.random.default_rng(11)
    v, W, H = 15, 481, 321
    lab_img = rand_lab(1, H, W, 12)[0]
    K = (W // v) * (H // v)
    xc, yc = cnn.centre(W, H, v)
    mu = np.zeros((K, 5))
    mu[:, 0] = xc + rng.uniform(-0.9, 0.9, K) * v
    mu[:, 1] = yc + rng.uniform(-0.9, 0.9, K) * v
    mu[:, 2:] = rng.uniform(-50, 80, (K, 3))
    cs = np.zeros((K, 3))
    cs[:, 0], cs[:, 2] = rng.uniform(3, 80, K), rng.uniform(3, 80, K)
    cc = np.zeros((K, 6))
    cc[:, 0], cc[:, 3], cc[:, 5] = rng.uniform(9, 400, K), rng.uniform(9, 400, K), rng.uniform(9, 400, K)
    t = cnn.targets(mu, cs, cc, lab_img, v)
    mu2, cs2, cc2 = cnn.theta0_from_outputs(t.astype(np.float32), lab_img, v)
    np.testing.assert_allclose(mu2, mu, rtol=1e-5, atol=1e-4)
    np.testing.assert_allclose(cs2, cs, rtol=1e-5)
    np.testing.assert_allclose(cc2, cc, rtol=1e-5)
    # the floors and the window clip of theta_0
    o = np.zeros((K, 16))
    o[:, 0] = 5.0
    o[:, 5:10] = -30.0
    mu3, cs3, cc3 = cnn.theta0_from_outputs(o, lab_img, v, eps_s=2.0, eps_c=8.0)
    kx = np.arange(K) % (W // v)
    np.testing.assert_array_equal(mu3[:, 0], (kx + 2) * v)
    assert np.all(cs3[:, [0, 2]] == 2.0) and np.all(cc3[:, [0, 3, 5]] == 8.0)
    assert np.all(cs3[:, 1] == 0) and np.all(cc3[:, [1, 2, 4]] == 0)


def test_loss_of_a_constant_network():
    # all weights zero: out = b6 everywhere, loss = mean (b6_j - t)^2 over the used outputs
    flat = np.zeros(cnn.param_count())
    b6 = np.arange(16) * 0.1
    flat[-16:] = b6
    lab = rand_lab(1, 30, 30, 13)
    out, _ = cnn.forward(flat, lab, 15)
    t = np.random.default_rng(14).normal(size=(1, 4, 10))
    val, g = cnn.loss(out, t)
    assert val == pytest.approx(np.mean((b6[None, None, :10] - t) ** 2), rel=1e-14)
    assert np.all(g[..., 10:] == 0)
