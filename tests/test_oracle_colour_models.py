"""Pins of the oracle's two further colour models against things other than itself.

  split (Eq. BlockSigma1)   Sigma_c = diag(sigma_l^2, Sigma_(a,b))
  gray (Sec. III-A, III-C)  c_i = L*, a scalar; Sigma_c = sigma^2

E-steps against scipy's multivariate normal over all K Gaussians (masked by
Eq. Ik) with the covariance written out here; M-steps against numpy weighted
moments and eigh; the grey-level conversion against its closed form and the
colour conversion of greys; both models against the full model on images
whose a, b channels are zero, where the three must agree up to the constant
density factor of the (a, b) block; EM monotonicity (Sec. III-B).
"""
import numpy as np
import pytest
from scipy.special import logsumexp
from scipy.stats import multivariate_normal

import oracle
from synth import voronoi_image
from tests.test_oracle_pins import in_window, pixel_z, random_spd, random_theta, unpack

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def split_full(cs, cc):
    """The 5x5 covariance of Eq. (BlockSigma) with the colour block of Eq. (BlockSigma1)."""
    S = np.zeros((5, 5))
    S[0, 0], S[0, 1], S[1, 1] = cs
    S[1, 0] = S[0, 1]
    S[2, 2] = cc[0]
    S[3, 3], S[3, 4], S[4, 4] = cc[3], cc[4], cc[5]
    S[4, 3] = S[3, 4]
    return S


def gray_full(cs, cc):
    """The 3x3 covariance of (x, y, L) for a grayscale image."""
    S = np.zeros((3, 3))
    S[0, 0], S[0, 1], S[1, 1] = cs
    S[1, 0] = S[0, 1]
    S[2, 2] = cc[0]
    return S


def mixture_reference(z, th, g, W, H, cov_of, mean_of):
    logp = np.stack([multivariate_normal(mean_of(th.mu[k]), cov_of(th.cs[k], th.cc[k])).logpdf(z)
                     for k in range(g.K)], axis=1)
    mask = np.array([[in_window(k % g.nx, g.v, W, i % W) and in_window(k // g.nx, g.v, H, i // W)
                      for k in range(g.K)] for i in range(W * H)])
    lm = np.where(mask, logp, -np.inf)
    lse = logsumexp(lm, axis=1)
    return lse, np.exp(lm - lse[:, None])


def check_posteriors(R, cand, ncand, post, K):
    for i in range(post.shape[0]):
        got = np.zeros(K)
        got[cand[i, :ncand[i]]] = R[i, :ncand[i]]
        np.testing.assert_allclose(got, post[i], atol=1e-12)


@pytest.mark.parametrize("W,H,v,seed", [(16, 16, 4, 0), (19, 17, 5, 1), (16, 16, 7, 2)])
def test_split_estep_matches_block_mixture(W, H, v, seed):
    rng = np.random.default_rng(seed)
    lab = rng.uniform([0, -60, -60], [100, 60, 60], size=(H, W, 3))
    g = oracle.grid(W, H, spacing=v)
    th = random_theta(rng, g, lab)     # its colour blocks have L-a, L-b entries: the model ignores them
    R, ll, L, cand, ncand = oracle.estep(lab, g, th, colour="split")
    lse, post = mixture_reference(pixel_z(W, H, lab), th, g, W, H, split_full, lambda m: m)
    np.testing.assert_allclose(ll, lse, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(L, lse.sum(), rtol=1e-12)
    check_posteriors(R, cand, ncand, post, g.K)


@pytest.mark.parametrize("W,H,v,seed", [(16, 16, 4, 3), (19, 17, 5, 4)])
def test_gray_estep_matches_3d_mixture(W, H, v, seed):
    rng = np.random.default_rng(seed)
    lab = rng.uniform([0, -60, -60], [100, 60, 60], size=(H, W, 3))
    g = oracle.grid(W, H, spacing=v)
    th = random_theta(rng, g, lab)     # a, b of mu and of the colour block are not read
    R, ll, L, cand, ncand = oracle.estep(lab, g, th, colour="gray")
    z = pixel_z(W, H, lab)[:, :3]      # (x, y, L)
    lse, post = mixture_reference(z, th, g, W, H, gray_full, lambda m: m[:3])
    np.testing.assert_allclose(ll, lse, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(L, lse.sum(), rtol=1e-12)
    check_posteriors(R, cand, ncand, post, g.K)


def test_log_gauss_models_match_scipy():
    rng = np.random.default_rng(5)
    for _ in range(20):
        S = random_spd(rng, 2, 10.0)
        C = random_spd(rng, 3, 40.0)
        mu = rng.normal(size=5) * 10
        z = mu + rng.normal(size=5) * 5
        cs = [S[0, 0], S[0, 1], S[1, 1]]
        cc = [C[0, 0], C[0, 1], C[0, 2], C[1, 1], C[1, 2], C[2, 2]]
        ref = multivariate_normal(mu, split_full(cs, cc)).logpdf(z)
        assert abs(oracle.log_gauss(z, mu, cs, cc, colour="split") - ref) < 1e-11
        ref = multivariate_normal(mu[:3], gray_full(cs, cc)).logpdf(z[:3])
        assert abs(oracle.log_gauss(z, mu, cs, cc, colour="gray") - ref) < 1e-11


@pytest.mark.parametrize("colour", ["split", "gray"])
@pytest.mark.parametrize("W,H,v,seed", [(16, 16, 4, 0), (23, 17, 4, 2)])
def test_mstep_matches_weighted_moments(colour, W, H, v, seed):
    rng = np.random.default_rng(seed)
    lab = rng.uniform([0, -60, -60], [100, 60, 60], size=(H, W, 3))
    g = oracle.grid(W, H, spacing=v)
    cand, ncand = oracle.candidates(g)
    R = np.zeros((W * H, 9))
    for i in range(W * H):
        w = rng.uniform(0.05, 1.0, size=ncand[i])
        R[i, :ncand[i]] = w / w.sum()
    th0 = oracle.init_theta(lab, g, colour=colour)
    eps_s, eps_c = 2.0, 8.0
    th, cs_raw, cc_raw, wsum, dead, _ = oracle.mstep(lab, g, th0, R, cand, ncand, eps_s, eps_c, colour=colour)
    assert dead == 0
    z = pixel_z(W, H, lab)
    for k in range(g.K):
        w = np.zeros(W * H)
        for i in range(W * H):
            for j in range(ncand[i]):
                if cand[i, j] == k:
                    w[i] = R[i, j]
        mu = np.average(z, axis=0, weights=w)
        full = np.cov(z.T, aweights=w, bias=True)
        S = full[:2, :2]
        lam, Q = np.linalg.eigh(S)
        np.testing.assert_allclose(unpack(th.cs[k]), Q @ np.diag(np.maximum(lam, eps_s)) @ Q.T, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(th.mu[k, :3], mu[:3], rtol=1e-12, atol=1e-10)
        np.testing.assert_allclose(cc_raw[k, 0], full[2, 2], rtol=1e-10)
        assert th.cc[k, 0] == pytest.approx(max(full[2, 2], eps_c), rel=1e-10)
        assert th.cc[k, 1] == 0.0 and th.cc[k, 2] == 0.0          # no L-(a, b) entries in either model
        if colour == "split":
            np.testing.assert_allclose(th.mu[k, 3:], mu[3:], rtol=1e-12, atol=1e-10)
            AB = full[3:, 3:]
            np.testing.assert_allclose(unpack(cc_raw[k, 3:]), AB, rtol=1e-10, atol=1e-9)
            lam, Q = np.linalg.eigh(AB)
            np.testing.assert_allclose(unpack(th.cc[k, 3:]), Q @ np.diag(np.maximum(lam, eps_c)) @ Q.T,
                                       rtol=1e-9, atol=1e-9)
        else:
            assert np.all(th.mu[k, 3:] == 0.0) and np.all(th.cc[k, 3:] == 0.0)


def test_gray2l_closed_form_and_greys_of_rgb2lab():
    c = np.arange(256)
    s = c / 255.0
    Y = np.where(s <= 0.04045, s / 12.92, ((s + 0.055) / 1.055) ** 2.4)
    d = 6 / 29
    f = np.where(Y > d ** 3, np.cbrt(Y), Y / (3 * d * d) + 4 / 29)
    L = oracle.gray2l(c.astype(np.uint8))
    np.testing.assert_allclose(L, 116 * f - 16, rtol=0, atol=1e-12)
    # the colour conversion of (c, c, c): the tabulated matrix's Y row sums to 1 within 1e-7
    np.testing.assert_allclose(L, oracle.rgb2lab(np.stack([c, c, c], 1).astype(np.uint8))[:, 0], atol=2e-5)
    assert L[0] == 0.0 and L[255] == pytest.approx(100.0, abs=1e-12)


def zero_ab_image(W, H, seed):
    lab = oracle.rgb2lab(voronoi_image(W, H, 12, 8.0, seed=seed))
    lab[..., 1:] = 0.0
    return lab


def test_models_agree_when_ab_is_zero():
    # With a = b = 0 everywhere the full model's colour covariance has zero
    # L-a, L-b and a-b entries and an (a, b) block floored to eps_c I (lambda^2 I
    # at the start): the same for every k, so the posteriors of all three models
    # are equal and each density carries the factor 1 / (2 pi eps_c) of that block.
    W, H, v, T, lam, eps_c = 96, 72, 8, 6, 8.0, 8.0
    lab = zero_ab_image(W, H, 3)
    full = oracle.em(lab, W, H, spacing=v, T=T)
    split = oracle.em(lab, W, H, spacing=v, T=T, colour="split")
    gray = oracle.em(lab, W, H, spacing=v, T=T, colour="gray")
    N = W * H
    np.testing.assert_array_equal(split.labels, full.labels)
    np.testing.assert_allclose(split.theta.mu, full.theta.mu, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(split.theta.cs, full.theta.cs, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(split.theta.cc, full.theta.cc, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(split.loglik, full.loglik, rtol=1e-13)
    np.testing.assert_array_equal(gray.labels, full.labels)
    np.testing.assert_allclose(gray.theta.mu[:, :3], full.theta.mu[:, :3], rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(gray.theta.cs, full.theta.cs, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(gray.theta.cc[:, 0], full.theta.cc[:, 0], rtol=1e-12)
    np.testing.assert_allclose(full.theta.cc[:, 3], eps_c)
    np.testing.assert_allclose(full.theta.cc[:, 5], eps_c)
    gap = gray.loglik - full.loglik
    assert gap[0] == pytest.approx(N * np.log(2 * np.pi * lam * lam), rel=1e-10)
    np.testing.assert_allclose(gap[1:], N * np.log(2 * np.pi * eps_c), rtol=1e-10)


def test_gray_reads_only_L():
    W, H = 64, 48
    lab = oracle.rgb2lab(voronoi_image(W, H, 8, 8.0, seed=5))
    other = lab.copy()
    other[..., 1:] = np.random.default_rng(6).uniform(-80, 80, size=(H, W, 2))
    a = oracle.em(lab, W, H, spacing=8, T=4, colour="gray")
    b = oracle.em(other, W, H, spacing=8, T=4, colour="gray")
    np.testing.assert_array_equal(a.labels, b.labels)
    np.testing.assert_array_equal(a.theta.mu, b.theta.mu)
    np.testing.assert_array_equal(a.loglik, b.loglik)


def test_split_differs_from_full_on_colour_images():
    # the L-(a, b) correlation of a real colour image is not zero: the models part
    lab = oracle.rgb2lab(voronoi_image(96, 72, 12, 8.0, seed=7))
    full = oracle.em(lab, 96, 72, spacing=8, T=3)
    split = oracle.em(lab, 96, 72, spacing=8, T=3, colour="split")
    assert np.abs(full.theta.cc[:, 1:3]).max() > 1.0
    assert np.all(split.theta.cc[:, 1:3] == 0.0)
    assert split.loglik[-1] < full.loglik[-1]   # a constrained family fits no better


@pytest.mark.parametrize("colour", ["split", "gray"])
def test_loglik_non_decreasing(colour):
    # Sec. III-B: the argument holds in any family over which the M-step maximises Q.
    img = voronoi_image(96, 72, 12, 8.0, seed=3)
    lab = oracle.rgb2lab(img)
    res = oracle.em(lab, 96, 72, spacing=8, T=10, eps_s=1e-9, eps_c=1e-9, colour=colour)
    assert res.raised.sum() == 0
    assert np.all(np.diff(res.loglik) >= -1e-9 * np.abs(res.loglik[1:])), res.loglik
    res = oracle.em(lab, 96, 72, spacing=8, T=10, colour=colour)
    assert res.raised.sum() > 0
    assert np.all(np.diff(res.loglik) >= -1e-9 * np.abs(res.loglik[1:])), res.loglik


def test_single_gaussian_gray_is_sample_moments():
    rng = np.random.default_rng(8)
    lab = rng.uniform([0, -60, -60], [100, 60, 60], size=(16, 16, 3))
    res = oracle.em(lab, 16, 16, spacing=16, T=1, colour="gray")
    z = pixel_z(16, 16, lab)
    np.testing.assert_allclose(res.theta.mu[0, :3], z[:, :3].mean(0), rtol=1e-13)
    assert res.theta.cc[0, 0] == pytest.approx(max(z[:, 2].var(), 8.0), rel=1e-12)
    np.testing.assert_allclose(unpack(res.theta.cs[0]), np.diag([255 / 12, 255 / 12]), atol=1e-12)
