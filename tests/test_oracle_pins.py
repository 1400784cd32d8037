"""Pins for the FP64 CPU oracle, against things other than the oracle itself.

Each test checks one routine of ``oracle/`` against a closed form, a
published table, a library routine (scipy / numpy) or a brute-force
evaluation written here from the paper's definitions:

  grid                 Eq. (vxy), (nxyK): hand-computed grid facts
  candidate sets       Eq. (Ik), (kxy): brute force over all k; 1 <= |K_i| <= 9
  CIELAB               tabulated sRGB primaries; closed form on greys
  E-step               Eq. (Rik): full mixture over all K with scipy's
                       multivariate normal, masked by Eq. (Ik)
  M-step               Eq. (UpdateMu/SigS/SigC): numpy weighted moments
  eigenvalue floor     Eq. (mlams/mlamc): numpy eigh; diagonal -> max
  K = 1                one Gaussian: sample mean and covariance
  constant colour      Sigma_c = eps_c I exactly
  EM monotonicity      Sec. III-B (Jensen bound): L(theta_t) non-decreasing
"""
import numpy as np
import pytest
from scipy.special import logsumexp
from scipy.stats import multivariate_normal

import oracle
from synth import voronoi_image

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


# ---------------------------------------------------------------- helpers
def blocks_to_full(cs, cc):
    S = np.zeros((5, 5))
    S[0, 0], S[0, 1], S[1, 1] = cs
    S[1, 0] = S[0, 1]
    S[2, 2], S[2, 3], S[2, 4], S[3, 3], S[3, 4], S[4, 4] = cc
    S[3, 2], S[4, 2], S[4, 3] = S[2, 3], S[2, 4], S[3, 4]
    return S


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    if p.size == 3:
        return np.array([[p[0], p[1]], [p[1], p[2]]])
    return np.array([[p[0], p[1], p[2]], [p[1], p[3], p[4]], [p[2], p[4], p[5]]])


def in_window(kq, v, extent, p):
    """Eq. (Ik) bounds along one axis, written out."""
    b = max(0, v * (kq - 1))
    e = min(extent, v * (kq + 2))
    return b <= p < e


def brute_candidates(W, H, v, nx, ny):
    out = []
    for y in range(H):
        for x in range(W):
            out.append([k for k in range(nx * ny)
                        if in_window(k % nx, v, W, x) and in_window(k // nx, v, H, y)])
    return out


def random_spd(rng, n, scale):
    A = rng.normal(size=(n, n))
    return scale * (A @ A.T / n + 0.3 * np.eye(n))


def random_theta(rng, g, lab):
    K = g.K
    mu = np.zeros((K, 5))
    cs = np.zeros((K, 3))
    cc = np.zeros((K, 6))
    for k in range(K):
        kx, ky = k % g.nx, k // g.nx
        mu[k, 0] = kx * g.v + g.v / 2 + rng.normal()
        mu[k, 1] = ky * g.v + g.v / 2 + rng.normal()
        mu[k, 2:] = lab.reshape(-1, 3).mean(0) + rng.normal(scale=10, size=3)
        S = random_spd(rng, 2, g.v * g.v / 2)
        C = random_spd(rng, 3, 60.0)
        cs[k] = [S[0, 0], S[0, 1], S[1, 1]]
        cc[k] = [C[0, 0], C[0, 1], C[0, 2], C[1, 1], C[1, 2], C[2, 2]]
    return oracle.Theta(mu, cs, cc)


def pixel_z(W, H, lab):
    ys, xs = np.mgrid[0:H, 0:W]
    return np.concatenate([xs.reshape(-1, 1), ys.reshape(-1, 1), lab.reshape(-1, 3)], axis=1).astype(np.float64)


# ---------------------------------------------------------------- grid
@pytest.mark.parametrize("W,H,K,sp,expect", [
    (320, 240, 0, 12, (12, 26, 20, 520)),          # 320 = 26*12 + 8, 240 = 20*12
    (481, 321, 1000, 0, (12, 40, 26, 1040)),       # sqrt(154401/1000) = 12.43 -> 12
    (3840, 2160, 20000, 0, (20, 192, 108, 20736)),  # sqrt(414.72) = 20.36 -> 20
    (481, 321, 0, 15, (15, 32, 21, 672)),
    (16, 16, 0, 16, (16, 1, 1, 1)),
    (100, 100, 100, 0, (10, 10, 10, 100)),         # exact square: sqrt(100) = 10
    (99, 100, 100, 0, (9, 11, 11, 121)),           # 9900/100 = 99 -> floor(sqrt) = 9
])
def test_grid_closed_forms(W, H, K, sp, expect):
    g = oracle.grid(W, H, K, sp)
    assert (g.v, g.nx, g.ny, g.K) == expect


@pytest.mark.parametrize("W,H,K,sp", [(320, 240, 1, 0), (10, 10, 0, 11), (0, 5, 3, 0), (5, 5, 0, 0)])
def test_grid_empty_is_rejected(W, H, K, sp):
    with pytest.raises(ValueError):
        oracle.grid(W, H, K, sp)


# ---------------------------------------------------------------- candidate sets
@pytest.mark.parametrize("W,H,v", [(16, 16, 3), (16, 16, 4), (16, 16, 5), (16, 16, 7), (23, 17, 4), (37, 23, 6)])
def test_candidates_match_brute_force(W, H, v):
    g = oracle.grid(W, H, spacing=v)
    cand, ncand = oracle.candidates(g)
    brute = brute_candidates(W, H, v, g.nx, g.ny)
    for i, ks in enumerate(brute):
        assert ncand[i] == len(ks)
        assert list(cand[i, :ncand[i]]) == ks
    # Sec. III-D: 1 <= |K_i| <= 9 and v^2 <= |I_k| <= 9 v^2
    assert ncand.min() >= 1 and ncand.max() <= 9
    sizes = np.bincount(np.concatenate([cand[i, :ncand[i]] for i in range(W * H)]), minlength=g.K)
    assert sizes.min() >= v * v and sizes.max() <= 9 * v * v


def test_candidates_remainder_strip_has_one_column():
    # 320 = 26*12 + 8: the 8 remainder columns can only come from k_x = n_x - 1.
    g = oracle.grid(320, 240, spacing=12)
    cand, ncand = oracle.candidates(g)
    x = 315
    for y in (0, 100, 239):
        ks = cand[y * 320 + x, :ncand[y * 320 + x]]
        assert set(k % g.nx for k in ks) == {g.nx - 1}


# ---------------------------------------------------------------- CIELAB
def test_cielab_anchor_colours():
    rows = np.loadtxt("tests/golden/cielab_srgb_d65_anchors.txt", comments="#")
    rgb = rows[:, :3].astype(np.uint8)
    lab = oracle.rgb2lab(rgb)
    for (exp, tol, got) in zip(rows[:, 3:6], rows[:, 6], lab):
        np.testing.assert_allclose(got, exp, atol=tol)


def test_cielab_greys_closed_form():
    # A grey (c, c, c) has a = b = 0 and L = 116 f(Y) - 16 with Y the decoded c.
    c = np.arange(256)
    rgb = np.stack([c, c, c], 1).astype(np.uint8)
    lab = oracle.rgb2lab(rgb)
    s = c / 255.0
    Y = np.where(s <= 0.04045, s / 12.92, ((s + 0.055) / 1.055) ** 2.4)
    d = 6 / 29
    f = np.where(Y > d ** 3, np.cbrt(Y), Y / (3 * d * d) + 4 / 29)
    np.testing.assert_allclose(lab[:, 0], 116 * f - 16, atol=1e-9)
    np.testing.assert_allclose(lab[:, 1:], 0.0, atol=2e-4)


# ---------------------------------------------------------------- init
def test_init_centre_pixels():
    W, H = 37, 23
    rng = np.random.default_rng(1)
    lab = rng.uniform(-50, 100, size=(H, W, 3))
    g = oracle.grid(W, H, spacing=6)
    th = oracle.init_theta(lab, g, lambda_c=8.0)
    for k in range(g.K):
        kx, ky = k % g.nx, k // g.nx
        x, y = kx * 6 + 3, ky * 6 + 3
        np.testing.assert_array_equal(th.mu[k], [x, y, *lab[y, x]])
        np.testing.assert_array_equal(th.cs[k], [36, 0, 36])
        np.testing.assert_array_equal(th.cc[k], [64, 0, 0, 64, 0, 64])


# ---------------------------------------------------------------- E-step
@pytest.mark.parametrize("W,H,v,seed", [(16, 16, 3, 0), (16, 16, 4, 1), (16, 16, 5, 2), (16, 16, 7, 3), (19, 17, 5, 4)])
def test_estep_matches_full_mixture(W, H, v, seed):
    rng = np.random.default_rng(seed)
    lab = rng.uniform([0, -60, -60], [100, 60, 60], size=(H, W, 3))
    g = oracle.grid(W, H, spacing=v)
    th = random_theta(rng, g, lab)
    R, ll, L, cand, ncand = oracle.estep(lab, g, th)
    z = pixel_z(W, H, lab)
    # log p(z_i; theta_k) for ALL k with scipy, then the Eq. (Ik) mask.
    logp = np.stack([multivariate_normal(th.mu[k], blocks_to_full(th.cs[k], th.cc[k])).logpdf(z)
                     for k in range(g.K)], axis=1)
    mask = np.array([[in_window(k % g.nx, v, W, i % W) and in_window(k // g.nx, v, H, i // W)
                      for k in range(g.K)] for i in range(W * H)])
    lm = np.where(mask, logp, -np.inf)
    lse = logsumexp(lm, axis=1)
    post = np.exp(lm - lse[:, None])
    np.testing.assert_allclose(ll, lse, rtol=1e-12, atol=1e-10)
    np.testing.assert_allclose(L, lse.sum(), rtol=1e-12)
    for i in range(W * H):
        got = np.zeros(g.K)
        got[cand[i, :ncand[i]]] = R[i, :ncand[i]]
        np.testing.assert_allclose(got, post[i], atol=1e-12)
    np.testing.assert_allclose(R.sum(1), 1.0, atol=1e-13)


def test_log_gauss_matches_scipy():
    rng = np.random.default_rng(5)
    for _ in range(20):
        S = random_spd(rng, 2, 10.0)
        C = random_spd(rng, 3, 40.0)
        mu = rng.normal(size=5) * 10
        z = mu + rng.normal(size=5) * 5
        cs = [S[0, 0], S[0, 1], S[1, 1]]
        cc = [C[0, 0], C[0, 1], C[0, 2], C[1, 1], C[1, 2], C[2, 2]]
        ref = multivariate_normal(mu, blocks_to_full(cs, cc)).logpdf(z)
        assert abs(oracle.log_gauss(z, mu, cs, cc) - ref) < 1e-11


# ---------------------------------------------------------------- M-step
@pytest.mark.parametrize("W,H,v,seed", [(16, 16, 4, 0), (16, 16, 5, 1), (23, 17, 4, 2)])
def test_mstep_matches_weighted_moments(W, H, v, seed):
    rng = np.random.default_rng(seed)
    lab = rng.uniform([0, -60, -60], [100, 60, 60], size=(H, W, 3))
    g = oracle.grid(W, H, spacing=v)
    cand, ncand = oracle.candidates(g)
    # Any posteriors that are non-negative and sum to one over K_i define an M-step.
    R = np.zeros((W * H, 9))
    for i in range(W * H):
        w = rng.uniform(0.05, 1.0, size=ncand[i])
        R[i, :ncand[i]] = w / w.sum()
    th0 = oracle.init_theta(lab, g)
    eps_s, eps_c = 2.0, 8.0
    th, cs_raw, cc_raw, wsum, dead, _ = oracle.mstep(lab, g, th0, R, cand, ncand, eps_s, eps_c)
    assert dead == 0
    z = pixel_z(W, H, lab)
    for k in range(g.K):
        w = np.zeros(W * H)
        for i in range(W * H):
            for j in range(ncand[i]):
                if cand[i, j] == k:
                    w[i] = R[i, j]
        kx, ky = k % g.nx, k // g.nx
        inside = np.array([in_window(kx, v, W, i % W) and in_window(ky, v, H, i // W) for i in range(W * H)])
        assert np.all(w[~inside] == 0)
        np.testing.assert_allclose(wsum[k], w.sum(), rtol=1e-13)
        mu = np.average(z, axis=0, weights=w)
        np.testing.assert_allclose(th.mu[k], mu, rtol=1e-12, atol=1e-10)
        full = np.cov(z.T, aweights=w, bias=True)
        S, C = full[:2, :2], full[2:, 2:]
        np.testing.assert_allclose(unpack(cs_raw[k]), S, rtol=1e-10, atol=1e-9)
        np.testing.assert_allclose(unpack(cc_raw[k]), C, rtol=1e-10, atol=1e-9)
        for raw_blk, got, eps in ((S, th.cs[k], eps_s), (C, th.cc[k], eps_c)):
            lam, Q = np.linalg.eigh(raw_blk)
            ref = Q @ np.diag(np.maximum(lam, eps)) @ Q.T
            np.testing.assert_allclose(unpack(got), ref, rtol=1e-9, atol=1e-9)


def test_single_gaussian_is_sample_moments():
    # K = 1 (16x16 at v = 16): R == 1, so one M-step gives the sample mean and
    # the (biased) sample covariance blocks, floored.
    rng = np.random.default_rng(7)
    lab = rng.uniform([0, -60, -60], [100, 60, 60], size=(16, 16, 3))
    res = oracle.em(lab, 16, 16, spacing=16, T=1, keep_post=True)
    assert res.grid.K == 1
    np.testing.assert_array_equal(res.post[:, 0], 1.0)
    z = pixel_z(16, 16, lab)
    np.testing.assert_allclose(res.theta.mu[0], z.mean(0), rtol=1e-13)
    full = np.cov(z.T, bias=True)
    for blk, got, eps in ((full[:2, :2], res.theta.cs[0], 2.0), (full[2:, 2:], res.theta.cc[0], 8.0)):
        lam, Q = np.linalg.eigh(blk)
        np.testing.assert_allclose(unpack(got), Q @ np.diag(np.maximum(lam, eps)) @ Q.T, rtol=1e-10)
    # x and y of a full 16x16 grid: variance (16^2 - 1) / 12, no covariance
    np.testing.assert_allclose(unpack(res.theta.cs[0]), np.diag([255 / 12, 255 / 12]), atol=1e-12)


def test_constant_colour_gives_floor():
    lab = np.zeros((24, 36, 3))
    lab[...] = [50.0, 10.0, -20.0]
    res = oracle.em(lab, 36, 24, spacing=6, T=3)
    for k in range(res.grid.K):
        np.testing.assert_allclose(res.theta.mu[k, 2:], [50, 10, -20], atol=1e-12)
        np.testing.assert_allclose(unpack(res.theta.cc[k]), 8.0 * np.eye(3), atol=1e-12)


# ---------------------------------------------------------------- eigenvalue floor
def test_clamp_diagonal_is_elementwise_max():
    for d, eps in (([1.0, 5.0], 2.0), ([3.0, 0.5], 2.0), ([0.1, 0.2], 2.0)):
        out, raised = oracle.eig_clamp([d[0], 0.0, d[1]], eps)
        np.testing.assert_allclose(out, [max(d[0], eps), 0.0, max(d[1], eps)], atol=1e-15)
        assert raised == sum(x < eps for x in d)
    out, raised = oracle.eig_clamp([1.0, 0, 0, 20.0, 0, 4.0], 8.0)
    np.testing.assert_allclose(out, [8.0, 0, 0, 20.0, 0, 8.0], atol=1e-14)
    assert raised == 2


def test_clamp_random_spd_matches_eigh():
    rng = np.random.default_rng(11)
    for n, eps in ((2, 2.0), (3, 8.0)):
        for _ in range(200):
            A = random_spd(rng, n, rng.uniform(0.5, 30.0))
            if rng.uniform() < 0.2:  # exact multiple eigenvalues
                A = rng.uniform(0.1, 20) * np.eye(n)
            p = A[np.triu_indices(n)]
            out, _ = oracle.eig_clamp(p, eps)
            lam, Q = np.linalg.eigh(A)
            ref = Q @ np.diag(np.maximum(lam, eps)) @ Q.T
            np.testing.assert_allclose(unpack(out), ref, rtol=1e-11, atol=1e-11)
            assert oracle.sym_eigvals(out).min() >= eps - 1e-12
            np.testing.assert_allclose(oracle.sym_eigvals(p), lam, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- whole loop
def test_em_invariants_config0():
    img = voronoi_image(320, 240, 40, 8.0, seed=0)
    lab = oracle.rgb2lab(img)
    res = oracle.em(lab, 320, 240, spacing=12, T=10, keep_post=True)
    np.testing.assert_allclose(res.post.sum(1), 1.0, atol=1e-12)
    lab_flat = res.labels.ravel()
    member = (res.cand == lab_flat[:, None]) & (np.arange(9)[None, :] < res.ncand[:, None])
    assert member.any(1).all()                      # every label lies in K_i
    assert res.dead == 0
    # label = argmax posterior, ties to the smaller k (candidates are ascending)
    best = res.cand[np.arange(len(lab_flat)), np.argmax(np.where(
        np.arange(9)[None, :] < res.ncand[:, None], res.post, -1.0), axis=1)]
    np.testing.assert_array_equal(best, lab_flat)


def test_loglik_non_decreasing_when_floor_inactive():
    # Sec. III-B: E makes Q equal to L, M maximises Q, so L cannot decrease.
    img = voronoi_image(96, 72, 12, 8.0, seed=3)
    lab = oracle.rgb2lab(img)
    res = oracle.em(lab, 96, 72, spacing=8, T=10, eps_s=1e-9, eps_c=1e-9)
    assert res.raised.sum() == 0
    d = np.diff(res.loglik)
    assert np.all(d >= -1e-9 * np.abs(res.loglik[1:])), res.loglik


def test_loglik_non_decreasing_with_floor():
    # With the floor, the floored covariance is still the maximiser of Q over
    # {Sigma : eigenvalues >= eps} (eigenvalue-wise maximisation), and theta_0
    # is feasible, so L is non-decreasing as well.
    img = voronoi_image(320, 240, 40, 8.0, seed=0)
    lab = oracle.rgb2lab(img)
    res = oracle.em(lab, 320, 240, spacing=12, T=10)
    assert res.raised.sum() > 0
    d = np.diff(res.loglik)
    assert np.all(d >= -1e-9 * np.abs(res.loglik[1:])), res.loglik


def test_thread_count_does_not_change_results():
    img = voronoi_image(160, 120, 20, 8.0, seed=9)
    lab = oracle.rgb2lab(img)
    n = oracle.max_threads()
    try:
        oracle.set_threads(1)
        a = oracle.em(lab, 160, 120, spacing=10, T=4)
        oracle.set_threads(max(2, n))
        b = oracle.em(lab, 160, 120, spacing=10, T=4)
    finally:
        oracle.set_threads(n)
    np.testing.assert_array_equal(a.theta.mu, b.theta.mu)
    np.testing.assert_array_equal(a.theta.cc, b.theta.cc)
    np.testing.assert_array_equal(a.labels, b.labels)
    np.testing.assert_array_equal(a.loglik, b.loglik)


def test_resume_equals_uninterrupted():
    img = voronoi_image(120, 96, 16, 8.0, seed=4)
    lab = oracle.rgb2lab(img)
    full = oracle.em(lab, 120, 96, spacing=12, T=6)
    half = oracle.em(lab, 120, 96, spacing=12, T=3)
    rest = oracle.em(lab, 120, 96, spacing=12, T=3, theta0=half.theta)
    np.testing.assert_array_equal(full.theta.mu, rest.theta.mu)
    np.testing.assert_array_equal(full.labels, rest.labels)
    np.testing.assert_allclose(full.loglik[3:], rest.loglik, rtol=0, atol=0)


def test_generator_is_seeded():
    a = voronoi_image(64, 48, 5, 8.0, seed=1)
    b = voronoi_image(64, 48, 5, 8.0, seed=1)
    c = voronoi_image(64, 48, 5, 8.0, seed=2)
    assert a.dtype == np.uint8 and a.shape == (48, 64, 3)
    np.testing.assert_array_equal(a, b)
    assert (a != c).any()
