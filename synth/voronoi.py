"""Seeded Voronoi test images standing in for the paper's photographs.

The paper evaluates on BSDS500 (481x321 photographs), which is not available
here; these images have the same shapes and a piecewise-smooth structure:

  * ``regions`` Voronoi sites drawn uniformly in the image; each pixel takes
    the colour of its nearest site (ties cannot occur with continuous sites);
  * each region has a constant colour uniform in [0, 255]^3 plus a linear
    gradient: a random direction and a per-channel amplitude uniform in
    [0, 30] levels over the image extent;
  * i.i.d. Gaussian noise of standard deviation ``sigma``, then rounding and
    clipping to uint8.

Everything is drawn from ``numpy.random.default_rng(seed)`` in a fixed order,
so an image is a pure function of its arguments.
"""
from __future__ import annotations

import numpy as np

try:  # scipy is present on both machines; fall back to a blocked numpy search.
    from scipy.spatial import cKDTree as _KDTree
except Exception:  # pragma: no cover
    _KDTree = None


def _nearest_site(sites: np.ndarray, W: int, H: int) -> np.ndarray:
    ys, xs = np.mgrid[0:H, 0:W]
    pts = np.stack([xs.ravel(), ys.ravel()], axis=1).astype(np.float64)
    if _KDTree is not None:
        _, idx = _KDTree(sites).query(pts)
        return idx.astype(np.int64).reshape(H, W)
    out = np.empty(len(pts), dtype=np.int64)
    step = 65536
    for s in range(0, len(pts), step):
        d = ((pts[s:s + step, None, :] - sites[None, :, :]) ** 2).sum(-1)
        out[s:s + step] = d.argmin(1)
    return out.reshape(H, W)


def voronoi_image(W: int, H: int, regions: int = 40, sigma: float = 8.0, seed: int = 0,
                  grad_max: float = 30.0, return_regions: bool = False):
    """(H, W, 3) uint8 sRGB image; optionally the (H, W) region map too."""
    rng = np.random.default_rng(seed)
    R = max(1, int(regions))
    sites = rng.uniform([0.0, 0.0], [W, H], size=(R, 2))
    base = rng.uniform(0.0, 255.0, size=(R, 3))
    angle = rng.uniform(0.0, 2.0 * np.pi, size=R)
    amp = rng.uniform(0.0, grad_max, size=(R, 3))
    reg = _nearest_site(sites, W, H)
    ys, xs = np.mgrid[0:H, 0:W]
    s = sites[reg]
    proj = ((xs - s[..., 0]) * np.cos(angle[reg]) + (ys - s[..., 1]) * np.sin(angle[reg])) / max(W, H)
    img = base[reg] + amp[reg] * proj[..., None]
    img = img + rng.normal(0.0, sigma, size=img.shape)
    img = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    if return_regions:
        return img, reg.astype(np.int32)
    return img


# Workload shapes of the benchmark and parity tests (see the design notes).
CONFIGS = {
    # 320x240, 40 regions, sigma 8, spacing 12 (K = 520), 10 iterations
    "c0": dict(W=320, H=240, regions=40, sigma=8.0, K=0, spacing=12, T=10),
    # 481x321, 150 regions, K = 1000 requested -> v = 12, K = 1040
    "c1": dict(W=481, H=321, regions=150, sigma=8.0, K=1000, spacing=0, T=10),
    # 3840x2160, 2000 regions, sigma 6, K = 20000 requested -> v = 20, K = 20736
    "c3": dict(W=3840, H=2160, regions=2000, sigma=6.0, K=20000, spacing=0, T=10),
    # 481x321 at spacing 15 (learned initialiser workload)
    "c4": dict(W=481, H=321, regions=150, sigma=8.0, K=0, spacing=15, T=10),
}

BATCH_SHAPES = [(320, 240), (481, 321), (640, 480), (1280, 720), (1920, 1080)]


def batch_sizes(n: int = 256, seed: int = 0):
    """Image sizes of the batched workload: uniform over the five shapes."""
    rng = np.random.default_rng(seed + 7919)
    idx = rng.integers(0, len(BATCH_SHAPES), size=n)
    return [BATCH_SHAPES[i] for i in idx]


def batch_regions(W: int, H: int) -> int:
    """Region count proportional to area (40 regions at 320x240)."""
    return max(1, int(round(40 * W * H / 76800)))
