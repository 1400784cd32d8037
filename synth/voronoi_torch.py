"""Seeded Voronoi images generated on a CUDA device (for training data).

Same recipe as ``voronoi.voronoi_image``: the sites, region colours,
gradient directions and amplitudes are the very same numpy draws for a given
seed, so the region map matches ``voronoi_image`` (up to floating-point ties
at region borders); the Gaussian noise is drawn on the device from a
``torch.Generator`` seeded with the same seed, so it is a different
realisation of the same distribution.  Holds none of the method's
arithmetic.
"""
from __future__ import annotations

import numpy as np


def _draws(W: int, H: int, regions: int, seed: int, grad_max: float):
    rng = np.random.default_rng(seed)
    R = max(1, int(regions))
    sites = rng.uniform([0.0, 0.0], [W, H], size=(R, 2))
    base = rng.uniform(0.0, 255.0, size=(R, 3))
    angle = rng.uniform(0.0, 2.0 * np.pi, size=R)
    amp = rng.uniform(0.0, grad_max, size=(R, 3))
    return sites, base, angle, amp


def voronoi_batch(W: int, H: int, regions: int, sigma: float, seeds, device="cuda", grad_max: float = 30.0,
                  out=None, regions_out=None):
    """(B, H, W, 3) uint8 tensor on `device`, image i drawn from seeds[i].  With
    regions_out (a (B, H, W) int32 tensor) the region (Voronoi site) map of every
    image is written there too: the ground truth of the accuracy metrics."""
    import torch
    seeds = list(seeds)
    if out is None:
        out = torch.empty((len(seeds), H, W, 3), dtype=torch.uint8, device=device)
    ys = torch.arange(H, device=device, dtype=torch.float64)[:, None]
    xs = torch.arange(W, device=device, dtype=torch.float64)[None, :]
    gen = torch.Generator(device=device)
    for i, seed in enumerate(seeds):
        sites, base, angle, amp = _draws(W, H, regions, int(seed), grad_max)
        s = torch.from_numpy(sites).to(device)
        # nearest site (the first of equal distances), sites in chunks of ~64M distances
        best = torch.full((H, W), float("inf"), dtype=torch.float64, device=device)
        reg = torch.zeros((H, W), dtype=torch.int64, device=device)
        step = max(1, (1 << 26) // (H * W))
        for r0 in range(0, len(sites), step):
            c = s[r0:r0 + step]
            d = (xs[None] - c[:, 0, None, None]) ** 2 + (ys[None] - c[:, 1, None, None]) ** 2
            dmin, arg = d.min(dim=0)
            closer = dmin < best
            best = torch.where(closer, dmin, best)
            reg = torch.where(closer, arg + r0, reg)
        sx, sy = s[reg, 0], s[reg, 1]
        a = torch.from_numpy(angle).to(device)[reg]
        proj = ((xs - sx) * torch.cos(a) + (ys - sy) * torch.sin(a)) / max(W, H)
        img = torch.from_numpy(base).to(device)[reg] + torch.from_numpy(amp).to(device)[reg] * proj[..., None]
        gen.manual_seed(int(seed))
        img = img + sigma * torch.randn(img.shape, generator=gen, device=device, dtype=torch.float64)
        out[i] = torch.clamp(torch.round(img), 0, 255).to(torch.uint8)
        if regions_out is not None:
            regions_out[i] = reg.to(torch.int32)
    return out
