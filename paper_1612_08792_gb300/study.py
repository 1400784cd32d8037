"""Parameter and colour-model studies on synthetic images.

Sec. IV-B of the paper studies the initial colour deviation lambda and the
colour eigenvalue floor eps_c (values 2, 4, 6, 8, 10 each, at several
superpixel counts, scored by BR, UE and ASA), and Sec. III-C suggests the L |
(a, b) split of Eq. (BlockSigma1) to save computation.  The paper runs its
studies on BSDS500, which is not available here; these run on the seeded
synthetic Voronoi images of the training and evaluation workload (481x321,
150 regions, noise sigma 8, held-out seeds), whose region map is the ground
truth.  Every segmentation and every score runs in the library's kernels
(batch contexts, gmmsp_segmentation_metrics_many); this module only sequences
the calls.

Command line:
    python -m paper_1612_08792_gb300.study sweep --param eps_c --values 2 4 6 8 10
    python -m paper_1612_08792_gb300.study sweep --param lambda_c --values 2 4 6 8 10
    python -m paper_1612_08792_gb300.study colour
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import SuperpixelsBatch, gmmsp_segmentation_metrics_many
from .learned_init import HELD_OUT_SEED0, TRAIN

SPACINGS = (10, 15, 20, 30)   # 1,536 / 672 / 384 / 160 superpixels at 481x321


def _images(seeds, buf, regs):
    from synth.voronoi_torch import voronoi_batch
    voronoi_batch(TRAIN["W"], TRAIN["H"], TRAIN["regions"], TRAIN["sigma"], seeds, out=buf, regions_out=regs)
    return [buf[i] for i in range(buf.shape[0])]


def _scores(labels, regs, K, take):
    acc = {"br": [], "ue": [], "asa": []}
    for m in gmmsp_segmentation_metrics_many(list(labels[:take]), [regs[i] for i in range(take)], K,
                                             TRAIN["regions"]):
        for key in acc:
            acc[key].append(m[key])
    return acc


def sweep(param: str = "eps_c", values=(2, 4, 6, 8, 10), spacings=SPACINGS, n_images: int = 64,
          iters: int = 10, colour: str = "full", batch: int = 64, seed0: int = HELD_OUT_SEED0):
    """Mean BR (radius 2), UE (eps 0.05) and ASA over n_images held-out images, and the mean
    log-likelihood per pixel, for each value of `param` ("eps_c" or "lambda_c"; the other
    stays at the paper's 8) and each spacing.  Returns a list of rows."""
    import torch
    if param not in ("eps_c", "lambda_c"):
        raise ValueError("param must be eps_c or lambda_c")
    W, H = TRAIN["W"], TRAIN["H"]
    nb = min(batch, n_images)
    buf = torch.empty((nb, H, W, 3), dtype=torch.uint8, device="cuda")
    regs = torch.empty((nb, H, W), dtype=torch.int32, device="cuda")
    rows = []
    for v in spacings:
        K = (W // v) * (H // v)
        for val in values:
            kw = {"eps_c": 8.0, "lambda_c": 8.0}
            kw[param] = float(val)
            bt = SuperpixelsBatch([(H, W)] * nb, spacing=v, colour=colour, **kw)
            acc = {"br": [], "ue": [], "asa": []}
            ll = []
            for s0 in range(0, n_images, nb):
                take = min(nb, n_images - s0)
                imgs = _images([seed0 + s0 + i for i in range(nb)], buf, regs)
                labels, lls = bt.segment(imgs, iters=iters, want_loglik=True)
                ll += list(np.asarray(lls[:take]) / (W * H))
                for key, vals in _scores(labels, regs, K, take).items():
                    acc[key] += vals
            bt.close()
            rows.append({param: float(val), "spacing": v, "K": K, "images": n_images, "iters": iters,
                         "colour": colour, "loglik_per_pixel": float(np.mean(ll)),
                         **{key: float(np.mean(vals)) for key, vals in acc.items()}})
    return rows


def colour_models(n_images: int = 256, iters: int = 10, spacing: int = 15, reps: int = 5,
                  seed0: int = HELD_OUT_SEED0, models=("full", "split", "gray")):
    """The three colour models on the same n_images held-out images in one batch: step
    time (CUDA events around the graph-captured segment, best of `reps`), throughput,
    the autotuned E + M pass time, mean log-likelihood per pixel (grayscale's is that of
    a 3-dimensional model: not comparable with the colour models'), and BR / UE / ASA."""
    import torch
    W, H = TRAIN["W"], TRAIN["H"]
    K = (W // spacing) * (H // spacing)
    buf = torch.empty((n_images, H, W, 3), dtype=torch.uint8, device="cuda")
    regs = torch.empty((n_images, H, W), dtype=torch.int32, device="cuda")
    imgs = _images([seed0 + i for i in range(n_images)], buf, regs)
    out = {}
    stream = torch.cuda.current_stream()
    for colour in models:
        bt = SuperpixelsBatch([(H, W)] * n_images, spacing=spacing, colour=colour)
        bps, tune = bt.autotune(imgs, reps=3)
        bt.segment(imgs, iters=iters)
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bt.segment(imgs, iters=iters)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        labels, ll = bt.segment(imgs, iters=iters, want_loglik=True)
        acc = _scores(labels, regs, K, n_images)
        ms = min(times)
        out[colour] = {"step_ms": ms, "mpix_per_s": n_images * W * H / (ms * 1e3),
                       "em_pass_ms": tune[bps], "blocks_per_sm": bps,
                       "loglik_per_pixel": float(np.mean(ll)) / (W * H),
                       **{key: float(np.mean(vals)) for key, vals in acc.items()}}
        bt.close()
    return {"images": n_images, "iters": iters, "spacing": spacing, "K": K, "models": out}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    sub = ap.add_subparsers(dest="cmd", required=True)
    sw = sub.add_parser("sweep")
    sw.add_argument("--param", default="eps_c", choices=["eps_c", "lambda_c"])
    sw.add_argument("--values", type=float, nargs="+", default=[2, 4, 6, 8, 10])
    sw.add_argument("--spacings", type=int, nargs="+", default=list(SPACINGS))
    sw.add_argument("--images", type=int, default=64)
    sw.add_argument("--colour", default="full", choices=["full", "split", "gray"])
    co = sub.add_parser("colour")
    co.add_argument("--images", type=int, default=256)
    co.add_argument("--spacing", type=int, default=15)
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    if args.cmd == "sweep":
        res = sweep(args.param, args.values, args.spacings, args.images, colour=args.colour)
    else:
        res = colour_models(args.images, spacing=args.spacing)
    print(json.dumps(res, indent=1))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
