"""The learned initialiser: network object, training and evaluation.

The network (include/gmmsp_cnn.h) predicts, per superpixel, the fitted mean's
offset from the Sec. III-C start and the log of the fitted covariance
diagonal.  It is trained here on synthetic images: each step draws a batch of
seeded Voronoi images on the device, fits them with many EM iterations
through a batch context (gmmsp_batch_segment), turns the fitted parameters
into targets (gmmsp_batch_targets) and takes one Adam step
(gmmsp_net_train_step).  Every step of that loop runs in the library's CUDA
kernels; this module only sequences the calls.

Command line:
    python -m paper_1612_08792_gb300.learned_init train --steps 2000 --out weights.npz
    python -m paper_1612_08792_gb300.learned_init eval --weights weights.npz
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np

from . import (SuperpixelsBatch, gmmsp_net_check, gmmsp_net_create, gmmsp_net_destroy, gmmsp_net_forward,
               gmmsp_net_get_adam, gmmsp_net_get_weights, gmmsp_net_grad, gmmsp_net_param_count,
               gmmsp_net_set_adam, gmmsp_net_set_weights, gmmsp_net_train_step, gmmsp_segmentation_metrics)

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS_DIR = os.path.join(HERE, "weights")
OUTPUTS, CHANNELS = 10, 16
# (taps, cout) of the six layers; every layer has 32 input channels
LAYERS = [(1, 32), (1, 32), (9, 32), (9, 32), (9, 32), (9, 16)]

# Training data: the 481 x 321 synthetic workload at spacing 15.
TRAIN = dict(W=481, H=321, regions=150, sigma=8.0, spacing=15)
HELD_OUT_SEED0 = 1_000_000


def layer_slices():
    """[(weight slice, bias slice, (cout, taps*32))] in the flat parameter vector."""
    out, o = [], 0
    for taps, cout in LAYERS:
        w = slice(o, o + cout * taps * 32)
        o += cout * taps * 32
        b = slice(o, o + cout)
        o += cout
        out.append((w, b, (cout, taps * 32)))
    return out


def init_weights(seed: int = 0) -> np.ndarray:
    """He-normal weights (input channels 27..31 of the first layer unused), zero biases,
    a small last layer."""
    rng = np.random.default_rng(seed)
    flat = np.zeros(gmmsp_net_param_count(), dtype=np.float32)
    for l, (ws, _, shape) in enumerate(layer_slices()):
        fan_in = 27 if l == 0 else shape[1]
        std = math.sqrt(2.0 / fan_in) * (0.1 if l == 5 else 1.0)
        W = rng.normal(0.0, std, shape).astype(np.float32)
        if l == 0:
            W[:, 27:] = 0.0
        flat[ws] = W.ravel()
    return flat


class InitNet:
    """A network on the device (gmmsp_net)."""

    def __init__(self, spacing: int = 15, weights=None, seed: int = 0, stream=None):
        import torch
        self.spacing = int(spacing)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.n = gmmsp_net_create(self.spacing, self.stream)
        self.set_weights(init_weights(seed) if weights is None else weights)

    def set_weights(self, w) -> None:
        gmmsp_net_set_weights(self.n, w)

    def get_weights(self) -> np.ndarray:
        return gmmsp_net_get_weights(self.n)

    def forward(self, lab, B: int, W: int, H: int):
        """Outputs (B, n_y, n_x, 16) float32 on the device for B images of CIELAB planes: a float32
        CUDA tensor, or a device address that stays valid until the queued work has run (an address
        whose tensor is dropped at once can be reused by the next allocation before the kernels read it)."""
        import torch
        nx, ny = W // self.spacing, H // self.spacing
        out = torch.empty((B, ny, nx, CHANNELS), dtype=torch.float32, device="cuda")
        gmmsp_net_forward(self.n, lab, B, W, H, out)
        return out

    def grad(self, lab, B: int, W: int, H: int, target):
        """(loss, flat gradient) for B images (a tensor or an address, as for forward)."""
        return gmmsp_net_grad(self.n, lab, B, W, H, target)

    def train_step(self, lab, B: int, W: int, H: int, target, lr: float, want_loss=True):
        return gmmsp_net_train_step(self.n, lab, B, W, H, target, lr, want_loss)

    def check(self) -> None:
        gmmsp_net_check(self.n)

    def save(self, path: str, meta: dict | None = None, optimizer: bool = False) -> None:
        """One .npz file: the weights, the spacing, `meta` and, with `optimizer`, the Adam
        moments and step count (a training checkpoint that resumes exactly)."""
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        extra = {}
        if optimizer:
            m, v, step = gmmsp_net_get_adam(self.n)
            extra = dict(adam_m=m, adam_v=v, adam_step=step)
        np.savez(path, weights=self.get_weights(), spacing=self.spacing, meta=json.dumps(meta or {}), **extra)

    @classmethod
    def load(cls, path: str, stream=None) -> "InitNet":
        """A network from save(); the optimiser state too when the file holds it."""
        z = np.load(path)
        net = cls(int(z["spacing"]), weights=z["weights"], stream=stream)
        if "adam_m" in z.files:
            gmmsp_net_set_adam(net.n, z["adam_m"], z["adam_v"], int(z["adam_step"]))
        return net

    def close(self) -> None:
        if getattr(self, "n", None):
            gmmsp_net_destroy(self.n)
            self.n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pretrained_path(spacing: int = 15) -> str:
    return os.path.join(WEIGHTS_DIR, f"init_net_v{spacing}.npz")


def load_pretrained(spacing: int = 15, stream=None) -> InitNet:
    return InitNet.load(pretrained_path(spacing), stream=stream)


def _images(seeds, buf, regions_out=None):
    from synth.voronoi_torch import voronoi_batch
    voronoi_batch(TRAIN["W"], TRAIN["H"], TRAIN["regions"], TRAIN["sigma"], seeds, out=buf,
                  regions_out=regions_out)
    return [buf[i] for i in range(buf.shape[0])]


def train(steps: int = 2000, batch: int = 32, lr: float = 3e-3, lr_final: float = 5e-5, n_train: int = 20000,
          target_iters: int = 20, seed: int = 0, log_every: int = 100, log=print, net: InitNet | None = None):
    """Trains (or continues training) a network on the synthetic 481 x 321 workload.

    Training images are the seeds 0 .. n_train - 1 (visited in a seeded random
    order, batch images per step); targets come from target_iters EM iterations."""
    import torch
    W, H, v = TRAIN["W"], TRAIN["H"], TRAIN["spacing"]
    K = (W // v) * (H // v)
    net = net or InitNet(v, seed=seed)
    bt = SuperpixelsBatch([(H, W)] * batch, spacing=v)
    tgt = torch.empty(batch * K * OUTPUTS, dtype=torch.float32, device="cuda")
    buf = torch.empty((batch, H, W, 3), dtype=torch.uint8, device="cuda")
    order = np.random.default_rng(seed + 1).permutation(n_train)
    history = []
    t0 = time.time()
    for step in range(steps):
        seeds = [int(order[(step * batch + i) % n_train]) for i in range(batch)]
        imgs = _images(seeds, buf)
        bt.segment(imgs, iters=target_iters)
        bt.targets(tgt)
        if step == 0 and net is not None and np.all(net.get_weights()[layer_slices()[5][1]] == 0):
            # start the output biases at the mean target
            w = net.get_weights()
            mean = tgt.view(-1, OUTPUTS).mean(0).cpu().numpy()
            b6 = layer_slices()[5][1]
            w[b6.start:b6.start + OUTPUTS] = mean
            net.set_weights(w)
        frac = step / max(1, steps - 1)
        lr_t = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * frac))
        want = (step % log_every == 0) or step == steps - 1
        loss = net.train_step(bt.lab_ptr(), batch, W, H, tgt, lr_t, want_loss=want)
        if want:
            history.append((step, loss))
            log(f"step {step:5d}  loss {loss:.5f}  lr {lr_t:.2e}  {time.time() - t0:.1f}s")
    net.check()
    bt.close()
    return net, history


def evaluate(net: InitNet, n_images: int = 64, seed0: int = HELD_OUT_SEED0, plain_iters=(2, 3, 10),
             learned_iters=(2,), batch: int = 64, accuracy: bool = True):
    """Held-out images, for the paper's start (plain) and the network's start
    (learned):
      * the mean per-pixel log-likelihood L(theta_T) / (W H);
      * the fraction of pixels whose label after each learned run equals the
        label after the longest plain run;
      * with `accuracy`, the mean BR, UE and ASA (Sec. IV) against the
        generator's regions."""
    import torch
    W, H, v = TRAIN["W"], TRAIN["H"], TRAIN["spacing"]
    K = (W // v) * (H // v)
    runs = [f"plain{t}" for t in plain_iters] + [f"learned{t}" for t in learned_iters]
    res = {r: [] for r in runs}
    acc = {r: {"br": [], "ue": [], "asa": []} for r in runs}
    agree = {f"learned{t}": 0 for t in learned_iters}
    ref_t = max(plain_iters)
    nb = min(batch, n_images)
    buf = torch.empty((nb, H, W, 3), dtype=torch.uint8, device="cuda")
    regs = torch.empty((nb, H, W), dtype=torch.int32, device="cuda")
    bt = SuperpixelsBatch([(H, W)] * nb, spacing=v)
    done = 0

    def score(run, labels, take):
        if not accuracy:
            return
        for i in range(take):
            m = gmmsp_segmentation_metrics(labels[i], regs[i], K, TRAIN["regions"])
            for key in ("br", "ue", "asa"):
                acc[run][key].append(m[key])

    for s0 in range(0, n_images, nb):
        seeds = [seed0 + s0 + i for i in range(nb)]
        imgs = _images(seeds, buf, regs)
        take = min(nb, n_images - s0)
        bt.set_init_net(None)
        ref_labels = None
        for t in plain_iters:
            labels, ll = bt.segment(imgs, iters=t, want_loglik=True)
            res[f"plain{t}"] += list(ll[:take] / (W * H))
            score(f"plain{t}", labels, take)
            if t == ref_t:
                ref_labels = [x.clone() for x in labels[:take]]
        bt.set_init_net(net)
        for t in learned_iters:
            labels, ll = bt.segment(imgs, iters=t, want_loglik=True)
            res[f"learned{t}"] += list(ll[:take] / (W * H))
            score(f"learned{t}", labels, take)
            agree[f"learned{t}"] += sum(int((a == b).sum().item()) for a, b in zip(labels[:take], ref_labels))
        bt.set_init_net(None)
        done += take
    bt.close()
    out = {k: float(np.mean(v_)) for k, v_ in res.items()}
    out.update({f"label_agreement_{k}_vs_plain{ref_t}": a / (done * W * H) for k, a in agree.items()})
    if accuracy:
        out["accuracy"] = {r: {k: float(np.mean(v_)) for k, v_ in d.items()} for r, d in acc.items()}
    out["images"] = done
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train")
    tr.add_argument("--steps", type=int, default=2000)
    tr.add_argument("--batch", type=int, default=32)
    tr.add_argument("--lr", type=float, default=3e-3)
    tr.add_argument("--seed", type=int, default=0)
    tr.add_argument("--out", default=pretrained_path(15))
    tr.add_argument("--eval-images", type=int, default=64)
    ev = sub.add_parser("eval")
    ev.add_argument("--weights", default=pretrained_path(15))
    ev.add_argument("--images", type=int, default=64)
    ev.add_argument("--plain", default="2,3,10", help="plain-EM iteration counts (comma separated)")
    ev.add_argument("--learned", default="2", help="iteration counts after the learned start")
    args = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    if args.cmd == "train":
        t0 = time.time()
        net, hist = train(steps=args.steps, batch=args.batch, lr=args.lr, seed=args.seed)
        secs = time.time() - t0
        ev = evaluate(net, n_images=args.eval_images)
        meta = dict(steps=args.steps, batch=args.batch, lr=args.lr, seed=args.seed, train_seconds=round(secs, 1),
                    history=hist, heldout=ev, workload=TRAIN, target_iters=20)
        net.save(args.out, meta)
        print(json.dumps({"train_seconds": round(secs, 1), "final_loss": hist[-1][1], "heldout": ev}))
    else:
        net = InitNet.load(args.weights)
        print(json.dumps(evaluate(net, n_images=args.images,
                                  plain_iters=tuple(int(t) for t in args.plain.split(",")),
                                  learned_iters=tuple(int(t) for t in args.learned.split(",")))))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
