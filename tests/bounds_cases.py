"""Small cases of every EM entry point, run against the library that GMMSP_LIBRARY names
(tests/test_gpu_bounds.py points it at the bounds-checked build).  Prints one JSON line:
the bounds status after each case and the parity of a few results against the oracle."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    import torch
    import oracle
    import paper_1612_08792_gb300 as gm
    from paper_1612_08792_gb300.learned_init import load_pretrained
    from synth import voronoi_image
    from tests import parity

    torch.cuda.set_device(0)
    out = {"library": gm.library_path(), "cases": []}

    def status(name, extra=None):
        checked, viol = gm.gmmsp_bounds_status()
        rec = {"case": name, "checked": checked, "violation": viol}
        rec.update(extra or {})
        out["cases"].append(rec)

    def lab_of(W, H, seed, regions=12):
        return oracle.rgb2lab(voronoi_image(W, H, regions, 8.0, seed)).astype(np.float32)

    # single images, every launch shape, against the oracle
    for (W, H, v) in [(16, 16, 4), (37, 23, 5), (97, 61, 8), (70, 52, 8)]:
        lab = lab_of(W, H, 3)
        ref = oracle.em(lab.astype(np.float64), W, H, spacing=v, T=3)
        for wpc in (1, 2, 4):
            sp = gm.Superpixels(torch.from_numpy(lab).cuda(), spacing=v)
            sp.set_launch(wpc)
            sp.em_iters(3, want_loglik=True)
            labels, _ = sp.labels(want_loglik=True)
            mu, cs, cc = sp.get_params()
            sp.close()
            agree, _, worst = parity.label_report(labels.cpu().numpy(), ref.labels, ref.margin)
            status(f"single {W}x{H} v={v} wpc={wpc}",
                   {"mean_err": parity.mean_rel_err(mu, ref.theta.mu), "agree": agree, "worst_margin": worst})
    # a batch of uneven sizes at every launch variant
    sizes = [(37, 23), (97, 61), (320, 240), (481, 321)]
    labs = [lab_of(W, H, 10 + i, regions=max(4, W * H // 1000)) for i, (W, H) in enumerate(sizes)]
    dev = [torch.from_numpy(x).cuda() for x in labs]
    ref3 = oracle.em(labs[3].astype(np.float64), 481, 321, spacing=8, T=3)
    for bps in (3, 5, 6, 7):
        for fin16 in (False, True):
            bt = gm.SuperpixelsBatch([(H, W) for (W, H) in sizes], spacing=8, lab_input=True)
            gm.gmmsp_batch_set_tuning(bt.b, bps, fin16)
            labels, _ = bt.segment(dev, iters=3, want_loglik=True)
            torch.cuda.synchronize()
            mu, _, _ = bt.get_params(3, ref3.grid.K)
            agree, _, worst = parity.label_report(labels[3].cpu().numpy(), ref3.labels, ref3.margin)
            bt.close()
            status(f"batch bps={bps} fin16={fin16}",
                   {"mean_err": parity.mean_rel_err(mu, ref3.theta.mu), "agree": agree, "worst_margin": worst})
    # the allocation-free entry point with padded rows
    W, H = 97, 61
    padded = np.zeros((H, W + 3, 3), dtype=np.float32)
    padded[:, :W] = lab_of(W, H, 20)
    p = gm.gmmsp_default_params()
    p.spacing = 8
    lt = torch.empty((H, W), dtype=torch.int32, device="cuda")
    gm.gmmsp_segment_lab_noalloc(torch.from_numpy(padded).cuda(), W, H, (W + 3) * 12, p, 3, lt)
    torch.cuda.synchronize()
    status("noalloc 97x61 pitched")
    # the learned start and the RGB path
    imgs = [torch.from_numpy(voronoi_image(96, 64, 8, 8.0, 200 + i)).cuda() for i in range(2)]
    net = load_pretrained(15)
    bt = gm.SuperpixelsBatch([(64, 96)] * 2, spacing=15)
    bt.set_init_net(net)
    bt.segment(imgs, iters=2, want_loglik=True)
    torch.cuda.synchronize()
    bt.close()
    net.close()
    status("learned start 2 x 96x64")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
