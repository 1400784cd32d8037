"""Comparison helpers for CUDA-vs-oracle parity (the tolerances live here).

Tolerances (from the target for this path):
  * means: |mu_gpu - mu_ref| / max(|mu_ref|, 1) <= 1e-4 per component;
  * covariances: ||Sigma_gpu - Sigma_ref||_F / ||Sigma_ref||_F <= 1e-4 per block;
  * labels: >= 99.9 % agreement, and a disagreement only where the oracle's
    posterior margin R_(1) - R_(2) is small (MARGIN_TOL);
  * log-likelihood per E-step: relative 1e-6 (FP32 E-step, FP64 sums).
"""
import numpy as np

MEAN_TOL = 1e-4
COV_TOL = 1e-4
LABEL_AGREE = 0.999
MARGIN_TOL = 1e-5
LL_RTOL = 1e-6


def unpack(p):
    p = np.asarray(p)
    if p.shape[-1] == 3:
        return np.stack([np.stack([p[..., 0], p[..., 1]], -1), np.stack([p[..., 1], p[..., 2]], -1)], -2)
    return np.stack([np.stack([p[..., 0], p[..., 1], p[..., 2]], -1),
                     np.stack([p[..., 1], p[..., 3], p[..., 4]], -1),
                     np.stack([p[..., 2], p[..., 4], p[..., 5]], -1)], -2)


def mean_rel_err(mu, mu_ref):
    return float(np.max(np.abs(mu - mu_ref) / np.maximum(np.abs(mu_ref), 1.0)))


def cov_rel_err(c, c_ref):
    A, B = unpack(c), unpack(c_ref)
    num = np.sqrt(((A - B) ** 2).sum(axis=(-1, -2)))
    den = np.sqrt((B ** 2).sum(axis=(-1, -2)))
    return float(np.max(num / den))


def label_report(labels, ref_labels, ref_margin):
    labels = np.asarray(labels).ravel()
    ref = np.asarray(ref_labels).ravel()
    diff = labels != ref
    agree = 1.0 - diff.mean()
    worst = float(np.max(np.asarray(ref_margin).ravel()[diff])) if diff.any() else 0.0
    return agree, int(diff.sum()), worst
