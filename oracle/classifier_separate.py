"""FP64 oracle of the classifier with one MPS per label (Sec. IV.A: the score
of label l is the overlap of the image's product state with MPS l) --
TEST INFRASTRUCTURE (tests, smoke and the bench's CPU leg only).

Each MPS's overlap is the oracle's float64 classifier sweep (oracle.c) run
with a single label, its middle core read as a (D, 2, 1, D') label core; the
L per-label (ftilde, log-scale) pairs are then brought to one log-scale per
sample, the largest: ftilde[b, l] = ftilde_l[b] exp(lam_l[b] - lam[b]).
The loss is the label-core classifier's: mean cross-entropy of softmax(z),
z = f / |f| per sample.
"""
from __future__ import annotations

import numpy as np


def classify_separate(mps_list, pixels):
    """(ftilde [B, L], log_scale [B]) with scores = ftilde * exp(log_scale[:, None])."""
    from . import classify
    fts, lams = [], []
    for cores in mps_list:
        c = [np.asarray(x, dtype=np.float64) for x in cores]
        m = len(c) // 2
        a, d, b = c[m].shape
        c[m] = c[m].reshape(a, d, 1, b)
        ft, lam = classify(c, m, pixels)
        fts.append(ft[:, 0])
        lams.append(lam)
    lam = np.max(np.stack(lams), axis=0)
    ft = np.stack([f * np.exp(l - lam) for f, l in zip(fts, lams)], axis=1)
    return ft, lam


def classify_separate_loss(mps_list, pixels, labels) -> float:
    ft, _ = classify_separate(mps_list, pixels)
    z = ft / np.linalg.norm(ft, axis=1, keepdims=True)
    zmax = z.max(axis=1, keepdims=True)
    logp = z - zmax - np.log(np.sum(np.exp(z - zmax), axis=1, keepdims=True))
    y = np.asarray(labels, dtype=np.int64)
    return float(-np.mean(logp[np.arange(len(y)), y]))
