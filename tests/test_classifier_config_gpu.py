"""Classifier parity at the workload's own sizes, on a deterministic subset.

The forward runs the whole workload on the GPU (784 sites, label core at site
392 with 10 labels, batch 4096, cores near identity with N(0, 1e-2) noise,
chi 32 / 64 / 128) and the FP64 oracle scores its first 256 samples; the
training-step gradient runs chi = 64 with checkpoints every 28 sites on the
first 256 samples of the batch (a gradient is a sum over the batch, so the
subset is its own batch on both sides).

Bounds, per sample (scores, log domain) or per core (gradients, normwise):
float32 1e-5 * sqrt(sites) (scores) and 1e-5 * sqrt(2 sites) (gradients);
split BF16x3 median <= 2 * 2^-16 * sqrt(sites), largest <= 40 * 2^-16 *
sqrt(sites), gradients <= 8 * 2^-16 * sqrt(2 sites); bf16 (one rounding of
each operand per step, 2^-9, times a conditioning of about 4, a random walk
over the sites) median <= 4 * 2^-9 * sqrt(sites).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1905_01330_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

B, N, LS, L = 4096, 784, 392, 10
SUB = 256
U16 = 2.0 ** -16


@pytest.fixture(scope="module")
def tn():
    from paper_1905_01330_gb300 import build, tn as tnmod
    build.build()
    tnmod.load()
    return tnmod


@pytest.fixture(scope="module")
def data():
    return synth.pixels(B, N, seed=3), synth.labels(B, L, seed=4)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def score_err(ft, lam, ft_ref, lam_ref):
    ft = ft.double().cpu().numpy()
    got = ft * np.exp(lam.cpu().numpy() - lam_ref)[:, None]
    return np.linalg.norm(got - ft_ref, axis=1) / np.linalg.norm(ft_ref, axis=1)


@pytest.mark.parametrize("chi", [32, 64, 128])
def test_forward_workload_first_samples(tn, data, chi):
    px_h, _ = data
    cores_h = synth.classifier_mps(N, chi, LS, L, seed=30 + chi, eps_std=0.1)
    ft_ref, lam_ref = oracle.classify(cores_h, LS, px_h[:SUB])
    cores = [dev(c) for c in cores_h]
    px = dev(px_h)
    ws = tn.classifier_workspace(cores, LS, L, B, 0)
    for prec in ("fp32", "bf16x3", "bf16"):
        ft, lam, _ = tn.mps_classify(cores, LS, px, prec=prec, ckpt_every=0, workspace=ws)
        assert tn.sync_status() == 0
        err = score_err(ft[:SUB], lam[:SUB], ft_ref, lam_ref)
        med, mx = float(np.median(err)), float(err.max())
        if prec == "fp32":
            assert mx <= 1e-5 * math.sqrt(N), (prec, med, mx)
        elif prec == "bf16x3":
            assert med <= 2 * U16 * math.sqrt(N), (prec, med, mx)
            assert mx <= 40 * U16 * math.sqrt(N), (prec, med, mx)
        else:
            assert med <= 4 * 2.0 ** -9 * math.sqrt(N), (prec, med, mx)


def test_training_gradient_workload_first_samples(tn, data):
    px_h, y_h = data
    chi, ck = 64, 28
    cores_h = synth.classifier_mps(N, chi, LS, L, seed=30 + chi, eps_std=0.1)
    _, g_ref = oracle.classify_grad(cores_h, LS, px_h[:SUB], y_h[:SUB])
    cores = [dev(c) for c in cores_h]
    px, y = dev(px_h[:SUB]), dev(y_h[:SUB])
    ws = tn.classifier_workspace(cores, LS, L, SUB, ck)
    for prec, bound in (("fp32", 1e-5 * math.sqrt(2 * N)), ("bf16x3", 8 * U16 * math.sqrt(2 * N))):
        ft, lam, _ = tn.mps_classify(cores, LS, px, prec=prec, ckpt_every=ck, workspace=ws)
        _, dft = tn.mps_classify_loss(ft, y)
        grads = tn.mps_classify_backward(cores, LS, px, dft, ws, prec=prec, ckpt_every=ck)
        assert tn.sync_status() == 0
        errs = [np.linalg.norm(g.double().cpu().numpy() - r) / np.linalg.norm(r) for g, r in zip(grads, g_ref)]
        assert max(errs) <= bound, (prec, float(np.median(errs)), max(errs))
