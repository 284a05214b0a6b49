"""Pins for the oracle's MPS classifier forward pass, loss and gradient (CPU)."""
import math

import numpy as np
import pytest

import oracle
from paper_1905_01330_gb300 import synth


def label_slices(cores, ls):
    """The classifier as L ordinary MPS: slice the label leg of the label core."""
    L = cores[ls].shape[2]
    return [[c if i != ls else c[:, :, l, :] for i, c in enumerate(cores)] for l in range(L)]


def feature_product_state(x):
    """Dense tensor product of the local feature vectors (cos pi x/2, sin pi x/2)."""
    out = np.array([1.0])
    for p in x:
        out = np.kron(out, np.array([math.cos(math.pi * p / 2), math.sin(math.pi * p / 2)]))
    return out


def test_identity_cores_closed_form():
    n, chi, ls, L = 12, 4, 6, 3
    cores = synth.classifier_mps(n, chi, ls, L, seed=1, eps_std=0.0)
    x = synth.pixels(5, n, seed=2)
    ft, lam = oracle.classify(cores, ls, x)
    for b in range(5):
        ref = sum(math.log(math.cos(math.pi * p / 2) + math.sin(math.pi * p / 2)) for p in x[b].astype(np.float64))
        for l in range(L):
            assert ft[b, l] > 0
            assert abs(math.log(ft[b, l]) + lam[b] - ref) < 1e-12


@pytest.mark.parametrize("seed", [3, 4])
def test_scores_equal_inner_product_with_feature_state(seed):
    n, chi, ls, L = 8, 4, 3, 4
    cores = synth.classifier_mps(n, chi, ls, L, seed=seed, eps_std=0.3)
    x = synth.pixels(3, n, seed=seed + 10)
    ft, lam = oracle.classify(cores, ls, x)
    for l, mps in enumerate(label_slices(cores, ls)):
        psi = oracle.mps_state(mps)
        for b in range(3):
            ref = float(feature_product_state(x[b].astype(np.float64)) @ psi)
            assert abs(ft[b, l] * math.exp(lam[b]) - ref) <= 1e-12 * max(1.0, abs(ref))


def test_binary_pixels_select_one_component():
    # p in {0, 1} maps to one-hot (1,0) / (0,1): the score is psi_l(s) with s = p
    n, chi, ls, L = 6, 3, 2, 2
    cores = synth.classifier_mps(n, chi, ls, L, seed=5, eps_std=0.5)
    bits = np.array([[1, 0, 1, 1, 0, 0], [0, 0, 0, 0, 0, 1]], dtype=np.float64)
    ft, lam = oracle.classify(cores, ls, bits)
    for l, mps in enumerate(label_slices(cores, ls)):
        psi = oracle.mps_state(mps)
        for b in range(2):
            idx = int("".join(str(int(v)) for v in bits[b]), 2)
            assert abs(ft[b, l] * math.exp(lam[b]) - psi[idx]) <= 1e-12 * max(1.0, abs(psi[idx]))


def test_equal_scores_give_log_L_loss():
    # identity cores give the same score for every label: z = 1/sqrt(L), softmax uniform
    n, chi, ls, L = 10, 3, 5, 10
    cores = synth.classifier_mps(n, chi, ls, L, seed=6, eps_std=0.0)
    x = synth.pixels(4, n, seed=7)
    y = synth.labels(4, L, seed=8)
    assert abs(oracle.classify_loss(cores, ls, x, y) - math.log(L)) < 1e-12


def test_long_chain_does_not_overflow():
    n, chi, ls, L = 784, 8, 392, 10
    cores = synth.classifier_mps(n, chi, ls, L, seed=9, eps_std=0.1)
    x = synth.pixels(2, n, seed=10)
    ft, lam = oracle.classify(cores, ls, x)
    assert np.all(np.isfinite(ft)) and np.all(np.isfinite(lam))
    assert np.max(np.abs(ft)) > 1e-6 and lam.min() > 50.0  # raw scores far beyond float32 range


@pytest.mark.parametrize("seed", [11, 12])
def test_gradient_against_central_differences(seed):
    n, chi, ls, L, B = 8, 4, 4, 3, 8
    cores = [c.astype(np.float64) for c in synth.classifier_mps(n, chi, ls, L, seed=seed, eps_std=0.4)]
    x = synth.pixels(B, n, seed=seed + 1)
    y = synth.labels(B, L, seed=seed + 2)
    loss, grads = oracle.classify_grad(cores, ls, x, y)
    assert abs(loss - oracle.classify_loss(cores, ls, x, y)) < 1e-14
    h = 1e-6
    for i in range(n):
        fd = np.zeros_like(cores[i])
        flat = cores[i].reshape(-1)
        for e in range(flat.size):
            keep = flat[e]
            flat[e] = keep + h
            lp = oracle.classify_loss(cores, ls, x, y)
            flat[e] = keep - h
            lm = oracle.classify_loss(cores, ls, x, y)
            flat[e] = keep
            fd.reshape(-1)[e] = (lp - lm) / (2 * h)
        err = np.linalg.norm(grads[i] - fd) / max(np.linalg.norm(fd), 1e-30)
        assert err <= 1e-6, (i, err)


def test_gradient_directional_derivative_longer_chain():
    n, chi, ls, L, B = 32, 8, 16, 10, 6
    cores = [c.astype(np.float64) for c in synth.classifier_mps(n, chi, ls, L, seed=21, eps_std=0.2)]
    x = synth.pixels(B, n, seed=22)
    y = synth.labels(B, L, seed=23)
    _, grads = oracle.classify_grad(cores, ls, x, y)
    for trial in range(3):
        dirs = [synth.normal(synth.substream(30 + trial, i), c.size).reshape(c.shape) for i, c in enumerate(cores)]
        h = 1e-5
        plus = [c + h * d for c, d in zip(cores, dirs)]
        minus = [c - h * d for c, d in zip(cores, dirs)]
        fd = (oracle.classify_loss(plus, ls, x, y) - oracle.classify_loss(minus, ls, x, y)) / (2 * h)
        an = sum(float(np.sum(g * d)) for g, d in zip(grads, dirs))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


# ------------------------------------------- one MPS per label (Sec. IV.A)
def test_separate_identity_cores_closed_form():
    n, chi, L, B = 40, 6, 4, 9
    mps = synth.classifier_separate_mps(n, chi, L, seed=3, eps_std=0.0)
    px = synth.pixels(B, n, seed=4).astype(np.float64)
    ft, lam = oracle.classify_separate(mps, px)
    ref = np.sum(np.log(np.cos(np.pi * px / 2) + np.sin(np.pi * px / 2)), axis=1)
    assert np.allclose(np.log(ft) + lam[:, None], ref[:, None], rtol=0, atol=1e-10)


def test_separate_equals_label_core_model_with_shared_cores():
    """L MPS that share every core but the label site's, whose core is slice l
    of a label core, score exactly as the one-MPS label-core classifier."""
    n, chi, ls, L, B = 14, 5, 6, 4, 11
    cores = synth.classifier_mps(n, chi, ls, L, seed=7, eps_std=0.2)
    px = synth.pixels(B, n, seed=8)
    mps = [[c if i != ls else np.ascontiguousarray(cores[ls][:, :, l, :]) for i, c in enumerate(cores)]
           for l in range(L)]
    ft, lam = oracle.classify_separate(mps, px)
    ft_ref, lam_ref = oracle.classify(cores, ls, px)
    assert np.allclose(ft * np.exp(lam - lam_ref)[:, None], ft_ref, rtol=1e-12, atol=1e-14)


def test_separate_brute_force_tiny():
    """2^n state vector of each MPS against the product state of the pixels."""
    n, chi, L, B = 7, 3, 3, 5
    mps = synth.classifier_separate_mps(n, chi, L, seed=9, eps_std=0.5)
    px = synth.pixels(B, n, seed=10).astype(np.float64)
    ft, lam = oracle.classify_separate(mps, px)
    for l, cores in enumerate(mps):
        psi = oracle.mps_state([c.astype(np.float64) for c in cores]).reshape([2] * n)
        for b in range(B):
            phi = [np.array([np.cos(np.pi * x / 2), np.sin(np.pi * x / 2)]) for x in px[b]]
            f = psi
            for v in phi:
                f = np.tensordot(f, v, axes=([0], [0]))
            assert ft[b, l] * np.exp(lam[b]) == pytest.approx(float(f), rel=1e-11)


def test_separate_loss_equal_scores_is_log_L():
    n, chi, L, B = 10, 4, 5, 6
    one = synth.classifier_separate_mps(n, chi, 1, seed=11, eps_std=0.3)[0]
    mps = [one] * L
    px = synth.pixels(B, n, seed=12)
    assert oracle.classify_separate_loss(mps, px, np.arange(B) % L) == pytest.approx(np.log(L), rel=1e-12)
