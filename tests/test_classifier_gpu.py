"""GPU parity of the MPS classifier: forward scores, loss head and the adjoint
backward against the FP64 oracle.

Scores are compared per sample as vectors over labels, on the true scale
f = ftilde * exp(log_scale): ||f - f*|| / ||f*||. Gradients per core:
||dW - dW*||_F / ||dW*||_F. float32 path tolerances: 1e-5 * sqrt(sites) for
scores (independent float32 roundings per site), 1e-4 for gradients (sums of
products over the batch on top of the sweep). Split BF16x3 path: a step's
products carry ~2^-16 relative error (the dropped lo*lo term and the rounding
of lo), independent per site, so a random walk: median score error
<= 2 * 2^-16 * sqrt(sites), largest <= 40 * 2^-16 * sqrt(sites) (the tail over
samples is heavier: products of random matrices), gradients <= 8 * 2^-16 *
sqrt(2 sites) per core (forward and adjoint walks).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1905_01330_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    from paper_1905_01330_gb300 import build, tn as tnmod
    build.build()
    tnmod.load()
    return tnmod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def score_err(ft, lam, ft_ref, lam_ref):
    """Per-sample normwise relative error of the scores, computed in the log domain."""
    ft = ft.double().cpu().numpy()
    lam = lam.cpu().numpy()
    shift = lam - lam_ref  # f = ft e^lam; f* = ft_ref e^lam_ref
    got = ft * np.exp(shift)[:, None]
    return np.linalg.norm(got - ft_ref, axis=1) / np.linalg.norm(ft_ref, axis=1)


@pytest.mark.parametrize("n,chi,ls,L,B", [(12, 8, 5, 3, 40), (50, 16, 25, 10, 70), (784, 32, 392, 10, 96),
                                          (40, 128, 20, 10, 70)])
def test_forward_fp32_parity(tn, n, chi, ls, L, B):
    cores = synth.classifier_mps(n, chi, ls, L, seed=31, eps_std=0.1)
    px = synth.pixels(B, n, seed=32)
    ft_ref, lam_ref = oracle.classify(cores, ls, px)
    ft, lam, _ = tn.mps_classify([dev(c) for c in cores], ls, dev(px), prec="fp32", ckpt_every=0)
    assert tn.sync_status() == 0
    err = score_err(ft, lam, ft_ref, lam_ref)
    assert err.max() <= 1e-5 * math.sqrt(n), err.max()


def test_identity_cores_closed_form(tn):
    n, chi, ls, L, B = 100, 16, 40, 4, 33
    cores = synth.classifier_mps(n, chi, ls, L, seed=1, eps_std=0.0)
    px = synth.pixels(B, n, seed=2)
    ft, lam, _ = tn.mps_classify([dev(c) for c in cores], ls, dev(px), prec="fp32", ckpt_every=0)
    ref = np.sum(np.log(np.cos(np.pi * px.astype(np.float64) / 2) + np.sin(np.pi * px.astype(np.float64) / 2)), axis=1)
    got = np.log(ft.double().cpu().numpy()) + lam.cpu().numpy()[:, None]
    assert np.max(np.abs(got - ref[:, None])) <= 1e-5 * math.sqrt(n)


def test_loss_head_matches_oracle(tn):
    n, chi, ls, L, B = 20, 8, 10, 10, 64
    cores = synth.classifier_mps(n, chi, ls, L, seed=41, eps_std=0.3)
    px = synth.pixels(B, n, seed=42)
    y = synth.labels(B, L, seed=43)
    ft, lam, _ = tn.mps_classify([dev(c) for c in cores], ls, dev(px), prec="fp32", ckpt_every=0)
    loss, dft = tn.mps_classify_loss(ft, torch.from_numpy(y).cuda())
    ref = oracle.classify_loss(cores, ls, px, y)
    assert abs(loss.item() - ref) <= 1e-5 * abs(ref)
    # dLoss/dftilde is orthogonal to ftilde (the loss is scale-invariant)
    dots = (dft.double() * ft.double()).sum(1).abs() / (dft.double().norm(dim=1) * ft.double().norm(dim=1))
    assert dots.max().item() < 1e-4


@pytest.mark.parametrize("ck", [1, 3, 5])
def test_backward_fp32_parity_tiny(tn, ck):
    n, chi, ls, L, B = 12, 8, 6, 3, 40
    cores = synth.classifier_mps(n, chi, ls, L, seed=51, eps_std=0.3)
    px = synth.pixels(B, n, seed=52)
    y = synth.labels(B, L, seed=53)
    loss_ref, g_ref = oracle.classify_grad(cores, ls, px, y)
    dc = [dev(c) for c in cores]
    ft, lam, ws = tn.mps_classify(dc, ls, dev(px), prec="fp32", ckpt_every=ck)
    loss, dft = tn.mps_classify_loss(ft, torch.from_numpy(y).cuda())
    grads = tn.mps_classify_backward(dc, ls, dev(px), dft, ws, prec="fp32", ckpt_every=ck)
    assert tn.sync_status() == 0
    assert abs(loss.item() - loss_ref) <= 1e-5 * abs(loss_ref)
    for i, (g, r) in enumerate(zip(grads, g_ref)):
        err = np.linalg.norm(g.double().cpu().numpy() - r) / np.linalg.norm(r)
        assert err <= 1e-4, (i, err)


def test_backward_fp32_parity_longer_chain(tn):
    n, chi, ls, L, B = 64, 32, 30, 10, 100
    cores = synth.classifier_mps(n, chi, ls, L, seed=61, eps_std=0.1)
    px = synth.pixels(B, n, seed=62)
    y = synth.labels(B, L, seed=63)
    _, g_ref = oracle.classify_grad(cores, ls, px, y)
    dc = [dev(c) for c in cores]
    ft, lam, ws = tn.mps_classify(dc, ls, dev(px), prec="fp32", ckpt_every=8)
    _, dft = tn.mps_classify_loss(ft, torch.from_numpy(y).cuda())
    grads = tn.mps_classify_backward(dc, ls, dev(px), dft, ws, prec="fp32", ckpt_every=8)
    for i, (g, r) in enumerate(zip(grads, g_ref)):
        err = np.linalg.norm(g.double().cpu().numpy() - r) / np.linalg.norm(r)
        assert err <= 1e-4, (i, err)


def test_autograd_function_matches_direct_backward(tn):
    n, chi, ls, L, B = 16, 8, 7, 4, 48
    cores = synth.classifier_mps(n, chi, ls, L, seed=71, eps_std=0.3)
    px = dev(synth.pixels(B, n, seed=72))
    y = synth.labels(B, L, seed=73)
    params = [dev(c).requires_grad_(True) for c in cores]
    ft, lam = tn.MPSClassifierFn.apply(px, ls, "fp32", 2, *params)
    z = ft / ft.norm(dim=1, keepdim=True)
    loss = torch.nn.functional.cross_entropy(z, torch.from_numpy(y).cuda())
    loss.backward()
    _, g_ref = oracle.classify_grad(cores, ls, px.cpu().numpy(), y)
    for i, (p, r) in enumerate(zip(params, g_ref)):
        err = np.linalg.norm(p.grad.double().cpu().numpy() - r) / np.linalg.norm(r)
        assert err <= 1e-4, (i, err)


# --------------------------------------------------------------- bf16 path
def bf16_tol(steps):
    """Per-sample relative score error of the bf16 sweep: two bf16 roundings
    per product (2^-8), independent per site, so a random walk over steps;
    factor 2 of margin."""
    return 2.0 * 2.0 ** -8 * math.sqrt(steps)


def round_bf16(a):
    """float32 -> nearest bfloat16 (ties to even), returned as float32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(np.shape(a))


@pytest.mark.parametrize("n,chi,ls,L,B", [(12, 8, 5, 3, 40), (60, 32, 30, 10, 200), (200, 64, 100, 10, 130),
                                          (64, 128, 33, 10, 129)])
def test_forward_bf16_parity(tn, n, chi, ls, L, B):
    cores = synth.classifier_mps(n, chi, ls, L, seed=81, eps_std=0.1)
    px = synth.pixels(B, n, seed=82)
    ft, lam, _ = tn.mps_classify([dev(c) for c in cores], ls, dev(px), prec="bf16", ckpt_every=0)
    assert tn.sync_status() == 0
    # 1) against the oracle on the same bf16-rounded cores (the label core
    #    stays float32 on both sides): what is left is the rounding of each
    #    step's vector to bf16, 2^-9 per element times the step's conditioning
    #    (about 4 for near-identity cores with 0.1 noise), a random walk over
    #    sites; the tail over samples is heavier (products of random matrices)
    rc = [c if i == ls else round_bf16(c) for i, c in enumerate(cores)]
    ft_r, lam_r = oracle.classify(rc, ls, px)
    err_r = score_err(ft, lam, ft_r, lam_r)
    walk = 4.0 * 2.0 ** -9 * math.sqrt(n)
    assert np.median(err_r) <= walk, (np.median(err_r), err_r.max())
    assert err_r.max() <= 4.0 * walk, (err_r.max(), np.median(err_r))
    # 2) against the exact oracle: the cores' own bf16 roundings (2^-8, shared
    #    by every sample) add a walk of the same kind
    ft_ref, lam_ref = oracle.classify(cores, ls, px)
    err = score_err(ft, lam, ft_ref, lam_ref)
    assert np.median(err) <= 2.0 * walk, (np.median(err), err.max())
    assert err.max() <= 8.0 * walk, (err.max(), np.median(err))


def test_forward_bf16_identity_cores(tn):
    # identity cores are exact in bf16; only the feature values round
    n, chi, ls, L, B = 784, 64, 392, 10, 128
    cores = synth.classifier_mps(n, chi, ls, L, seed=1, eps_std=0.0)
    px = synth.pixels(B, n, seed=2)
    ft, lam, _ = tn.mps_classify([dev(c) for c in cores], ls, dev(px), prec="bf16", ckpt_every=0)
    ref = np.sum(np.log(np.cos(np.pi * px.astype(np.float64) / 2) + np.sin(np.pi * px.astype(np.float64) / 2)), axis=1)
    got = np.log(ft.double().cpu().numpy()) + lam.cpu().numpy()[:, None]
    assert np.max(np.abs(got - ref[:, None])) <= bf16_tol(n)


@pytest.mark.parametrize("ck", [1, 4])
def test_backward_bf16_parity(tn, ck):
    n, chi, ls, L, B = 24, 32, 12, 10, 150
    cores = synth.classifier_mps(n, chi, ls, L, seed=91, eps_std=0.2)
    px = synth.pixels(B, n, seed=92)
    y = synth.labels(B, L, seed=93)
    _, g_ref = oracle.classify_grad(cores, ls, px, y)
    dc = [dev(c) for c in cores]
    ft, lam, ws = tn.mps_classify(dc, ls, dev(px), prec="bf16", ckpt_every=ck)
    _, dft = tn.mps_classify_loss(ft, torch.from_numpy(y).cuda())
    grads = tn.mps_classify_backward(dc, ls, dev(px), dft, ws, prec="bf16", ckpt_every=ck)
    assert tn.sync_status() == 0
    for i, (g, r) in enumerate(zip(grads, g_ref)):
        err = np.linalg.norm(g.double().cpu().numpy() - r) / np.linalg.norm(r)
        assert err <= bf16_tol(2 * n), (i, err)


# ------------------------------------------------------- split bf16x3 path
U16 = 2.0 ** -16


@pytest.mark.parametrize("n,chi,ls,L,B", [(12, 8, 5, 3, 40), (12, 8, 0, 3, 70), (12, 8, 11, 1, 70),
                                          (60, 32, 30, 10, 300), (200, 64, 100, 10, 130),
                                          (64, 128, 33, 10, 129)])
def test_forward_bf16x3_parity(tn, n, chi, ls, L, B):
    # ragged batches (not a multiple of the 128-sample tile), the label core
    # at either end of the chain (one half-chain without steps), one label
    cores = synth.classifier_mps(n, chi, ls, L, seed=81, eps_std=0.1)
    px = synth.pixels(B, n, seed=82)
    ft, lam, _ = tn.mps_classify([dev(c) for c in cores], ls, dev(px), prec="bf16x3", ckpt_every=0)
    assert tn.sync_status() == 0
    ft_ref, lam_ref = oracle.classify(cores, ls, px)
    err = score_err(ft, lam, ft_ref, lam_ref)
    assert np.median(err) <= 2 * U16 * math.sqrt(n), (np.median(err), err.max())
    assert err.max() <= 40 * U16 * math.sqrt(n), (err.max(), np.median(err))


@pytest.mark.parametrize("n,chi,ls,L,B,ck", [(12, 8, 5, 3, 40, 1), (12, 8, 0, 3, 70, 3), (40, 32, 20, 10, 300, 4),
                                             (40, 64, 17, 10, 200, 5), (30, 64, 29, 1, 150, 7)])
def test_backward_bf16x3_parity(tn, n, chi, ls, L, B, ck):
    cores = synth.classifier_mps(n, chi, ls, L, seed=91, eps_std=0.1)
    px = synth.pixels(B, n, seed=92)
    y = synth.labels(B, L, seed=93)
    _, g_ref = oracle.classify_grad(cores, ls, px, y)
    dc = [dev(c) for c in cores]
    ft, lam, ws = tn.mps_classify(dc, ls, dev(px), prec="bf16x3", ckpt_every=ck)
    _, dft = tn.mps_classify_loss(ft, torch.from_numpy(y).cuda())
    grads = tn.mps_classify_backward(dc, ls, dev(px), dft, ws, prec="bf16x3", ckpt_every=ck)
    assert tn.sync_status() == 0
    for i, (g, r) in enumerate(zip(grads, g_ref)):
        nr = np.linalg.norm(r)
        if nr == 0.0:
            assert not g.any().item(), i
            continue
        err = np.linalg.norm(g.double().cpu().numpy() - r) / nr
        assert err <= 8 * U16 * math.sqrt(2 * n), (i, err)


def test_backward_bf16x3_chi128_is_unsupported(tn):
    # the split adjoint's staging at chi = 128 does not fit in shared memory
    n, chi, ls, L, B = 10, 128, 5, 2, 16
    cores = synth.classifier_mps(n, chi, ls, L, seed=3, eps_std=0.1)
    px = synth.pixels(B, n, seed=4)
    dc = [dev(c) for c in cores]
    ft, lam, ws = tn.mps_classify(dc, ls, dev(px), prec="bf16x3", ckpt_every=2)
    with pytest.raises(tn.TnError) as e:
        tn.mps_classify_backward(dc, ls, dev(px), torch.ones_like(ft), ws, prec="bf16x3", ckpt_every=2)
    assert e.value.code == 3


def test_backward_fp32_chi128(tn):
    n, chi, ls, L, B = 16, 128, 8, 4, 40
    cores = synth.classifier_mps(n, chi, ls, L, seed=95, eps_std=0.1)
    px = synth.pixels(B, n, seed=96)
    y = synth.labels(B, L, seed=97)
    _, g_ref = oracle.classify_grad(cores, ls, px, y)
    dc = [dev(c) for c in cores]
    ft, lam, ws = tn.mps_classify(dc, ls, dev(px), prec="fp32", ckpt_every=3)
    _, dft = tn.mps_classify_loss(ft, torch.from_numpy(y).cuda())
    grads = tn.mps_classify_backward(dc, ls, dev(px), dft, ws, prec="fp32", ckpt_every=3)
    for i, (g, r) in enumerate(zip(grads, g_ref)):
        err = np.linalg.norm(g.double().cpu().numpy() - r) / np.linalg.norm(r)
        assert err <= 1e-4, (i, err)


def test_backward_under_graph_capture(tn):
    # BF16 / BF16X3 only launch: the training step replays from a CUDA graph
    # with the eager gradients. The FP32 backward builds and uploads its
    # grouped plans in the call, from host lists a captured copy could not
    # replay, so it refuses a capturing stream (TN_ERR_UNSUPPORTED) with
    # nothing enqueued.
    n, chi, ls, L, B = 16, 8, 7, 4, 48
    cores = synth.classifier_mps(n, chi, ls, L, seed=71, eps_std=0.2)
    px, y = dev(synth.pixels(B, n, seed=72)), torch.from_numpy(synth.labels(B, L, seed=73)).cuda()
    dc = [dev(c) for c in cores]
    for prec in ("bf16", "bf16x3"):
        ws = tn.classifier_workspace(dc, ls, L, B, 4)

        def step():
            ft, lam, _ = tn.mps_classify(dc, ls, px, prec=prec, ckpt_every=4, workspace=ws)
            _, dft = tn.mps_classify_loss(ft, y)
            return tn.mps_classify_backward(dc, ls, px, dft, ws, prec=prec, ckpt_every=4)
        eager = [g.clone() for g in step()]
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            step()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            out = step()
        graph.replay()
        torch.cuda.synchronize()
        assert tn.sync_status() == 0
        for a, b in zip(eager, out):
            # float32 atomics in the gradient reductions: equal to rounding
            assert torch.allclose(a, b, rtol=1e-5, atol=1e-6 * float(a.abs().max()))
    ws = tn.classifier_workspace(dc, ls, L, B, 4)
    ft, lam, _ = tn.mps_classify(dc, ls, px, prec="fp32", ckpt_every=4, workspace=ws)
    _, dft = tn.mps_classify_loss(ft, y)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with pytest.raises(tn.TnError) as err:
        with torch.cuda.graph(graph):
            tn.mps_classify_backward(dc, ls, px, dft, ws, prec="fp32", ckpt_every=4)
    assert err.value.code == 3
    torch.cuda.synchronize()
    assert tn.sync_status() == 0
    grads = tn.mps_classify_backward(dc, ls, px, dft, ws, prec="fp32", ckpt_every=4)
    torch.cuda.synchronize()
    assert tn.sync_status() == 0 and all(bool(torch.isfinite(g).all()) for g in grads)
