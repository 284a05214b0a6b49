"""GPU parity of the classifier with one MPS per label (Sec. IV.A) against
the FP64 oracle: scores per sample on the true scale (log domain, as in
test_classifier_gpu), gradients per core (normwise) against the label-core
oracle's gradient when the MPS share their other cores, and directional
derivatives against central differences of the oracle's float64 loss.
Tolerances as for the label-core classifier: float32 scores 1e-5 sqrt(sites),
gradients 1e-4; bf16 scores within the rounding walk 4 2^-9 sqrt(sites)."""
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
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def score_err(ft, lam, ft_ref, lam_ref):
    ft = ft.double().cpu().numpy()
    got = ft * np.exp(lam.cpu().numpy() - lam_ref)[:, None]
    return np.linalg.norm(got - ft_ref, axis=1) / np.linalg.norm(ft_ref, axis=1)


def round_bf16(a):
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(np.shape(a))


@pytest.mark.parametrize("n,chi,L,B", [(16, 8, 10, 40), (101, 32, 10, 64), (60, 64, 3, 130)])
def test_forward_fp32_parity(tn, n, chi, L, B):
    mps = synth.classifier_separate_mps(n, chi, L, seed=41, eps_std=0.1)
    px = synth.pixels(B, n, seed=42)
    ft_ref, lam_ref = oracle.classify_separate(mps, px)
    ft, lam, _ = tn.mps_classify_separate([[dev(c) for c in cores] for cores in mps], dev(px), prec="fp32",
                                          ckpt_every=0)
    assert tn.sync_status() == 0
    assert tuple(ft.shape) == (B, L)
    err = score_err(ft, lam, ft_ref, lam_ref)
    assert err.max() <= 1e-5 * math.sqrt(n), err.max()


@pytest.mark.parametrize("n,chi,L,B", [(40, 32, 10, 70), (80, 64, 4, 129)])
def test_forward_bf16_parity(tn, n, chi, L, B):
    mps = synth.classifier_separate_mps(n, chi, L, seed=51, eps_std=0.1)
    px = synth.pixels(B, n, seed=52)
    ft, lam, _ = tn.mps_classify_separate([[dev(c) for c in cores] for cores in mps], dev(px), prec="bf16",
                                          ckpt_every=0)
    assert tn.sync_status() == 0
    # the oracle on the same bf16-rounded cores; each MPS's middle core is its
    # one-label label core and stays float32, as in the label-core classifier
    rounded = [[c if i == n // 2 else round_bf16(c) for i, c in enumerate(cores)] for cores in mps]
    ft_r, lam_r = oracle.classify_separate(rounded, px)
    err = score_err(ft, lam, ft_r, lam_r)
    walk = 4.0 * 2.0 ** -9 * math.sqrt(n)
    assert np.median(err) <= walk, (np.median(err), err.max())
    assert err.max() <= 4.0 * walk, (err.max(), np.median(err))


@pytest.mark.parametrize("ck", [1, 3])
def test_backward_matches_label_core_gradient_with_shared_cores(tn, ck):
    n, chi, ls, L, B = 12, 6, 5, 4, 24
    cores = synth.classifier_mps(n, chi, ls, L, seed=61, eps_std=0.2)
    px = synth.pixels(B, n, seed=62)
    y = synth.labels(B, L, seed=63)
    mps = [[c if i != ls else np.ascontiguousarray(cores[ls][:, :, l, :]) for i, c in enumerate(cores)]
           for l in range(L)]
    mps_d = [[dev(c) for c in m] for m in mps]
    ft, lam, ws = tn.mps_classify_separate(mps_d, dev(px), prec="fp32", ckpt_every=ck)
    loss, dft = tn.mps_classify_loss(ft, torch.from_numpy(y).cuda())
    grads = tn.mps_classify_separate_backward(mps_d, dev(px), dft, ws, prec="fp32", ckpt_every=ck)
    assert tn.sync_status() == 0
    assert float(loss) == pytest.approx(oracle.classify_loss(cores, ls, px, y), rel=1e-5)
    _, g_ref = oracle.classify_grad(cores, ls, px, y)
    for i in range(n):
        if i == ls:
            got = np.stack([grads[l][i].double().cpu().numpy() for l in range(L)], axis=2)
        else:
            got = sum(grads[l][i].double().cpu().numpy() for l in range(L))
        ref = g_ref[i]
        assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref), (i, np.linalg.norm(got - ref) / np.linalg.norm(ref))


def test_backward_directional_derivatives(tn):
    """Distinct MPS: the gradient along random directions against central
    differences of the oracle's float64 loss (h = 1e-5)."""
    n, chi, L, B = 9, 4, 3, 16
    mps = synth.classifier_separate_mps(n, chi, L, seed=71, eps_std=0.3)
    px = synth.pixels(B, n, seed=72)
    y = synth.labels(B, L, seed=73)
    mps_d = [[dev(c) for c in m] for m in mps]
    ft, lam, ws = tn.mps_classify_separate(mps_d, dev(px), prec="fp32", ckpt_every=2)
    _, dft = tn.mps_classify_loss(ft, torch.from_numpy(y).cuda())
    grads = tn.mps_classify_separate_backward(mps_d, dev(px), dft, ws, prec="fp32", ckpt_every=2)
    rng = np.random.default_rng(74)
    h = 1e-5
    for _ in range(4):
        V = [[rng.standard_normal(c.shape) for c in m] for m in mps]
        plus = [[c.astype(np.float64) + h * v for c, v in zip(m, vm)] for m, vm in zip(mps, V)]
        minus = [[c.astype(np.float64) - h * v for c, v in zip(m, vm)] for m, vm in zip(mps, V)]
        fd = (oracle.classify_separate_loss(plus, px, y) - oracle.classify_separate_loss(minus, px, y)) / (2 * h)
        an = sum(float(np.sum(g.double().cpu().numpy() * v)) for gl, vl in zip(grads, V) for g, v in zip(gl, vl))
        assert an == pytest.approx(fd, rel=1e-4, abs=1e-7)


def test_empty_batch_and_errors(tn):
    mps = synth.classifier_separate_mps(6, 4, 2, seed=81)
    mps_d = [[dev(c) for c in m] for m in mps]
    px = torch.empty((0, 6), device="cuda")
    ft, lam, ws = tn.mps_classify_separate(mps_d, px, prec="fp32", ckpt_every=1)
    assert tuple(ft.shape) == (0, 2)
    grads = tn.mps_classify_separate_backward(mps_d, px, torch.empty((0, 2), device="cuda"), ws, ckpt_every=1)
    assert all(float(g.abs().max()) == 0.0 for gl in grads for g in gl)
    short = [mps_d[0], mps_d[1][:5]]
    with pytest.raises(tn.TnError):
        tn.mps_classify_separate(short, torch.rand((3, 6), device="cuda"), ckpt_every=0)


def test_under_graph_capture(tn):
    # the L sweeps run on library streams forked from and joined into the
    # caller's stream, so forward (every precision) and the BF16 / BF16X3
    # training step replay from a CUDA graph with the eager results
    n, chi, L, B = 24, 16, 4, 64
    mps = [[dev(c) for c in cores] for cores in synth.classifier_separate_mps(n, chi, L, seed=81, eps_std=0.1)]
    px = dev(synth.pixels(B, n, seed=82))
    y = torch.from_numpy(synth.labels(B, L, seed=83)).cuda()

    def capture(fn):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            fn()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            out = fn()
        graph.replay()
        torch.cuda.synchronize()
        return out
    for prec in ("fp32", "bf16", "bf16x3"):
        ws = tn.classifier_separate_workspace(mps, B, 0)
        fwd = lambda: tn.mps_classify_separate(mps, px, prec=prec, ckpt_every=0, workspace=ws)[:2]
        eager = [t.clone() for t in fwd()]
        got = capture(fwd)
        assert tn.sync_status() == 0
        for a, b in zip(eager, got):
            assert torch.allclose(a, b, rtol=1e-6, atol=0.0), prec
    for prec in ("bf16", "bf16x3"):
        ws = tn.classifier_separate_workspace(mps, B, 3)

        def step():
            ft, lam, _ = tn.mps_classify_separate(mps, px, prec=prec, ckpt_every=3, workspace=ws)
            _, dft = tn.mps_classify_loss(ft, y)
            return tn.mps_classify_separate_backward(mps, px, dft, ws, prec=prec, ckpt_every=3)
        eager = [[g.clone() for g in m] for m in step()]
        got = capture(step)
        assert tn.sync_status() == 0
        for em, gm in zip(eager, got):
            for a, b in zip(em, gm):
                assert torch.allclose(a, b, rtol=1e-5, atol=1e-6 * float(a.abs().max())), prec
