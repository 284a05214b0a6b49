"""GPU parity of ncon (Appendix B): the network evaluated by tn_ncon_plan's
steps, each a tn_contract call on the GPU (a trace as a contraction with the
identity), against the FP64 oracle's ncon on the same inputs. float32
results within 1e-5 of the oracle's norm (a few contractions in sequence);
bf16 within 2e-2 (each step rounds its operands to bf16)."""
import numpy as np
import pytest

import oracle
from ncon_nets import random_network
from paper_1905_01330_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    from paper_1905_01330_gb300 import build, tn as tnmod
    build.build()
    tnmod.load()
    return tnmod


def run(tn, ts_h, net, prec="fp32", tol=1e-5, **kw):
    ts = [torch.from_numpy(np.ascontiguousarray(t, dtype=np.float32)).cuda() for t in ts_h]
    got = tn.ncon(ts, net, prec=prec, **kw)
    torch.cuda.synchronize()
    assert tn.sync_status() == 0
    ref = oracle.ncon([t.astype(np.float32).astype(np.float64) for t in ts_h], net, **kw)
    g = got.double().cpu().numpy()
    assert g.shape == np.shape(ref)
    assert np.linalg.norm(g - ref) <= tol * max(np.linalg.norm(ref), 1e-30)
    return got


def test_paper_example(tn):
    a = synth.normal(11, 4).reshape(2, 2)
    b = synth.normal(12, 4).reshape(2, 2)
    c = run(tn, [a, b], [(-1, 0), (0, -2)])
    assert np.linalg.norm(c.cpu().numpy() - (a.astype(np.float32) @ b.astype(np.float32))) < 1e-5


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16", 2e-2)])
@pytest.mark.parametrize("seed", range(8))
def test_random_networks(tn, seed, prec, tol):
    shapes, net = random_network(300 + seed, max_dim=7)
    rng = np.random.default_rng(seed)
    run(tn, [rng.standard_normal(sh) for sh in shapes], net, prec=prec, tol=tol)


def test_orders(tn):
    shapes, net = random_network(400, n_tensors=5, n_edges=6, n_open=3, max_dim=6)
    rng = np.random.default_rng(1)
    ts = [rng.standard_normal(sh) for sh in shapes]
    edges = sorted({x for labels in net for x in labels if x >= 0})
    run(tn, ts, net, con_order=list(reversed(edges)), out_order=[-3, -1, -2])


def test_mps_norm_network(tn):
    cores = synth.random_mps(8, 2, 16, seed=9)
    n = len(cores)
    net, ts = [], []
    for side, base in ((0, 10), (1, 30)):
        for i, c in enumerate(cores):
            left = (base + i) if i > 0 else 0
            right = (base + i + 1) if i < n - 1 else 1
            net.append((left, 100 + i, right))
            ts.append(c)
    # boundary legs (dimension 1) of bra and ket joined: labels 0 and 1 twice
    got = run(tn, ts, net)
    v, lg = oracle.mps_inner(cores, cores)
    assert float(got) == pytest.approx(v * np.exp(lg), rel=1e-5)


def test_larger_contraction_chain(tn):
    rng = np.random.default_rng(3)
    A, B, C = rng.standard_normal((64, 48, 32)), rng.standard_normal((32, 48, 80)), rng.standard_normal((80, 64))
    run(tn, [A, B, C], [(-1, 1, 2), (2, 1, 3), (3, -2)])
    run(tn, [A, B, C], [(-1, 1, 2), (2, 1, 3), (3, -2)], prec="bf16", tol=2e-2)


def test_invalid_network(tn):
    with pytest.raises(tn.TnError):
        tn.ncon([torch.zeros(2, 2, device="cuda"), torch.zeros(3, 2, device="cuda")], [(0, -1), (0, -2)])


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16", 2e-2)])
def test_plan_eager_and_graph(tn, prec, tol):
    """NconPlan: planned once, run eagerly and replayed from a CUDA graph,
    after the inputs' values change in place."""
    shapes, net = random_network(500, n_tensors=5, n_edges=6, n_open=3, max_dim=6)
    rng = np.random.default_rng(2)
    hs = [rng.standard_normal(sh).astype(np.float32) for sh in shapes]
    ts = [torch.from_numpy(h).cuda() for h in hs]
    plan = tn.NconPlan(ts, net, prec=prec)
    ref = oracle.ncon([h.astype(np.float64) for h in hs], net)
    got = plan.run().double().cpu().numpy()
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    plan.capture()
    hs2 = [rng.standard_normal(sh).astype(np.float32) for sh in shapes]
    for t, h in zip(ts, hs2):
        t.copy_(torch.from_numpy(h))
    got2 = plan.replay().double().cpu().numpy()
    torch.cuda.synchronize()
    ref2 = oracle.ncon([h.astype(np.float64) for h in hs2], net)
    assert np.linalg.norm(got2 - ref2) <= tol * np.linalg.norm(ref2)
    assert tn.sync_status() == 0
