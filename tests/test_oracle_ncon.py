"""Pins for the oracle's ncon (Appendix B; CPU only): the paper's check that
ncon([a, b], [(-1, 0), (0, -2)]) equals matmul(a, b); numpy einsum (the
library routine that evaluates a labelled network by its definition) on
random networks with traces, multi-edges and unconnected pieces; order
independence of the contraction sequence; the MPS norm network against the
oracle's transfer sweep; a trace and an outer product by hand."""
import numpy as np
import pytest

import oracle
from conftest import read_golden
from ncon_nets import einsum_spec, random_network
from paper_1905_01330_gb300 import synth


def test_paper_example_equals_matmul():
    g = read_golden("ncon_matmul.txt")
    a = synth.normal(11, 4).reshape(g["shape_a"])
    b = synth.normal(12, 4).reshape(g["shape_b"])
    c = oracle.ncon([a, b], [(-1, 0), (0, -2)])
    assert np.linalg.norm(c - a @ b) <= g["diff_norm"][0] + 1e-15


@pytest.mark.parametrize("seed", range(12))
def test_random_networks_against_einsum(seed):
    shapes, net = random_network(100 + seed)
    rng = np.random.default_rng(seed)
    ts = [rng.standard_normal(sh) for sh in shapes]
    got = oracle.ncon(ts, net)
    ref = np.einsum(einsum_spec(net), *ts)
    assert got.shape == ref.shape
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_contraction_order_does_not_change_the_result(seed):
    shapes, net = random_network(200 + seed, n_tensors=5, n_edges=6, n_open=2)
    rng = np.random.default_rng(seed)
    ts = [rng.standard_normal(sh) for sh in shapes]
    edges = sorted({x for labels in net for x in labels if x >= 0})
    ref = oracle.ncon(ts, net)
    for _ in range(3):
        order = list(rng.permutation(edges))
        assert np.allclose(oracle.ncon(ts, net, con_order=order), ref, rtol=1e-12, atol=1e-12)


def test_out_order_permutes_the_result():
    rng = np.random.default_rng(5)
    a, b = rng.standard_normal((2, 3, 4)), rng.standard_normal((4, 5))
    c = oracle.ncon([a, b], [(-1, -2, 0), (0, -3)])
    d = oracle.ncon([a, b], [(-1, -2, 0), (0, -3)], out_order=[-3, -1, -2])
    assert np.array_equal(d, np.transpose(c, (2, 0, 1)))


def test_mps_norm_network_matches_the_transfer_sweep():
    cores = synth.random_mps(6, 2, 4, seed=9)
    # bra cores labelled 10+i (bonds) and 100+i (physical), ket 20+i and the same physical
    net, ts = [], []
    n = len(cores)
    for i, c in enumerate(cores):
        left = (10 + i) if i > 0 else 0
        right = (10 + i + 1) if i < n - 1 else 1
        net.append((left, 100 + i, right))
        ts.append(c)
    for i, c in enumerate(cores):
        left = (20 + i) if i > 0 else 2
        right = (20 + i + 1) if i < n - 1 else 3
        net.append((left, 100 + i, right))
        ts.append(c)
    # the four unit-dimension boundary legs: edges 0-2 and 1-3
    net = [tuple({0: 0, 1: 1, 2: 0, 3: 1}.get(x, x) for x in labels) for labels in net]
    got = oracle.ncon(ts, net)
    v, lg = oracle.mps_inner(cores, cores)
    assert float(got) == pytest.approx(v * np.exp(lg), rel=1e-12)


def test_trace_and_outer_product_by_hand():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((3, 4, 3))
    tr = oracle.ncon([A], [(0, -1, 0)])
    assert np.allclose(tr, [sum(A[i, j, i] for i in range(3)) for j in range(4)], rtol=1e-14)
    g = read_golden("outer_product_shape.txt")
    a, b = rng.standard_normal(g["shape_a"]), rng.standard_normal(g["shape_b"])
    c = oracle.ncon([a, b], [(-1, -2), (-3, -4, -5)])
    assert list(c.shape) == g["shape_out"]
    assert c[1, 2, 3, 4, 5] == a[1, 2] * b[3, 4, 5]


@pytest.mark.parametrize("net", [[(0, -1), (0, 0)], [(0, -1), (1, -1)], [(0, -2), (0, -3)], [(-1, 0), (1,)]])
def test_invalid_networks(net):
    ts = [np.zeros((2,) * len(labels)) for labels in net]
    with pytest.raises(ValueError):
        oracle.ncon(ts, net)
