"""Pins for the oracle's tensordot and trace (CPU only).

Each check fixes the oracle against something other than itself: values the
paper prints, hand-computed closed forms, brute force in plain Python on tiny
inputs, a library routine for the special case it covers, and identities of
the contraction (order independence, flatten-then-contract).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1905_01330_gb300 import synth
from conftest import read_golden


def brute_tensordot(A, legsA, B, legsB):
    """Pure-Python loops over every index of A and B (tiny inputs only)."""
    freeA = [p for p in range(A.ndim) if p not in legsA]
    freeB = [p for p in range(B.ndim) if p not in legsB]
    out = np.zeros([A.shape[p] for p in freeA] + [B.shape[p] for p in freeB])
    for ia in itertools.product(*[range(s) for s in A.shape]):
        for ib in itertools.product(*[range(s) for s in B.shape]):
            if all(ia[legsA[j]] == ib[legsB[j]] for j in range(len(legsA))):
                key = tuple(ia[p] for p in freeA) + tuple(ib[p] for p in freeB)
                out[key] += A[ia] * B[ib]
    return out


def test_ones_dot_is_two():
    g = read_golden("ones_dot.txt")
    a = np.ones(g["shape_a"])
    b = np.ones(g["shape_b"])
    c = oracle.tensordot(a, g["legs_a"], b, g["legs_b"])
    assert c.shape == ()
    assert float(c) == g["value"][0]


def test_elementary_contractions_closed_forms():
    # inner product sum_i A_i B_i
    assert float(oracle.tensordot([1.0, 2.0, 3.0], [0], [4.0, 5.0, 6.0], [0])) == 32.0
    # matrix-vector sum_j A_ij B_j
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    assert oracle.tensordot(A, [1], [5.0, 6.0], [0]).tolist() == [17.0, 39.0]
    # matrix-matrix sum_j A_ij B_jk
    B = np.array([[5.0, 6.0], [7.0, 8.0]])
    assert oracle.tensordot(A, [1], B, [0]).tolist() == [[19.0, 22.0], [43.0, 50.0]]
    # contracting the other legs gives A^T B and A B^T
    assert oracle.tensordot(A, [0], B, [0]).tolist() == [[26.0, 30.0], [38.0, 44.0]]
    assert oracle.tensordot(A, [1], B, [1]).tolist() == [[17.0, 23.0], [39.0, 53.0]]
    # trace sum_i A_ii
    assert float(oracle.trace(A, 0, 1)) == 5.0


def test_ncon_example_equals_matmul():
    g = read_golden("ncon_matmul.txt")
    a = synth.normal(11, 4).reshape(g["shape_a"])
    b = synth.normal(12, 4).reshape(g["shape_b"])
    c = oracle.tensordot(a, g["legs_a"], b, g["legs_b"])
    assert np.linalg.norm(c - a @ b) <= g["diff_norm"][0] + 1e-15


def test_hadamard_chain():
    g = read_golden("hadamard_chain.txt")
    H = np.array([[1.0, 1.0], [1.0, -1.0]]) / math.sqrt(2.0)
    q = np.array([1.0, 0.0])
    for _ in range(g["applications"][0]):
        q = oracle.tensordot(H, [1], q, [0])  # qubit edge into the gate's input leg
    np.testing.assert_allclose(q, g["out"], rtol=0, atol=1e-15)


def test_outer_product_shape_and_values():
    g = read_golden("outer_product_shape.txt")
    A = synth.normal(13, 6).reshape(g["shape_a"])
    B = synth.normal(14, 120).reshape(g["shape_b"])
    C = oracle.tensordot(A, [], B, [])
    assert list(C.shape) == g["shape_out"]
    for idx in [(0, 0, 0, 0, 0), (1, 2, 3, 4, 5), (1, 0, 2, 3, 1)]:
        assert C[idx] == A[idx[:2]] * B[idx[2:]]


@pytest.mark.parametrize("seed", range(6))
def test_random_small_against_brute_force(seed):
    st = synth.Stream(100 + seed)
    spec = synth.contraction_spec(st, dims=(2, 3, 4), cap=200)
    sha, la, shb, lb = spec
    A = synth.normal(200 + seed, int(np.prod(sha))).reshape(sha)
    B = synth.normal(300 + seed, int(np.prod(shb))).reshape(shb)
    C = oracle.tensordot(A, la, B, lb)
    np.testing.assert_allclose(C, brute_tensordot(A, list(la), B, list(lb)), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", range(8))
def test_random_specs_against_einsum(seed):
    # numpy einsum is the library routine for the general pairwise contraction
    st = synth.Stream(400 + seed)
    sha, la, shb, lb = synth.contraction_spec(st, dims=(2, 3, 5, 8), cap=4096)
    A = synth.normal(500 + seed, int(np.prod(sha))).reshape(sha)
    B = synth.normal(600 + seed, int(np.prod(shb))).reshape(shb)
    letters = "abcdefghijklmnop"
    ia = list(letters[:A.ndim])
    ib = list(letters[A.ndim:A.ndim + B.ndim])
    for j in range(len(la)):
        ib[lb[j]] = ia[la[j]]
    out = [ia[p] for p in range(A.ndim) if p not in la] + [ib[p] for p in range(B.ndim) if p not in lb]
    ref = np.einsum("".join(ia) + "," + "".join(ib) + "->" + "".join(out), A, B)
    np.testing.assert_allclose(oracle.tensordot(A, la, B, lb), ref, rtol=1e-12, atol=1e-12)


def test_shared_leg_order_does_not_matter():
    A = synth.normal(21, 3 * 4 * 5).reshape(3, 4, 5)
    B = synth.normal(22, 5 * 6 * 3).reshape(5, 6, 3)
    c1 = oracle.tensordot(A, [0, 2], B, [2, 0])
    c2 = oracle.tensordot(A, [2, 0], B, [0, 2])
    np.testing.assert_allclose(c1, c2, rtol=1e-13, atol=1e-13)


def test_flatten_then_contract_equals_contract_then_trace():
    # Two nodes joined by two edges (Sec. III.B.2): contracting one edge leaves
    # the other as a trace edge; flattening both first contracts them at once.
    A = synth.normal(31, 4 * 3 * 5).reshape(4, 3, 5)
    B = synth.normal(32, 3 * 5 * 6).reshape(3, 5, 6)
    flat = oracle.tensordot(A, [1, 2], B, [0, 1])          # (4, 6)
    one = oracle.tensordot(A, [1], B, [0])                  # (4, 5, 5, 6): a trace edge remains
    traced = oracle.trace(one, 1, 2)                        # (4, 6)
    np.testing.assert_allclose(flat, traced, rtol=1e-12, atol=1e-12)
    assert flat.size < one.size  # the flattened route never builds the larger node


def test_contraction_order_independence():
    # A triangle network A-B-C with one dangling leg per node.
    A = synth.normal(41, 3 * 4 * 5).reshape(3, 4, 5)  # legs (x, ab, ac)
    B = synth.normal(42, 4 * 6 * 7).reshape(4, 6, 7)  # legs (ab, y, bc)
    C = synth.normal(43, 5 * 7 * 2).reshape(5, 7, 2)  # legs (ac, bc, z)
    ab = oracle.tensordot(A, [1], B, [0])            # (x, ac, y, bc)
    r1 = oracle.tensordot(ab, [1, 3], C, [0, 1])     # (x, y, z)
    bc = oracle.tensordot(B, [2], C, [1])            # (ab, y, ac, z)
    r2 = oracle.tensordot(A, [1, 2], bc, [0, 2])     # (x, y, z)
    np.testing.assert_allclose(r1, r2, rtol=1e-12, atol=1e-12)


def test_rank_zero_and_scalar_cases():
    s = oracle.tensordot(np.array(3.0), [], np.array(4.0), [])
    assert s.shape == () and float(s) == 12.0
    v = oracle.tensordot(np.array(2.0), [], np.array([1.0, -1.0]), [])
    assert v.tolist() == [2.0, -2.0]


def test_invalid_contractions_rejected():
    with pytest.raises(ValueError):
        oracle.tensordot(np.ones((2, 3)), [1], np.ones((4, 2)), [0])  # dims differ
    with pytest.raises(ValueError):
        oracle.tensordot(np.ones((2, 2)), [0, 0], np.ones((2, 2)), [0, 1])  # duplicate leg
