"""Pins for the oracle's node splitting (CPU only).

The checks fix the oracle against the paper's printed shapes and counts (Sec.
III.B "Node Splitting", Appendix A), against inputs whose decomposition is
known by construction (a spectrum planted between two orthogonal factors, a
rank-1 outer product, a diagonal matrix), and against identities every SVD
split satisfies (reconstruction, orthonormal factors, sqrt(S) on both sides,
the Eckart-Young error of the truncated product), so that a dropped factor, a
transposed view, a wrong leg order or a wrong truncation rule fails one of them.
"""
import numpy as np
import pytest

import oracle
from conftest import read_golden


def planted(m, n, s, seed):
    """Q1 diag(s) Q2^T with Q1, Q2 orthonormal (QR of Gaussian matrices): its
    singular values are s by construction."""
    rng = np.random.default_rng(seed)
    r = len(s)
    q1, _ = np.linalg.qr(rng.standard_normal((m, r)))
    q2, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return (q1 * np.asarray(s)[None, :]) @ q2.T


def test_paper_split_shapes():
    g = read_golden("split_node_shapes.txt")
    A = np.random.default_rng(0).standard_normal(g["shape"])
    us, svh, dropped = oracle.split_node(A, g["left"], g["right"])
    assert list(us.shape) == g["shape_left"]
    assert list(svh.shape) == g["shape_right"]
    assert dropped.shape == (0,)
    u, s, vh, _ = oracle.split_node(A, g["left"], g["right"], full_svd=True)
    assert list(u.shape) == g["shape_left"] and s.shape == (24,) and list(vh.shape) == g["shape_right"]


def test_paper_truncation_counts():
    g = read_golden("split_node_truncation.txt")
    m, n = g["shape"]
    # spectrum 1, 0.99, ... : 1000 distinct values, a long tail below 0.1 in sum
    s = 0.99 ** np.arange(min(m, n))
    A = planted(m, n, s, 1)
    us, svh, dropped = oracle.split_node(A, [0], [1], max_singular_values=g["max_singular_values"][0])
    assert list(us.shape) == g["shape_u"] and list(svh.shape) == g["shape_vh"]
    assert dropped.shape == (g["dropped"][0],)
    err = g["max_truncation_err"][0]
    _, _, dropped = oracle.split_node(A, [0], [1], max_truncation_err=err)
    assert dropped.sum() <= err
    # maximal: the smallest kept value would push the dropped sum past the limit
    kept = s[: len(s) - len(dropped)]
    assert dropped.sum() + kept[-1] > err


def test_planted_spectrum_is_recovered():
    s = np.array([7.0, 3.0, 2.5, 1.0, 0.25, 1e-3])
    A = planted(40, 25, s, 2)
    _, S, _, _, _ = oracle.svd(A, [0], [1])
    assert np.allclose(S[:6], s, rtol=1e-12, atol=1e-13)
    assert np.all(np.abs(S[6:]) < 1e-12)


def test_rank_one_outer_product():
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal(12), rng.standard_normal(20)
    A = np.multiply.outer(x, y).reshape(3, 4, 20)
    _, S, _, _, _ = oracle.svd(A, [0, 1], [2])
    assert S[0] == pytest.approx(np.linalg.norm(x) * np.linalg.norm(y), rel=1e-13)
    assert np.all(S[1:] < 1e-12 * S[0])


def test_diagonal_matrix_sorted_absolute_values():
    d = np.array([0.5, -4.0, 2.0, 0.0, 3.0])
    _, S, _, _, _ = oracle.svd(np.diag(d), [0], [1])
    assert np.allclose(S, [4.0, 3.0, 2.0, 0.5, 0.0], atol=1e-15)


@pytest.mark.parametrize("shape,left,right", [((6, 5, 4), [0, 1], [2]), ((6, 5, 4), [2, 0], [1]),
                                              ((3, 4, 5, 2), [3, 1], [0, 2]), ((7, 30), [1], [0])])
def test_reconstruction_and_orthonormal_factors(shape, left, right):
    rng = np.random.default_rng(4)
    A = rng.standard_normal(shape)
    mat = np.transpose(A, list(left) + list(right)).reshape(int(np.prod([shape[p] for p in left])), -1)
    us, svh, dropped = oracle.split_node(A, left, right)
    k = us.shape[-1]
    assert k == min(mat.shape) and dropped.size == 0
    assert list(us.shape) == [shape[p] for p in left] + [k]
    assert list(svh.shape) == [k] + [shape[p] for p in right]
    rec = us.reshape(-1, k) @ svh.reshape(k, -1)
    assert np.abs(rec - mat).max() < 1e-12 * np.abs(mat).max()
    u, s, vh, _ = oracle.split_node(A, left, right, full_svd=True)
    U, V = u.reshape(-1, k), vh.reshape(k, -1)
    assert np.abs(U.T @ U - np.eye(k)).max() < 1e-12
    assert np.abs(V @ V.T - np.eye(k)).max() < 1e-12
    assert np.all(np.diff(s) <= 0) and np.all(s >= 0)
    # sqrt(S) on both sides: column j of U sqrt(S) and row j of sqrt(S) V^T
    # both have norm sqrt(s_j)
    assert np.allclose(np.linalg.norm(us.reshape(-1, k), axis=0), np.sqrt(s), rtol=1e-12)
    assert np.allclose(np.linalg.norm(svh.reshape(k, -1), axis=1), np.sqrt(s), rtol=1e-12)


def test_truncated_product_error_is_eckart_young():
    s = np.linspace(5.0, 0.1, 30)
    A = planted(50, 40, s, 5)
    us, svh, dropped = oracle.split_node(A, [0], [1], max_singular_values=12)
    rec = us @ svh
    # 40 values: the 30 planted ones, then 10 zeros (rank 30)
    assert dropped.shape == (28,)
    assert np.allclose(dropped[:18], s[12:], rtol=1e-12) and np.all(dropped[18:] < 1e-12)
    assert np.linalg.norm(A - rec) == pytest.approx(np.sqrt(np.sum(s[12:] ** 2)), rel=1e-10)


@pytest.mark.parametrize("s,max_sv,max_err,k", [
    ([5, 3, 0.06, 0.03, 0.02], None, 0.1, 3),      # 0.02 + 0.03 <= 0.1, + 0.06 > 0.1
    ([5, 3, 0.06, 0.03, 0.02], None, 0.11, 2),     # all three fit exactly
    ([5, 3, 0.06, 0.03, 0.02], 2, None, 2),
    ([5, 3, 0.06, 0.03, 0.02], 4, 0.1, 3),         # the smaller of the two counts
    ([5, 3, 0.06, 0.03, 0.02], 1, 0.0, 1),
    ([5, 3, 0.06, 0.03, 0.02], None, 0.0, 5),      # nothing is <= 0 but zeros
    ([2, 1, 0, 0], None, 0.0, 2),                  # exact zeros are dropped by a zero limit
    ([0.05, 0.01], None, 1.0, 1),                  # at least one value is kept
    ([], None, 1.0, 0),
])
def test_truncation_rule(s, max_sv, max_err, k):
    assert oracle.truncation_count(s, max_sv, max_err) == k


def test_legs_must_partition_the_node():
    A = np.zeros((2, 3, 4))
    for left, right in (([0], [1]), ([0, 1], [1, 2]), ([0, 3], [1, 2])):
        with pytest.raises(ValueError):
            oracle.split_node(A, left, right)
