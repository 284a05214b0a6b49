"""FP64 oracle of node splitting -- TEST INFRASTRUCTURE (tests, smoke and the
bench's CPU leg only; the GPU library never imports it).

Node splitting (TensorNetwork paper, Sec. III.B "Node Splitting"): the legs of
a node are grouped into a left and a right effective leg, the node is read as
the matrix whose rows run over the left legs (in the order given, last
fastest) and whose columns run over the right legs, and that matrix is
decomposed by the singular value decomposition A = U S V^T. The new bond has
dimension min(prod left dims, prod right dims) before truncation.

 * split_node: the two new nodes hold U sqrt(S) (shape left dims + (k,)) and
   sqrt(S) V^T (shape (k,) + right dims).
 * split_node_full_svd: three nodes U, S, V^T; S is returned as its diagonal.

Truncation (Appendix A "Saving Memory"): max_singular_values keeps at most
that many values; max_truncation_err drops the smallest singular values whose
sum does not exceed it. The dropped values are returned (descending), so that
the 1000 x 1000 node split with max_singular_values=5 returns 995 of them.
Readings where the paper is silent: with both limits the kept count is the
smaller of the two; at least one singular value is always kept.

The decomposition step is LAPACK's SVD through numpy (a library primitive, in
float64); the grouping, ordering, truncation and the absorption of sqrt(S)
are written out here.
"""
from __future__ import annotations

import numpy as np


def truncation_count(s_desc, max_singular_values=None, max_truncation_err=None) -> int:
    """How many of the singular values s_desc (descending) are kept.

    max_truncation_err: drop values from the smallest upwards while the sum of
    the dropped ones stays <= max_truncation_err (Appendix A). Then keep at
    most max_singular_values. At least one value is kept when there is any.
    """
    s = [float(v) for v in s_desc]
    k = len(s)
    if max_truncation_err is not None and max_truncation_err >= 0:
        dropped = 0.0
        while k > 0 and dropped + s[k - 1] <= max_truncation_err:
            dropped += s[k - 1]
            k -= 1
    if max_singular_values is not None and max_singular_values > 0:
        k = min(k, int(max_singular_values))
    if len(s) > 0:
        k = max(k, 1)
    return k


def matrix_view(A, left_legs, right_legs):
    """The node as a matrix: rows over left_legs (given order), columns over right_legs."""
    A = np.asarray(A, dtype=np.float64)
    left, right = list(left_legs), list(right_legs)
    if sorted(left + right) != list(range(A.ndim)):
        raise ValueError("left and right legs must partition the node's legs")
    ldims = [A.shape[p] for p in left]
    rdims = [A.shape[p] for p in right]
    M = int(np.prod(ldims)) if ldims else 1
    N = int(np.prod(rdims)) if rdims else 1
    return np.transpose(A, left + right).reshape(M, N), ldims, rdims


def svd(A, left_legs, right_legs):
    """(U, S, Vt, left dims, right dims) of the node's matrix view, S descending, r = min(M, N)."""
    mat, ldims, rdims = matrix_view(A, left_legs, right_legs)
    U, S, Vt = np.linalg.svd(mat, full_matrices=False)
    return U, S, Vt, ldims, rdims


def split_node(A, left_legs, right_legs, max_singular_values=None, max_truncation_err=None,
               full_svd=False):
    """split_node -> (u_s, s_vh, dropped); full_svd -> (u, s, vh, dropped)."""
    U, S, Vt, ldims, rdims = svd(A, left_legs, right_legs)
    k = truncation_count(S, max_singular_values, max_truncation_err)
    u, s, vt, dropped = U[:, :k], S[:k], Vt[:k], S[k:].copy()
    if full_svd:
        return u.reshape(ldims + [k]), s.copy(), vt.reshape([k] + rdims), dropped
    root = np.sqrt(s)
    return (u * root[None, :]).reshape(ldims + [k]), (root[:, None] * vt).reshape([k] + rdims), dropped
