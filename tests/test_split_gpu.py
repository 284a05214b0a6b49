"""GPU parity of node splitting (tn_split_node, Sec. III.B "Node Splitting",
Appendix A) against the FP64 oracle on the same float32 inputs.

What is unique is compared: the singular values (kept and dropped), the kept
count (the truncation rule applied to the GPU's own values must give the
GPU's count exactly, and the oracle's count where no limit sits near a partial
sum), and the truncated product U S V^T when the kept and dropped values are
separated. Singular vectors are unique only up to sign, so they are checked
for what must hold instead: orthonormal columns of U and rows of V^T (for
non-zero values) and sqrt(S) carried on both sides by split_node.

Tolerances (float32 one-sided Jacobi, rotation angles in float64): singular
values within 5e-5 of the largest one; products within 5e-5 of |A|_F;
orthonormality within 1e-4.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    from paper_1905_01330_gb300 import build, tn as tnmod
    build.build()
    tnmod.load()
    return tnmod


def planted(m, n, s, seed):
    rng = np.random.default_rng(seed)
    r = len(s)
    q1, _ = np.linalg.qr(rng.standard_normal((m, r)))
    q2, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return ((q1 * np.asarray(s)[None, :]) @ q2.T).astype(np.float32)


def check(tn, A, left, right, max_sv=None, max_err=None, At=None, expect_k=None):
    """A: float32 numpy array (the node's values); At: the device tensor (a view) if not A itself."""
    At = torch.from_numpy(A).cuda() if At is None else At
    info = {}
    us, svh, drop = tn.split_node(At, left, right, max_sv, max_err, info=info)
    u, s, vh, drop2 = tn.split_node(At, left, right, max_sv, max_err, full_svd=True)
    torch.cuda.synchronize()
    assert info["sweeps"] > 0
    mat, ldims, rdims = oracle.matrix_view(A.astype(np.float64), left, right)
    U, S, Vt, _, _ = oracle.svd(A.astype(np.float64), left, right)
    r = len(S)
    k = us.shape[-1]
    assert list(us.shape) == ldims + [k] and list(svh.shape) == [k] + rdims
    assert list(u.shape) == ldims + [k] and list(vh.shape) == [k] + rdims
    assert s.shape == (k,) and drop.shape == (r - k,) and drop2.shape == (r - k,)
    sg = np.concatenate([s.cpu().numpy(), drop2.cpu().numpy()]).astype(np.float64)
    assert np.array_equal(drop.cpu().numpy(), drop2.cpu().numpy())
    smax = max(S[0], 1e-30)
    assert np.all(np.diff(sg) <= 0)
    assert np.abs(sg - S).max() <= 5e-5 * smax, np.abs(sg - S).max() / smax
    # the kept count: the rule on the GPU's own values, and the oracle's count
    assert k == oracle.truncation_count([float(v) for v in s.cpu().numpy()] + [float(v) for v in drop2.cpu().numpy()],
                                        max_sv, max_err)
    k_or = oracle.truncation_count(S, max_sv, max_err)
    assert k == (k_or if expect_k is None else expect_k)
    if k == 0:
        return
    # truncated product against the oracle's, when the cut separates the values
    nrm = max(np.linalg.norm(mat), 1e-30)
    rec = us.reshape(-1, k).double().cpu().numpy() @ svh.reshape(k, -1).double().cpu().numpy()
    rec_or = (U[:, :k] * S[:k]) @ Vt[:k]
    if k == r or S[k - 1] - S[k] > 1e-3 * smax:
        assert np.linalg.norm(rec - rec_or) <= 5e-5 * nrm
    rec_full = u.reshape(-1, k).double().cpu().numpy() @ np.diag(s.double().cpu().numpy()) @ \
        vh.reshape(k, -1).double().cpu().numpy()
    assert np.linalg.norm(rec_full - rec) <= 5e-5 * nrm
    # orthonormal factors for the non-zero values; sqrt(S) on both sides
    nz = s.cpu().numpy() > 1e-3 * smax
    Ug = u.reshape(-1, k).double().cpu().numpy()[:, nz]
    Vg = vh.reshape(k, -1).double().cpu().numpy()[nz]
    assert np.abs(Ug.T @ Ug - np.eye(Ug.shape[1])).max() <= 1e-4
    assert np.abs(Vg @ Vg.T - np.eye(Vg.shape[0])).max() <= 1e-4
    root = np.sqrt(s.double().cpu().numpy())
    assert np.allclose(np.linalg.norm(us.reshape(-1, k).double().cpu().numpy(), axis=0)[nz], root[nz], rtol=1e-4)
    assert np.allclose(np.linalg.norm(svh.reshape(k, -1).double().cpu().numpy(), axis=1)[nz], root[nz], rtol=1e-4)


def rand(seed, shape):
    return np.random.default_rng(seed).standard_normal(shape).astype(np.float32)


def test_paper_shapes(tn):
    A = rand(1, (2, 3, 4, 5, 6))
    check(tn, A, [0, 1, 2], [3, 4])                     # (2,3,4,24) and (24,5,6)


@pytest.mark.parametrize("shape,left,right", [
    ((50, 20), [0], [1]),              # M > N: W is the matrix view
    ((20, 50), [0], [1]),              # M < N: W is its transpose
    ((64, 64), [1], [0]),              # square, legs swapped
    ((6, 5, 8), [2, 0], [1]),          # left legs out of order
    ((3, 4, 5, 2), [3, 1], [0, 2]),
    ((1, 50), [0], [1]), ((50, 1), [0], [1]),           # one singular value
    ((33, 7, 3), [0], [1, 2]),         # odd r: a dummy slot in every round
])
def test_random_nodes(tn, shape, left, right):
    check(tn, rand(2, shape), left, right)


@pytest.mark.parametrize("shape", [(256, 256), (512, 512), (700, 650)])
def test_two_site_sizes(tn, shape):
    """Square and near-square nodes of the sizes a two-site split of an MPS
    sweep meets (chi = 128, 256): hundreds of rounds per sweep."""
    check(tn, rand(9, shape), [0], [1])


def test_strided_view(tn):
    base = rand(3, (8, 6, 10))
    At = torch.from_numpy(base).cuda().permute(2, 0, 1)[:, ::2]   # (10, 4, 6), non-contiguous
    A = np.ascontiguousarray(base.transpose(2, 0, 1)[:, ::2])
    check(tn, A, [1, 0], [2], At=At)


def test_rank_deficient(tn):
    rng = np.random.default_rng(4)
    A = np.multiply.outer(rng.standard_normal(30), rng.standard_normal(40)).astype(np.float32)
    check(tn, A, [0], [1])
    check(tn, A, [0], [1], max_err=1e-3, expect_k=1)    # the zeros (and rounding noise) dropped


def test_truncation(tn):
    s = np.linspace(4.0, 0.02, 200)
    A = planted(300, 200, s, 5)
    check(tn, A, [0], [1], max_sv=5)
    # limit halfway between two partial sums of the tail: no rounding decides k
    tail = np.cumsum(s[::-1])
    check(tn, A, [0], [1], max_err=0.5 * (tail[59] + tail[60]))
    check(tn, A, [0], [1], max_sv=100, max_err=0.5 * (tail[59] + tail[60]))


def test_paper_truncation_example(tn):
    """Appendix A: a (1000, 1000) node with max_singular_values=5 keeps 5 and
    drops 995 (largest size in this suite)."""
    A = planted(1000, 1000, 0.99 ** np.arange(1000), 6)
    us, svh, drop = tn.split_node(torch.from_numpy(A).cuda(), [0], [1], max_singular_values=5)
    assert tuple(us.shape) == (1000, 5) and tuple(svh.shape) == (5, 1000) and tuple(drop.shape) == (995,)
    check(tn, A, [0], [1], max_sv=5)


def test_empty_node(tn):
    At = torch.empty((0, 5), device="cuda")
    us, svh, drop = tn.split_node(At, [0], [1])
    assert tuple(us.shape) == (0, 0) and tuple(svh.shape) == (0, 5) and drop.numel() == 0


def test_legs_must_partition(tn):
    At = torch.zeros((2, 3, 4), device="cuda")
    with pytest.raises(tn.TnError):
        tn.split_node(At, [0], [1])
