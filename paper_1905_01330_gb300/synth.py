"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds no arithmetic of the method itself: it only draws random
numbers and lays them out as the tensors, contraction specs, matrix product
states (MPS), matrix product operators (MPO) and pixel batches that the
workloads are made of. Both sides of every parity test take their inputs from
here, so the GPU kernels and the oracle see bit-identical values.

Generator: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), used in its
counter form -- draw ``i`` of a stream with seed ``s`` is
``mix(s + (i + 1) * 0x9E3779B97F4A7C15)`` -- so any slice of a stream can be
produced without producing what precedes it. Uniform doubles take the top 53
bits. Normals use the Box-Muller transform (Box and Muller, 1958) on pairs of
uniforms. Values are produced in float64 and rounded to float32 once.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK = (1 << 64) - 1


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+n-1`` of the SplitMix64 stream ``seed`` (uint64)."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + i * _GOLDEN
    return _mix(z)


def substream(seed: int, tag: int) -> int:
    """A seed for an independent stream derived from ``seed`` and a small tag."""
    return int(splitmix64((seed * 1000003 + tag) & _MASK, 1)[0])


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` float64 uniforms in [0, 1) from stream ``seed``."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int, std: float = 1.0) -> np.ndarray:
    """``n`` float64 N(0, std^2) values by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 lies in (0, 1]
    z = np.empty(2 * m, dtype=np.float64)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:n] * std


def normal_f32(seed: int, shape, std: float = 1.0) -> np.ndarray:
    n = int(np.prod(shape)) if len(shape) else 1
    return normal(seed, n, std).astype(np.float32).reshape(shape)


class Stream:
    """Sequential integer draws from one SplitMix64 stream (for small host decisions)."""

    def __init__(self, seed: int):
        self.seed = seed & _MASK
        self.i = 0

    def u64(self) -> int:
        v = int(splitmix64(self.seed, 1, self.i)[0])
        self.i += 1
        return v

    def below(self, n: int) -> int:
        """Uniform integer in [0, n) (multiply-shift; bias < 2^-50 for small n)."""
        return (self.u64() >> 11) * n >> 53

    def choice(self, seq):
        return seq[self.below(len(seq))]

    def sample(self, n: int, k: int) -> list[int]:
        """k distinct values of range(n) in random order (partial Fisher-Yates)."""
        pool = list(range(n))
        for j in range(k):
            r = j + self.below(n - j)
            pool[j], pool[r] = pool[r], pool[j]
        return pool[:k]


# ---------------------------------------------------------------------------
# Pairwise tensordot specs (random ranks, dims, leg positions and pairings)
# ---------------------------------------------------------------------------

SPEC_DIMS = (8, 16, 24, 32, 48, 64)
SPEC_CAP = 1 << 24  # elements per operand and per result; larger draws are redrawn


def contraction_spec(st: Stream, dims=SPEC_DIMS, cap=SPEC_CAP):
    """One random spec: (shapeA, legsA, shapeB, legsB).

    Ranks rA, rB ~ U{3,4,5}; shared legs k ~ U{1,2,3}; every dim ~ U(dims).
    legsA lists the shared legs of A in random order, legsB the legs of B they
    pair with (legsA[j] <-> legsB[j]); B takes the paired dims from A. A spec
    whose A, B or result exceeds ``cap`` elements is drawn again from the same
    stream.
    """
    while True:
        ra = 3 + st.below(3)
        rb = 3 + st.below(3)
        k = 1 + st.below(3)
        sha = [st.choice(dims) for _ in range(ra)]
        legsa = st.sample(ra, k)
        legsb = st.sample(rb, k)
        shb = [0] * rb
        for j in range(k):
            shb[legsb[j]] = sha[legsa[j]]
        for p in range(rb):
            if shb[p] == 0:
                shb[p] = st.choice(dims)
        na = int(np.prod(sha))
        nb = int(np.prod(shb))
        kk = int(np.prod([sha[p] for p in legsa]))
        nc = (na // kk) * (nb // kk)
        if na <= cap and nb <= cap and nc <= cap:
            return tuple(sha), tuple(legsa), tuple(shb), tuple(legsb)


def contraction_specs(n: int = 2048, seed: int = 2, dims=SPEC_DIMS, cap=SPEC_CAP):
    st = Stream(seed)
    return [contraction_spec(st, dims, cap) for _ in range(n)]


def spec_sizes(spec):
    """(M, N, K) of the GEMM view of a spec, and its element counts."""
    sha, legsa, shb, legsb = spec
    k = int(np.prod([sha[p] for p in legsa])) if legsa else 1
    na, nb = int(np.prod(sha)), int(np.prod(shb))
    return na // k, nb // k, k


# ---------------------------------------------------------------------------
# Matrix product states and operators
# ---------------------------------------------------------------------------

def mps_bonds(n_sites: int, d: int, chi: int) -> list[int]:
    """Open-boundary bond dims D_0..D_N with D_i = min(chi, d^i, d^(N-i))."""
    out = []
    for i in range(n_sites + 1):
        out.append(int(min(chi, d ** min(i, 60), d ** min(n_sites - i, 60))))
    return out


def random_mps(n_sites: int, d: int, chi: int, seed: int, std: float | None = None):
    """Cores (D_{i-1}, d, D_i) float32 with i.i.d. N(0, std^2), std = 1/sqrt(chi) by default."""
    if std is None:
        std = 1.0 / math.sqrt(chi)
    bonds = mps_bonds(n_sites, d, chi)
    cores = []
    for i in range(n_sites):
        shape = (bonds[i], d, bonds[i + 1])
        cores.append(normal_f32(substream(seed, i), shape, std))
    return cores


def left_canonical_mps(n_sites: int, d: int, chi: int, seed: int):
    """Left-canonical random MPS: per site, Q of the Householder QR of a Gaussian
    (D_{i-1} d) x D_i matrix, with the columns signed so that R has a positive
    diagonal; built in float64 and rounded to float32 once. The last site is
    normalised as a vector (D_N = 1)."""
    bonds = mps_bonds(n_sites, d, chi)
    cores = []
    for i in range(n_sites):
        rows, cols = bonds[i] * d, bonds[i + 1]
        g = normal(substream(seed, i), rows * cols).reshape(rows, cols)
        q, r = np.linalg.qr(g)
        sgn = np.sign(np.diag(r))
        sgn[sgn == 0] = 1.0
        q = q * sgn[None, :]
        cores.append(q.reshape(bonds[i], d, cols).astype(np.float32))
    return cores


def uneven_chis(count: int = 64, seed: int = 50, lo: int = 64, hi: int = 512, step: int = 32):
    """Bond dims for a batch of MPS: U{lo, lo+step, ..., hi}, with one lo and one hi forced."""
    st = Stream(seed)
    choices = list(range(lo, hi + 1, step))
    chis = [st.choice(choices) for _ in range(count)]
    if count >= 2:
        chis[0], chis[1] = lo, hi
    return chis


def tfim_mpo(n_sites: int, J: float = 1.0, h: float = 1.0):
    """MPO of H = -J sum Z_i Z_{i+1} - h sum X_i on an open chain, bond dim 3.

    Bulk tensor (w_left, w_right, s, s') = [[I,0,0],[Z,0,0],[-hX,-JZ,I]];
    the first site keeps row 2, the last site keeps column 0. float32.
    """
    I = np.eye(2)
    X = np.array([[0.0, 1.0], [1.0, 0.0]])
    Z = np.array([[1.0, 0.0], [0.0, -1.0]])
    W = np.zeros((3, 3, 2, 2))
    W[0, 0] = I
    W[1, 0] = Z
    W[2, 0] = -h * X
    W[2, 1] = -J * Z
    W[2, 2] = I
    cores = []
    for i in range(n_sites):
        w = W
        if i == 0:
            w = w[2:3]
        if i == n_sites - 1:
            w = w[:, 0:1]
        cores.append(np.ascontiguousarray(w).astype(np.float32))
    return cores


def spin1_xz_mpo(n_sites: int, h: float = 0.5):
    """MPO of H = sum (Sz_i Sz_{i+1} + Sx_i Sx_{i+1}) - h sum Sz_i for spin-1
    sites (d = 3, basis m = +1, 0, -1) on an open chain, bond dim 4.

    Bulk tensor (w_left, w_right, s, s') = [[I,0,0,0],[Sz,0,0,0],[Sx,0,0,0],
    [-h Sz, Sz, Sx, I]]; the first site keeps row 3, the last site keeps
    column 0. Every operator is real symmetric. float32.
    """
    I = np.eye(3)
    r = 1.0 / np.sqrt(2.0)
    Sx = np.array([[0.0, r, 0.0], [r, 0.0, r], [0.0, r, 0.0]])
    Sz = np.diag([1.0, 0.0, -1.0])
    W = np.zeros((4, 4, 3, 3))
    W[0, 0] = I
    W[1, 0] = Sz
    W[2, 0] = Sx
    W[3, 0] = -h * Sz
    W[3, 1] = Sz
    W[3, 2] = Sx
    W[3, 3] = I
    cores = []
    for i in range(n_sites):
        w = W
        if i == 0:
            w = w[3:4]
        if i == n_sites - 1:
            w = w[:, 0:1]
        cores.append(np.ascontiguousarray(w).astype(np.float32))
    return cores


# ---------------------------------------------------------------------------
# MPS classifier inputs
# ---------------------------------------------------------------------------

def pixels(batch: int, n_pixels: int, seed: int) -> np.ndarray:
    """Greyscale pixels uniform in [0, 1), float32 [batch, n_pixels]."""
    return uniform(seed, batch * n_pixels).astype(np.float32).reshape(batch, n_pixels)


def labels(batch: int, n_labels: int, seed: int) -> np.ndarray:
    st = uniform(seed, batch)
    return np.minimum((st * n_labels).astype(np.int64), n_labels - 1)


def classifier_mps(n_sites: int, chi: int, label_site: int, n_labels: int, seed: int,
                   eps_std: float = 0.1, d: int = 2, constant_bond: bool = True):
    """Classifier MPS near the identity: A[a,s,b] = delta_ab + eps, eps ~ N(0, eps_std^2).

    Edge cores have a bond of 1 (A[0,s,b] = delta_0b + eps, A[a,s,0] = delta_a0 + eps).
    The label core at ``label_site`` has shape (chi, d, n_labels, chi) with
    C[a,s,l,b] = delta_ab + eps. Inner bonds are ``chi`` (constant_bond) so every
    bulk site is the same GEMM shape.
    """
    bonds = [1] + [chi] * (n_sites - 1) + [1]
    cores = []
    for i in range(n_sites):
        a, b = bonds[i], bonds[i + 1]
        shape = (a, d, n_labels, b) if i == label_site else (a, d, b)
        eps = normal(substream(seed, i), int(np.prod(shape)), eps_std).reshape(shape)
        eye = np.zeros((a, b))
        for j in range(min(a, b)):
            eye[j, j] = 1.0
        if i == label_site:
            core = eye[:, None, None, :] + eps
        else:
            core = eye[:, None, :] + eps
        cores.append(core.astype(np.float32))
    return cores


def classifier_separate_mps(n_sites: int, chi: int, n_labels: int, seed: int, eps_std: float = 0.1,
                            d: int = 2):
    """One MPS per label (the paper's L separate MPS), each near the identity
    like classifier_mps without a label core: n_labels lists of n_sites cores
    (D, d, D'), MPS l drawn from substream (seed, l)."""
    return [classifier_mps(n_sites, chi, -1, 1, substream(seed, 1000 + l), eps_std, d) for l in range(n_labels)]
