"""Pins for the oracle's MPS inner product, MPO expectation and state vector (CPU)."""
import math

import numpy as np
import pytest

import oracle
from paper_1905_01330_gb300 import synth


def product_state(n, vec):
    """MPS with bond 1 everywhere: every core is (1, 2, 1) holding ``vec``."""
    return [np.asarray(vec, dtype=np.float64).reshape(1, 2, 1) for _ in range(n)]


def test_mps_state_matches_explicit_matrix_products():
    cores = synth.random_mps(3, 2, 2, seed=7)
    psi = oracle.mps_state(cores)
    for s1 in range(2):
        for s2 in range(2):
            for s3 in range(2):
                m = cores[0][:, s1, :].astype(np.float64) @ cores[1][:, s2, :] @ cores[2][:, s3, :]
                assert abs(psi[s1 * 4 + s2 * 2 + s3] - m[0, 0]) < 1e-12


def test_product_state_vector_is_kronecker_product():
    v = np.array([0.6, -0.8])
    psi = oracle.mps_state(product_state(4, v))
    ref = v
    for _ in range(3):
        ref = np.kron(ref, v)
    np.testing.assert_allclose(psi, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n,chi", [(6, 4), (10, 8), (20, 32)])
def test_inner_product_against_brute_force(n, chi):
    cores = synth.random_mps(n, 2, chi, seed=1)
    v, lg = oracle.mps_inner(cores, cores)
    psi = oracle.mps_state(cores)
    ref = float(np.dot(psi, psi))
    assert v > 0.0
    assert abs(v * math.exp(lg) - ref) <= 1e-10 * ref


def test_overlap_of_two_states_and_symmetry():
    a = synth.random_mps(8, 2, 6, seed=3)
    b = synth.random_mps(8, 2, 4, seed=4)
    v1, l1 = oracle.mps_inner(a, b)
    v2, l2 = oracle.mps_inner(b, a)
    ref = float(np.dot(oracle.mps_state(a), oracle.mps_state(b)))
    assert abs(v1 * math.exp(l1) - ref) <= 1e-10 * abs(ref)
    assert abs(v2 * math.exp(l2) - ref) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("n,chi", [(12, 8), (30, 16)])
def test_left_canonical_norm_is_one(n, chi):
    cores = synth.left_canonical_mps(n, 2, chi, seed=5)
    # canonical in float64 before rounding; float32 rounding moves it by ~1e-7 per site
    v, lg = oracle.mps_inner(cores, cores)
    assert abs(v * math.exp(lg) - 1.0) <= n * 1e-6


def test_dense_tfim_hand_cases():
    # single site: H = -h X; <0|H|0> = 0, <+|H|+> = -h
    assert oracle.tfim_energy_dense(1, 1.0, 0.7, np.array([1.0, 0.0])) == 0.0
    r = 1.0 / math.sqrt(2.0)
    assert abs(oracle.tfim_energy_dense(1, 1.0, 0.7, np.array([r, r])) + 0.7) < 1e-15
    # two sites: |00> -> -J (ZZ = +1); |01> -> +J
    assert oracle.tfim_energy_dense(2, 1.5, 0.3, np.array([1.0, 0, 0, 0])) == -1.5
    assert oracle.tfim_energy_dense(2, 1.5, 0.3, np.array([0, 1.0, 0, 0])) == 1.5
    # |00> + |11> over sqrt 2: ZZ = +1; X on either site maps into |10>,|01>: zero overlap
    assert abs(oracle.tfim_energy_dense(2, 1.0, 1.0, np.array([r, 0, 0, r])) + 1.0) < 1e-15


@pytest.mark.parametrize("n", [2, 5, 9])
def test_tfim_closed_forms_via_mpo(n):
    W = synth.tfim_mpo(n, J=1.0, h=1.0)
    v, lg = oracle.mpo_expect(product_state(n, [1.0, 0.0]), W)
    assert abs(v * math.exp(lg) - (-(n - 1))) < 1e-12   # |0..0>: E = -J (N-1)
    r = 1.0 / math.sqrt(2.0)
    v, lg = oracle.mpo_expect(product_state(n, [r, r]), W)
    assert abs(v * math.exp(lg) - (-n)) < 1e-12         # |+..+>: E = -h N


@pytest.mark.parametrize("n,seed", [(1, 11), (2, 12), (3, 13), (8, 14)])
def test_tfim_product_state_closed_form(n, seed):
    # site i in cos(t_i)|0> + sin(t_i)|1>: <Z_i> = cos 2t_i, <X_i> = sin 2t_i, and
    # a product state factorises <Z_i Z_i+1>, so
    # E = -J sum_i cos 2t_i cos 2t_i+1 - h sum_i sin 2t_i
    t = np.random.default_rng(seed).uniform(-math.pi, math.pi, n)
    J, h = 0.75, 1.25   # exact in float32, so the MPO holds them exactly
    cores = [np.array([math.cos(a), math.sin(a)]).reshape(1, 2, 1) for a in t]
    v, lg = oracle.mpo_expect(cores, synth.tfim_mpo(n, J=J, h=h))
    ref = -J * sum(math.cos(2 * t[i]) * math.cos(2 * t[i + 1]) for i in range(n - 1)) \
        - h * sum(math.sin(2 * a) for a in t)
    assert abs(v * math.exp(lg) - ref) < 1e-12


@pytest.mark.parametrize("n,seed", [(2, 31), (5, 32)])
def test_spin1_mpo_energy_against_dense_hamiltonian(n, seed):
    # d = 3: the state by explicit matrix products (numpy einsum) and H as a
    # dense sum of Kronecker products, with the MPO's float32 entries
    cores = synth.random_mps(n, 3, 6, seed=seed)
    psi = cores[0].astype(np.float64)[0]                      # (s1, D1)
    for c in cores[1:]:
        psi = np.einsum("xa,asb->xsb", psi, c.astype(np.float64)).reshape(-1, c.shape[2])
    psi = psi[:, 0]
    r = float(np.float32(1.0 / math.sqrt(2.0)))
    Sx = np.array([[0.0, r, 0.0], [r, 0.0, r], [0.0, r, 0.0]])
    Sz = np.diag([1.0, 0.0, -1.0])
    h = 0.5

    def site_op(ops):   # {site: operator} as a 3^n x 3^n matrix
        m = np.eye(1)
        for i in range(n):
            m = np.kron(m, ops.get(i, np.eye(3)))
        return m

    H = -h * sum(site_op({i: Sz}) for i in range(n))
    for i in range(n - 1):
        H = H + site_op({i: Sz, i + 1: Sz}) + site_op({i: Sx, i + 1: Sx})
    ref = float(psi @ H @ psi)
    v, lg = oracle.mpo_expect(cores, synth.spin1_xz_mpo(n, h=h))
    assert abs(v * math.exp(lg) - ref) <= 1e-10 * max(1.0, abs(ref))
    nv, ln = oracle.mps_inner(cores, cores)
    assert abs(nv * math.exp(ln) - float(psi @ psi)) <= 1e-10 * float(psi @ psi)


@pytest.mark.parametrize("n,chi,seed", [(6, 4, 1), (10, 8, 2), (12, 16, 3)])
def test_mpo_energy_against_dense_hamiltonian(n, chi, seed):
    cores = synth.random_mps(n, 2, chi, seed=seed)
    W = synth.tfim_mpo(n, J=1.0, h=1.0)
    v, lg = oracle.mpo_expect(cores, W)
    psi = oracle.mps_state(cores)
    ref = oracle.tfim_energy_dense(n, 1.0, 1.0, psi)
    assert abs(v * math.exp(lg) - ref) <= 1e-10 * max(1.0, abs(ref))
    # |E| / <psi|psi> is bounded by J (N-1) + h N
    norm = float(psi @ psi)
    assert abs(ref) / norm <= (n - 1) + n + 1e-9


def test_mpo_with_other_couplings_against_dense():
    n = 7
    cores = synth.random_mps(n, 2, 4, seed=9)
    W = synth.tfim_mpo(n, J=0.7, h=1.3)
    v, lg = oracle.mpo_expect(cores, W)
    # the MPO holds J and h rounded to float32
    ref = oracle.tfim_energy_dense(n, float(np.float32(0.7)), float(np.float32(1.3)), oracle.mps_state(cores))
    assert abs(v * math.exp(lg) - ref) <= 1e-10 * max(1.0, abs(ref))


def test_stored_energy_values_are_the_oracles():
    # tests/golden/energy_oracle.txt is written by make_energy_oracle.py from
    # oracle.mpo_expect / oracle.mps_inner; recompute its cheapest row (the
    # batch's chi = 64 state, N = 100) and check value and input fingerprint
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "energy_oracle.txt")
    rows = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows[parts[0]] = [float(x) for x in parts[1:]]
    chi, n, seed, e, le, v, lv, s, q = rows["batch0_chi64_n100"]
    cores = synth.left_canonical_mps(int(n), 2, int(chi), seed=int(seed))
    assert abs(sum(float(np.sum(c, dtype=np.float64)) for c in cores) - s) <= 1e-6 * abs(s)
    assert abs(sum(float(np.sum(c.astype(np.float64) ** 2)) for c in cores) - q) <= 1e-9 * q
    e2, le2 = oracle.mpo_expect(cores, synth.tfim_mpo(int(n)))
    v2, lv2 = oracle.mps_inner(cores, cores)
    assert abs(e2 * np.exp(le2) - e * np.exp(le)) <= 1e-12 * (2 * n)
    assert abs(v2 * np.exp(lv2) - v * np.exp(lv)) <= 1e-12
    # every stored state is left-canonical: its norm is 1 to float32 rounding
    for key, (chi, n, seed, e, le, v, lv, s, q) in rows.items():
        assert abs(v * np.exp(lv) - 1.0) <= n * 1e-6, key
        assert abs(e * np.exp(le)) <= (2 * n - 1), key  # |E| <= ||H|| for a unit state
