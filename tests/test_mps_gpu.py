"""GPU parity of the MPS inner-product and MPO-energy sweeps against the oracle.

Scalars are compared as value * exp(log_scale) on both sides, relative error
|x - x*| / |x*|. Tolerance of a sweep result made of c tensor-core
contractions: fp32 1e-5; bf16x3 2 * 2^-16 * sqrt(c); bf16 2 * 2^-8 * sqrt(c).
2^-16 is the per-contraction relative error of the three-term split (the
dropped lo*lo term and the rounding of lo), 2^-8 that of two bf16 roundings;
independent per-site errors add up like a random walk over the c steps.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1905_01330_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

UNIT = {"bf16x3": 2.0 ** -16, "bf16": 2.0 ** -8}


def tol(prec, contractions):
    if prec == "fp32":
        return 1e-5
    return 2.0 * UNIT[prec] * math.sqrt(contractions)


@pytest.fixture(scope="module")
def tn():
    from paper_1905_01330_gb300 import build, tn as tnmod
    build.build()
    tnmod.load()
    return tnmod


def to_dev(cores):
    return [torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in cores]


def rel(got, ref):
    return abs(got - ref) / abs(ref)


def val(r, j=0):
    r = r.cpu().numpy()
    return r[2 * j] * math.exp(r[2 * j + 1])


def test_config1_inner_product_small_chain(tn):
    # N=20, d=2, chi=32, cores N(0, 1/chi): the one-CTA float32 sweep
    cores = synth.random_mps(20, 2, 32, seed=1)
    v, lg = oracle.mps_inner(cores, cores)
    ref = v * math.exp(lg)
    # brute force over the 2^20 amplitudes pins the oracle here as well
    psi = oracle.mps_state(cores)
    assert rel(float(psi @ psi), ref) < 1e-10
    for prec in ("fp32", "bf16", "bf16x3"):
        r = tn.mps_inner(to_dev(cores), to_dev(cores), prec=prec)
        assert tn.sync_status() == 0
        assert rel(val(r), ref) <= 1e-5, prec


def test_overlap_of_different_states_small(tn):
    a = synth.random_mps(14, 2, 16, seed=3)
    b = synth.random_mps(14, 2, 24, seed=4)
    v, lg = oracle.mps_inner(a, b)
    r = tn.mps_inner(to_dev(a), to_dev(b), prec="fp32")
    assert rel(val(r), v * math.exp(lg)) <= 1e-5


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16"])
def test_inner_product_large_bond_contraction_path(tn, prec):
    # bonds above 64 run through the tensordot kernels with a workspace
    cores = synth.random_mps(16, 2, 96, seed=5)
    v, lg = oracle.mps_inner(cores, cores)
    r = tn.mps_inner(to_dev(cores), to_dev(cores), prec=prec)
    assert tn.sync_status() == 0
    assert rel(val(r), v * math.exp(lg)) <= tol(prec, 2 * 16)


def test_long_chain_log_scale(tn):
    # 400 sites of N(0,1) cores: the raw norm is far outside float32 range
    cores = synth.random_mps(400, 2, 8, seed=6, std=1.0)
    v, lg = oracle.mps_inner(cores, cores)
    r = tn.mps_inner(to_dev(cores), to_dev(cores), prec="fp32").cpu().numpy()
    assert lg > 200.0
    assert abs((math.log(r[0]) + r[1]) - (math.log(v) + lg)) <= 1e-4


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16"])
def test_tfim_energy_random_mps(tn, prec):
    n = 10
    cores = synth.random_mps(n, 2, 8, seed=7)
    W = synth.tfim_mpo(n)
    e, le = oracle.mpo_expect(cores, W)
    nv, ln = oracle.mps_inner(cores, cores)
    r = tn.mps_expect(to_dev(cores), to_dev(W), prec=prec)
    assert tn.sync_status() == 0
    # the energy per normalised state
    E_ref = e * math.exp(le) / (nv * math.exp(ln))
    E = val(r, 0) / val(r, 1)
    assert rel(val(r, 0), e * math.exp(le)) <= tol(prec, 2 * n), (E, E_ref)
    assert rel(val(r, 1), nv * math.exp(ln)) <= tol(prec, 2 * n)


def test_tfim_closed_forms_on_gpu(tn):
    n = 12
    W = synth.tfim_mpo(n)
    r2 = 1.0 / math.sqrt(2.0)
    for vec, E_exact in (([1.0, 0.0], -(n - 1)), ([r2, r2], -n)):
        cores = [np.asarray(vec, dtype=np.float32).reshape(1, 2, 1) for _ in range(n)]
        r = tn.mps_expect(to_dev(cores), to_dev(W), prec="fp32")
        assert abs(val(r, 0) / val(r, 1) - E_exact) <= 1e-5 * abs(E_exact)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16"])
def test_left_canonical_energy_large_bond(tn, prec):
    # config-5 shape at reduced length and bond: left-canonical, chi = 128
    n, chi = 16, 128
    cores = synth.left_canonical_mps(n, 2, chi, seed=5)
    W = synth.tfim_mpo(n)
    e, le = oracle.mpo_expect(cores, W)
    nv, ln = oracle.mps_inner(cores, cores)
    assert abs(nv * math.exp(ln) - 1.0) < n * 1e-6
    r = tn.mps_expect(to_dev(cores), to_dev(W), prec=prec)
    assert tn.sync_status() == 0
    assert rel(val(r, 0), e * math.exp(le)) <= tol(prec, 2 * n)
    assert abs(val(r, 1) - 1.0) <= tol(prec, 2 * n) + n * 1e-6


@pytest.mark.parametrize("chi,n", [(20, 12), (40, 12), (100, 16)])
@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_energy_ragged_bonds(tn, chi, n, prec):
    # Bonds whose step-(iii) operand (rows (w', b), shared (s', a')) ends in a
    # ragged row tile and a ragged 64-wide shared slab -- chi 20: 80 rows and
    # 40 shared indices, 40: 160 and 80, 100: 400 and 200 -- and bonds that
    # are not multiples of 8 (20, 100: one output column per thread in step
    # (ii)). The energy is bounded relative to ||H|| <psi|psi>, the norm (a
    # sum of squares) with the one-signed bias of its c = 2n contractions.
    cores = synth.left_canonical_mps(n, 2, chi, seed=11)
    W = synth.tfim_mpo(n)
    e, le = oracle.mpo_expect(cores, W)
    nv, ln = oracle.mps_inner(cores, cores)
    r = tn.mps_expect(to_dev(cores), to_dev(W), prec=prec)
    assert tn.sync_status() == 0
    norm = nv * math.exp(ln)
    h_norm = (n - 1) + n
    assert abs(val(r, 0) - e * math.exp(le)) <= tol(prec, 2 * n) * h_norm * norm
    bias = {"bf16x3": 2.0 ** -18, "bf16": 2.0 ** -16}[prec]
    assert rel(val(r, 1), norm) <= tol(prec, 2 * n) + 2 * n * bias


@pytest.mark.parametrize("n", [512, 600])
@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_energy_long_chain_both_launch_forms(tn, n, prec):
    # 512 sites: the most the one-launch persistent sweep takes (its site
    # table is a launch parameter); 600 sites: past it, so the sweep runs as
    # per-site launches. Same bound as the ragged-bond test.
    cores = synth.left_canonical_mps(n, 2, 16, seed=12)
    W = synth.tfim_mpo(n)
    e, le = oracle.mpo_expect(cores, W)
    nv, ln = oracle.mps_inner(cores, cores)
    r = tn.mps_expect(to_dev(cores), to_dev(W), prec=prec)
    assert tn.sync_status() == 0
    norm = nv * math.exp(ln)
    h_norm = (n - 1) + n
    assert abs(val(r, 0) - e * math.exp(le)) <= tol(prec, 2 * n) * h_norm * norm
    bias = {"bf16x3": 2.0 ** -18, "bf16": 2.0 ** -16}[prec]
    assert rel(val(r, 1), norm) <= tol(prec, 2 * n) + 2 * n * bias


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16"])
def test_energy_three_level_sites(tn, prec):
    # spin-1 sites (d = 3) with a bond-4 MPO: (bond + 1) d = 15, so the sweep
    # takes its general per-site launches. Bound as in the ragged-bond test,
    # with ||H|| <= 2 (n - 1) + h n (||Sz Sz|| = ||Sx Sx|| = 1, ||Sz|| = 1).
    n, d, chi, h = 8, 3, 12, 0.5
    cores = synth.random_mps(n, d, chi, seed=21)
    W = synth.spin1_xz_mpo(n, h=h)
    e, le = oracle.mpo_expect(cores, W)
    nv, ln = oracle.mps_inner(cores, cores)
    norm = nv * math.exp(ln)
    r = tn.mps_expect(to_dev(cores), to_dev(W), prec=prec)
    assert tn.sync_status() == 0
    assert abs(val(r, 0) - e * math.exp(le)) <= tol(prec, 2 * n) * (2 * (n - 1) + h * n) * norm
    assert rel(val(r, 1), norm) <= tol(prec, 2 * n)
    ri = tn.mps_inner(to_dev(cores), to_dev(cores), prec=prec).cpu().numpy()
    assert rel(ri[0] * math.exp(ri[1]), norm) <= tol(prec, 2 * n)


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16"])
def test_grouped_energy_uneven_bonds(tn, prec):
    # config-5 batch shape at reduced size: uneven chi (one smallest, one
    # largest forced), left-canonical states, one shared TFIM MPO
    n = 12
    chis = synth.uneven_chis(6, seed=50, lo=8, hi=48, step=8)
    assert min(chis) == 8 and max(chis) == 48
    states = [synth.left_canonical_mps(n, 2, chi, seed=60 + k) for k, chi in enumerate(chis)]
    W = synth.tfim_mpo(n)
    r = tn.mps_expect_grouped([to_dev(c) for c in states], to_dev(W), prec=prec)
    assert tn.sync_status() == 0
    r = r.cpu().numpy()
    assert r.shape == (len(chis), 4)
    # <psi|H|psi> is a sum of terms of both signs: its forward error is bounded
    # relative to the sum of their magnitudes, at most ||H|| <psi|psi> with
    # ||H|| <= J (n - 1) + h n, not relative to the (possibly small) sum itself
    h_norm = 1.0 * (n - 1) + 1.0 * n
    for k, cores in enumerate(states):
        e, le = oracle.mpo_expect(cores, W)
        nv, ln = oracle.mps_inner(cores, cores)
        norm = nv * math.exp(ln)
        err = abs(r[k, 0] * math.exp(r[k, 1]) - e * math.exp(le))
        assert err <= tol(prec, 2 * n) * h_norm * norm, (k, chis[k])
        assert rel(r[k, 2] * math.exp(r[k, 3]), norm) <= tol(prec, 2 * n), (k, chis[k])


@pytest.mark.parametrize("prec", ["fp32", "bf16x3", "bf16"])
def test_grouped_energy_three_level_sites(tn, prec):
    # spin-1 chains of uneven bonds in one grouped sweep (general step (ii):
    # (bond + 1) d = 15); bound as in the single-chain spin-1 test
    n, h = 8, 0.5
    states = [synth.random_mps(n, 3, chi, seed=90 + chi) for chi in (5, 12, 27)]
    W = synth.spin1_xz_mpo(n, h=h)
    r = tn.mps_expect_grouped([to_dev(c) for c in states], to_dev(W), prec=prec)
    assert tn.sync_status() == 0
    r = r.cpu().numpy()
    for k, cores in enumerate(states):
        e, le = oracle.mpo_expect(cores, W)
        nv, ln = oracle.mps_inner(cores, cores)
        norm = nv * math.exp(ln)
        err = abs(r[k, 0] * math.exp(r[k, 1]) - e * math.exp(le))
        assert err <= tol(prec, 2 * n) * (2 * (n - 1) + h * n) * norm, k
        assert rel(r[k, 2] * math.exp(r[k, 3]), norm) <= tol(prec, 2 * n), k


def test_grouped_energy_matches_single_sweeps(tn):
    # the grouped sweep and one tn_mps_expect per state agree (float32)
    n = 10
    states = [synth.random_mps(n, 2, chi, seed=70 + chi) for chi in (4, 16, 8)]
    W = synth.tfim_mpo(n)
    g = tn.mps_expect_grouped([to_dev(c) for c in states], to_dev(W), prec="fp32").cpu().numpy()
    for k, cores in enumerate(states):
        s = tn.mps_expect(to_dev(cores), to_dev(W), prec="fp32").cpu().numpy()
        for j in (0, 2):
            assert rel(g[k, j] * math.exp(g[k, j + 1]), s[j] * math.exp(s[j + 1])) <= 1e-5


def test_grouped_energy_rejects_mismatched_lengths(tn):
    W = synth.tfim_mpo(8)
    a = to_dev(synth.random_mps(8, 2, 4, seed=1))
    b = to_dev(synth.random_mps(9, 2, 4, seed=2))
    with pytest.raises(tn.TnError):
        tn.mps_expect_grouped([a, b], to_dev(W))


def test_grouped_energy_plan_runs_like_the_one_shot_call(tn):
    # planned once, run twice; core values changed in place are read by the next run
    n = 10
    states = [[torch.from_numpy(np.ascontiguousarray(c)).cuda() for c in synth.random_mps(n, 2, chi, seed=80 + chi)]
              for chi in (4, 16, 8)]
    W = to_dev(synth.tfim_mpo(n))
    plan = tn.ExpectGroupedPlan(states, W, prec="fp32")
    a = plan.run().cpu().numpy()
    b = plan.run().cpu().numpy()
    ref = tn.mps_expect_grouped(states, W, prec="fp32").cpu().numpy()
    assert np.array_equal(a, b)
    for k in range(3):
        for j in (0, 2):
            assert rel(a[k, j] * math.exp(a[k, j + 1]), ref[k, j] * math.exp(ref[k, j + 1])) <= 1e-6
    states[1][3].mul_(2.0)  # <psi|H|psi> and <psi|psi> of state 1 scale by 4
    c = plan.run().cpu().numpy()
    assert tn.sync_status() == 0
    for j in (0, 2):
        assert rel(c[1, j] * math.exp(c[1, j + 1]), 4.0 * a[1, j] * math.exp(a[1, j + 1])) <= 1e-5
        assert rel(c[0, j] * math.exp(c[0, j + 1]), a[0, j] * math.exp(a[0, j + 1])) <= 1e-12
