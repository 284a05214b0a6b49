"""Failure detection without a GPU fault: a bounded device wait that nothing
satisfies gives up, reports TN_ERR_TIMEOUT through the status word, and the
context stays usable for the next contraction. Two waits: an mbarrier phase
nothing completes, and the persistent energy sweep's device-wide barrier with
one CTA that never arrives."""
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


def test_bounded_wait_reports_timeout_and_recovers(tn):
    assert tn.sync_status() == 0
    tn.check_wait_timeout(20_000_000)  # 20 ms
    assert tn.sync_status() == 5       # TN_ERR_TIMEOUT, read and cleared
    assert tn.sync_status() == 0
    A = synth.normal_f32(1, (64, 48))
    B = synth.normal_f32(2, (48, 40))
    C = tn.contract(torch.from_numpy(A).cuda(), [1], torch.from_numpy(B).cuda(), [0], prec="bf16x3")
    assert tn.sync_status() == 0
    ref = oracle.tensordot(A, [1], B, [0])
    assert np.linalg.norm(C.double().cpu().numpy() - ref) <= 5e-5 * np.linalg.norm(ref)


def test_grid_barrier_reports_timeout_and_recovers(tn):
    assert tn.sync_status() == 0
    tn.check_grid_barrier_timeout(20_000_000)  # 20 ms
    assert tn.sync_status() == 5               # TN_ERR_TIMEOUT, read and cleared
    assert tn.sync_status() == 0
    # the next persistent sweep on the same context is correct
    n = 12
    cores = synth.left_canonical_mps(n, 2, 16, seed=3)
    W = synth.tfim_mpo(n)
    e, le = oracle.mpo_expect(cores, W)
    r = tn.mps_expect([torch.from_numpy(c).cuda() for c in cores], [torch.from_numpy(w).cuda() for w in W],
                      prec="bf16x3").cpu().numpy()
    assert tn.sync_status() == 0
    assert abs(r[0] * math.exp(r[1]) - e * math.exp(le)) <= 2 * 2.0 ** -16 * math.sqrt(2 * n) * (2 * n - 1)
