"""Failure detection without a GPU fault: a bounded device wait that nothing
satisfies gives up, reports TN_ERR_TIMEOUT through the status word, and the
context stays usable for the next contraction."""
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
