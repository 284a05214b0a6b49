"""tn_contract_grouped_static: the grouped contraction for callers that must
not allocate device memory (its work list lives in a fixed array inside
libtn.so). Called through the C ABI with ctypes, twice in a row, and checked
against the allocating entry point (tn_group_plan_*) on the same specs and
against the FP64 oracle.

This file is named to be collected last, so a run that stops at the first
failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1905_01330_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# normwise tolerance against || |A||B| ||_F, as in the parity tests
ABS_TOL = {"fp32": 2.0 ** -20, "bf16": 2.0 ** -8, "bf16x3": 2.0 ** -16}
UNSUPPORTED = 3


@pytest.fixture(scope="module")
def tn():
    from paper_1905_01330_gb300 import build, tn as tnmod
    build.build()
    tnmod.load()
    return tnmod


def static_fn(tn):
    lib = ctypes.CDLL(tn.library_path())
    fn = lib.tn_contract_grouped_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(tn.TnContractSpec), ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    return fn


def make_specs(tn):
    st = synth.Stream(321)
    specs = []
    for i in range(24):
        sha, la, shb, lb = synth.contraction_spec(st, dims=(3, 8, 16, 24), cap=1 << 15)
        A = torch.from_numpy(synth.normal_f32(700 + i, sha)).cuda()
        B = torch.from_numpy(synth.normal_f32(800 + i, shb)).cuda()
        specs.append((A, list(la), B, list(lb)))
    # one long shared index, so split-K (results zeroed first) is exercised
    A = torch.from_numpy(synth.normal_f32(901, (16, 4096))).cuda()
    B = torch.from_numpy(synth.normal_f32(902, (4096, 24))).cuda()
    specs.append((A, [1], B, [0]))
    # an empty shared leg: the result is zero (written by the zeroing kernel)
    specs.append((torch.empty(5, 0).cuda(), [1], torch.empty(0, 7).cuda(), [0]))
    return specs


def spec_array(tn, specs, outs):
    arr = (tn.TnContractSpec * len(specs))()
    for i, ((A, la, B, lb), C) in enumerate(zip(specs, outs)):
        arr[i].A = tn.tensor_desc(A)
        arr[i].B = tn.tensor_desc(B)
        arr[i].C = tn.tensor_desc(C)
        arr[i].nshared = len(la)
        for j in range(len(la)):
            arr[i].legsA[j] = la[j]
            arr[i].legsB[j] = lb[j]
    return arr


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x3"])
def test_static_grouped_matches_allocating_path_and_oracle(tn, prec):
    fn = static_fn(tn)
    specs = make_specs(tn)
    ref = [torch.empty(tn.result_shape(A, la, B, lb), device="cuda") for A, la, B, lb in specs]
    plan = tn.GroupPlan([(A, la, B, lb, C) for (A, la, B, lb), C in zip(specs, ref)], prec=prec)
    plan.run()
    torch.cuda.synchronize()
    exact = []
    for A, la, B, lb in specs:
        a, b = A.cpu().numpy(), B.cpu().numpy()
        exact.append((oracle.tensordot(a, la, b, lb), np.linalg.norm(oracle.tensordot(np.abs(a), la, np.abs(b), lb))))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        outs = [torch.full(r.shape, float("nan"), device="cuda") for r in ref]
        arr = spec_array(tn, specs, outs)
        assert fn(arr, len(specs), tn.PREC[prec], stream) == 0
        torch.cuda.synchronize()
        assert tn.sync_status() == 0
        for i, (got, want, (c_ref, absnorm)) in enumerate(zip(outs, ref, exact)):
            g = got.double().cpu().numpy()
            assert np.isfinite(g).all(), (call, i)
            if absnorm == 0.0:
                assert not g.any(), (call, i)  # empty shared index: exactly zero
                continue
            # against the allocating path, and against the FP64 oracle
            err_plan = np.linalg.norm(g - want.double().cpu().numpy()) / absnorm
            err_oracle = np.linalg.norm(g - c_ref) / absnorm
            assert err_plan <= ABS_TOL[prec], (call, i, err_plan)
            assert err_oracle <= ABS_TOL[prec], (call, i, err_oracle)


def test_static_grouped_rejects_too_many_specs(tn):
    fn = static_fn(tn)
    arr = (tn.TnContractSpec * 1)()
    assert fn(arr, 4097, 0, None) == UNSUPPORTED  # nothing launched


def test_static_grouped_rejects_work_list_larger_than_array(tn):
    # 4096 specs (the spec limit) of 8 x 24 output tiles each: 786,432 work
    # units, whose map (3 MiB) and descriptors (1.8 MiB) exceed the 4 MiB
    # array. The specs share one set of tensors; the call must refuse before
    # any copy or launch, so the result keeps its NaN fill.
    fn = static_fn(tn)
    A = torch.ones(1024, 16, device="cuda")
    B = torch.ones(16, 3072, device="cuda")
    C = torch.full((1024, 3072), float("nan"), device="cuda")
    specs = [(A, [1], B, [0])] * 4096
    arr = spec_array(tn, specs, [C] * 4096)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert fn(arr, 4096, tn.PREC["fp32"], stream) == UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.isnan(C).all().item()
    # a request within the limits still runs after the refusal
    specs = [(A, [1], B, [0])]
    C1 = torch.empty(1024, 3072, device="cuda")
    assert fn(spec_array(tn, specs, [C1]), 1, tn.PREC["fp32"], stream) == 0
    torch.cuda.synchronize()
    assert tn.sync_status() == 0
    assert torch.equal(C1, torch.full_like(C1, 16.0))


def test_static_grouped_refuses_a_capturing_stream(tn):
    # The work list is copied from host staging arrays the next call
    # overwrites, so a call on a capturing stream is refused with nothing
    # enqueued; the capture itself stays valid and the stream usable.
    fn = static_fn(tn)
    A = torch.ones(64, 16, device="cuda")
    B = torch.ones(16, 32, device="cuda")
    C = torch.full((64, 32), float("nan"), device="cuda")
    D = torch.zeros(8, device="cuda")
    arr = spec_array(tn, [(A, [1], B, [0])], [C])
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        rc = fn(arr, 1, tn.PREC["fp32"], ctypes.c_void_p(side.cuda_stream))
        D.add_(1.0)
    assert rc == UNSUPPORTED
    g.replay()
    torch.cuda.synchronize()
    assert torch.isnan(C).all().item()
    assert torch.equal(D, torch.ones_like(D))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert fn(arr, 1, tn.PREC["fp32"], stream) == 0
    torch.cuda.synchronize()
    assert tn.sync_status() == 0
    assert torch.equal(C, torch.full_like(C, 16.0))
