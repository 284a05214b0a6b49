"""tn_contract_grouped_static: the grouped contraction for callers that must
not allocate device memory (its work list lives in a fixed array inside
libtn.so). Called through the C ABI with ctypes, twice in a row, and checked
against the allocating entry point (tn_group_plan_*) on the same specs.

This file is named to be collected last, so a run that stops at the first
failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from paper_1905_01330_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# normwise tolerance against || |A||B| ||_F, as in the parity tests
ABS_TOL = {"fp32": 2.0 ** -20, "bf16": 2.0 ** -8, "bf16x3": 2.0 ** -16}


@pytest.fixture(scope="module")
def tn():
    from paper_1905_01330_gb300 import build, tn as tnmod
    build.build()
    tnmod.load()
    return tnmod


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


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_static_grouped_matches_allocating_path(tn, prec):
    lib = ctypes.CDLL(tn.library_path())
    fn = lib.tn_contract_grouped_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(tn.TnContractSpec), ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    specs = make_specs(tn)
    ref = [torch.empty(tn.result_shape(A, la, B, lb), device="cuda") for A, la, B, lb in specs]
    plan = tn.GroupPlan([(A, la, B, lb, C) for (A, la, B, lb), C in zip(specs, ref)], prec=prec)
    plan.run()
    torch.cuda.synchronize()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        outs = [torch.full(r.shape, float("nan"), device="cuda") for r in ref]
        arr = spec_array(tn, specs, outs)
        assert fn(arr, len(specs), tn.PREC[prec], stream) == 0
        torch.cuda.synchronize()
        assert tn.sync_status() == 0
        for (A, la, B, lb), got, want in zip(specs, outs, ref):
            absref = tn.contract(A.abs(), la, B.abs(), lb, prec="fp32")
            err = (got.double() - want.double()).norm().item() / max(absref.double().norm().item(), 1e-30)
            assert err <= ABS_TOL[prec], (call, err)


def test_static_grouped_rejects_too_many_specs(tn):
    lib = ctypes.CDLL(tn.library_path())
    fn = lib.tn_contract_grouped_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(tn.TnContractSpec), ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    arr = (tn.TnContractSpec * 1)()
    assert fn(arr, 4097, 0, None) == 3  # TN_ERR_UNSUPPORTED, nothing launched
