"""The C ABI builds, loads without a GPU, and exports every entry point that
include/tn.h declares; host-side marshalling layouts match the header."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        with open(os.path.join(ROOT, "include", hdr)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tn_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_1905_01330_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("tn_contract", "tn_group_plan_create", "tn_group_plan_run", "tn_sync_status"):
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\b(tn_\w+)\b", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    for n in declared_functions():
        assert hasattr(lib, n)
    lib.tn_status_string.restype = ctypes.c_char_p
    assert lib.tn_status_string(2) == b"shape mismatch"


def test_struct_layouts_match_header():
    from paper_1905_01330_gb300 import tn
    assert ctypes.sizeof(tn.TnTensor) == 8 + 4 + 4 + 8 * 8 + 8 * 8
    assert ctypes.sizeof(tn.TnContractSpec) == 3 * ctypes.sizeof(tn.TnTensor) + 4 + 32 + 32 + 4  # tail pad


def test_validation_errors_without_gpu(libpath):
    # argument checks run on the host before any CUDA call
    from paper_1905_01330_gb300 import tn
    lib = ctypes.CDLL(libpath)
    lib.tn_contract.restype = ctypes.c_int
    a, b, c = tn.TnTensor(), tn.TnTensor(), tn.TnTensor()
    for t, shape in ((a, (3, 4)), (b, (5, 6)), (c, (3, 6))):
        t.data = 0x1000
        t.rank = 2
        for i, n in enumerate(shape):
            t.shape[i] = n
    la = (ctypes.c_int * 1)(1)
    lb = (ctypes.c_int * 1)(0)
    assert lib.tn_contract(ctypes.byref(a), la, ctypes.byref(b), lb, 1, ctypes.byref(c), 0, None) == 2
    la2 = (ctypes.c_int * 1)(7)
    assert lib.tn_contract(ctypes.byref(a), la2, ctypes.byref(b), lb, 1, ctypes.byref(c), 0, None) == 1
    assert lib.tn_contract(None, la, ctypes.byref(b), lb, 1, ctypes.byref(c), 0, None) == 1
    assert lib.tn_contract(ctypes.byref(a), la, ctypes.byref(b), lb, 1, ctypes.byref(c), 9, None) == 1


def test_group_plan_launches_without_gpu(libpath):
    """Planning runs on the host: a BF16 plan sends a contraction whose
    narrower operand has at most 64 rows to the fused GEMM (its wider
    operand is never packed) and the rest to pack + GEMM; a BF16X3 plan packs
    everything. Algorithmic bytes per launch follow from the shapes."""
    from paper_1905_01330_gb300 import tn
    lib = ctypes.CDLL(libpath)
    for n, (res, args) in tn._signatures().items():
        getattr(lib, n).restype = res
        getattr(lib, n).argtypes = args

    def desc(shape, addr):
        t = tn.TnTensor()
        t.data, t.rank = addr, len(shape)
        for i, n in enumerate(shape):
            t.shape[i] = n
        return t

    specs = [((4096, 64), [1], (64, 32), [0], (4096, 32)),      # thin: P = A
             ((16, 96), [1], (96, 3000), [0], (16, 3000)),      # thin, swapped: P = B
             ((512, 256), [1], (256, 384), [0], (512, 384))]    # packed
    arr = (tn.TnContractSpec * len(specs))()
    for i, (sa, la, sb, lb, sc) in enumerate(specs):
        arr[i].A, arr[i].B, arr[i].C = desc(sa, 0x10000 * (3 * i + 1)), desc(sb, 0x10000 * (3 * i + 2)), \
            desc(sc, 0x10000 * (3 * i + 3))
        arr[i].nshared = 1
        arr[i].legsA[0], arr[i].legsB[0] = la[0], lb[0]

    def launches(prec):
        h = ctypes.c_void_p()
        assert lib.tn_group_plan_create(arr, len(specs), tn.PREC[prec], ctypes.byref(h)) == 0
        out = {lib.tn_group_plan_launch_name(h, i).decode(): lib.tn_group_plan_launch_bytes(h, i)
               for i in range(lib.tn_group_plan_launches(h))}
        assert lib.tn_group_plan_launch_bytes(h, lib.tn_group_plan_launches(h)) == -1.0
        lib.tn_group_plan_destroy(h)
        return out

    got = launches("bf16")
    assert got == {
        "pack": 6.0 * (64 * 32 + 16 * 96 + 512 * 256 + 256 * 384),           # only Q of the fused two
        "gemm": 2.0 * (512 * 256 + 256 * 384) + 4.0 * 512 * 384,
        "gemm_fused": 4.0 * (4096 * 64 + 3000 * 96) + 2.0 * (32 * 64 + 16 * 96) + 4.0 * (4096 * 32 + 16 * 3000),
    }
    got = launches("bf16x3")
    ops = 4096 * 64 + 64 * 32 + 16 * 96 + 96 * 3000 + 512 * 256 + 256 * 384
    assert got == {"pack": 8.0 * ops, "gemm": 4.0 * ops + 4.0 * (4096 * 32 + 16 * 3000 + 512 * 384)}


def _bound(libpath):
    from paper_1905_01330_gb300 import tn
    lib = ctypes.CDLL(libpath)
    for n, (res, args) in tn._signatures().items():
        getattr(lib, n).restype = res
        getattr(lib, n).argtypes = args
    return lib, tn


def test_split_truncation_rule_matches_the_oracle(libpath):
    """The host truncation rule of tn_split_node (Appendix A: drop the smallest
    singular values while their sum stays within max_truncation_err, keep at
    most max_singular_values, at least one) agrees with the oracle's on
    hand-made spectra and on random ones, limits placed between partial sums."""
    import numpy as np
    import oracle
    lib, _ = _bound(libpath)

    def k_lib(s, max_sv, max_err):
        arr = (ctypes.c_float * max(len(s), 1))(*[float(v) for v in s])
        return lib.tn_split_truncation(arr, len(s), max_sv or 0, -1.0 if max_err is None else max_err)

    cases = [([5, 3, 0.06, 0.03, 0.02], None, 0.1), ([5, 3, 0.06, 0.03, 0.02], 2, None),
             ([5, 3, 0.06, 0.03, 0.02], 4, 0.1), ([2, 1, 0, 0], None, 0.0), ([0.05, 0.01], None, 1.0),
             ([1.0], 1, 0.5), ([], None, 1.0)]
    rng = np.random.default_rng(7)
    for _ in range(200):
        s = np.sort(rng.exponential(size=int(rng.integers(1, 40))).astype(np.float32))[::-1]
        tail = np.cumsum(s[::-1].astype(np.float64))
        err = float(tail[int(rng.integers(0, len(s)))] * rng.uniform(0.5, 1.5))
        cases.append((list(s), int(rng.integers(0, len(s) + 2)) or None, err))
    for s, max_sv, max_err in cases:
        s32 = [float(np.float32(v)) for v in s]
        assert k_lib(s32, max_sv, max_err) == oracle.truncation_count(s32, max_sv, max_err), (s, max_sv, max_err)


def test_split_node_validation_without_gpu(libpath):
    lib, tn = _bound(libpath)
    a = tn.TnTensor()
    a.data, a.rank = 0x1000, 3
    for i, n in enumerate((2, 3, 4)):
        a.shape[i] = n
    ip = lambda *v: (ctypes.c_int * max(len(v), 1))(*v)  # noqa: E731
    assert lib.tn_split_node_workspace_bytes(ctypes.byref(a), ip(0, 1), 2, ip(2), 1) > 0
    for left, right in (((0,), (1,)), ((0, 1), (1, 2)), ((0, 3), (1, 2)), ((0, 0), (1, 2))):
        assert lib.tn_split_node_workspace_bytes(ctypes.byref(a), ip(*left), len(left), ip(*right), len(right)) == 0
    kept = ctypes.c_int64(-1)
    rc = lib.tn_split_node(ctypes.byref(a), ip(0, 1), 2, ip(1, 2), 2, 0, -1.0, 1, None, None, None, None,
                           ctypes.byref(kept), None, None, 0, None)
    assert rc == 1
    # valid legs but no outputs / no workspace: refused before any CUDA call
    rc = lib.tn_split_node(ctypes.byref(a), ip(0, 1), 2, ip(2), 1, 0, -1.0, 1, None, None, None, None,
                           ctypes.byref(kept), None, None, 0, None)
    assert rc == 1
    rc = lib.tn_split_node(ctypes.byref(a), ip(0, 1), 2, ip(2), 1, 0, -1.0, 1, 0x2000, None, 0x3000, None,
                           ctypes.byref(kept), None, None, 0, None)
    assert rc == 6


def test_ncon_planner_without_gpu(libpath):
    """tn_ncon_plan (host): the paper's example is one contraction of a's leg 1
    with b's leg 0; a trace step; unconnected pieces joined by outer products;
    contract_between semantics (all shared edges in one step); a custom
    contraction and output order; invalid labels refused."""
    lib, tn = _bound(libpath)
    steps, perm = tn.ncon_plan([(2, 2), (2, 2)], [(-1, 0), (0, -2)], lib=lib)
    assert steps == [(0, 1, [1], [0], [2, 2])] and perm == [0, 1]
    steps, perm = tn.ncon_plan([(3, 4, 3)], [(0, -1, 0)], lib=lib)
    assert steps == [(0, -1, [0], [2], [4])] and perm == [0]
    steps, perm = tn.ncon_plan([(2, 3), (4, 5), (6,)], [(-2, -1), (-3, -4), (-5,)], lib=lib)
    assert steps == [(0, 1, [], [], [2, 3, 4, 5]), (3, 2, [], [], [2, 3, 4, 5, 6])] and perm == [1, 0, 2, 3, 4]
    steps, perm = tn.ncon_plan([(2, 3, 4), (4, 3, 5)], [(-1, 0, 1), (1, 0, -2)], lib=lib)
    assert steps == [(0, 1, [1, 2], [1, 0], [2, 5])] and perm == [0, 1]
    steps, perm = tn.ncon_plan([(2, 3, 4), (4, 3, 5), (5, 6)], [(-1, 0, 1), (1, 0, 2), (2, -2)],
                               con_order=[2, 0, 1], out_order=[-2, -1], lib=lib)
    assert steps == [(1, 2, [2], [0], [4, 3, 6]), (0, 3, [1, 2], [1, 0], [2, 6])] and perm == [1, 0]
    bad = [([(2, 2), (2, 2)], [(0, -1), (1, -2)], None, None, 1),      # edges seen once
           ([(2, 2), (3, 2)], [(0, -1), (0, -2)], None, None, 2),      # edge dims differ
           ([(2, 2), (2, 2)], [(0, -1), (0, -3)], None, None, 1),      # dangling -1, -3
           ([(2, 2), (2, 2)], [(-1, 0), (0, -2)], [0, 0], None, 1),    # con_order repeats
           ([(2, 2), (2, 2)], [(-1, 0), (0, -2)], None, [-1], 1)]      # out_order short
    for shapes, net, co, oo, code in bad:
        with pytest.raises(tn.TnError) as e:
            tn.ncon_plan(shapes, net, co, oo, lib=lib)
        assert e.value.code == code


@pytest.mark.parametrize("seed", range(10))
def test_ncon_planner_steps_evaluate_the_network(libpath, seed):
    """The host planner's steps, executed with the FP64 oracle's tensordot and
    trace (CPU), give the oracle's ncon of the same random network (traces,
    multi-edges, unconnected pieces), for the default and a shuffled order."""
    import sys
    import numpy as np
    import oracle
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from ncon_nets import random_network
    lib, tn = _bound(libpath)
    shapes, net = random_network(600 + seed)
    rng = np.random.default_rng(seed)
    ts = [rng.standard_normal(sh) for sh in shapes]
    edges = sorted({x for labels in net for x in labels if x >= 0})
    for order in (None, list(rng.permutation(edges))):
        steps, perm = tn.ncon_plan(shapes, net, con_order=order, lib=lib)
        ops = list(ts)
        for a, b, la, lb, shape in steps:
            if b < 0:
                r = oracle.trace(ops[a], la[0], lb[0])
            else:
                r = oracle.tensordot(ops[a], la, ops[b], lb)
            assert list(np.shape(r)) == shape
            ops.append(r)
        got = np.transpose(ops[-1], perm) if perm else ops[-1]
        ref = oracle.ncon(ts, net, con_order=order)
        assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_separate_classifier_validation_without_gpu(libpath):
    """tn_mps_classify_separate*: counts, lengths and pointers are checked on the
    host before any CUDA call."""
    lib, tn = _bound(libpath)
    n, chi = 6, 4
    bonds = [1] + [chi] * (n - 1) + [1]

    def chain(nsites):
        b = bonds[:nsites] + [1]
        bond_arr = (ctypes.c_int64 * (nsites + 1))(*b)
        ptr_arr = (ctypes.c_void_p * nsites)(*[0x1000 * (i + 1) for i in range(nsites)])
        ch = tn.TnChain()
        ch.n, ch.d = nsites, 2
        ch.bond = ctypes.cast(bond_arr, ctypes.POINTER(ctypes.c_int64))
        ch.cores = ctypes.cast(ptr_arr, ctypes.POINTER(ctypes.c_void_p))
        return ch, (bond_arr, ptr_arr)
    (c0, k0), (c1, k1), (c2, k2) = chain(n), chain(n), chain(n - 1)
    two = (tn.TnChain * 2)(c0, c1)
    mixed = (tn.TnChain * 2)(c0, c2)
    assert lib.tn_mps_classify_separate_workspace_bytes(two, 2, 8, 1) > 0
    assert lib.tn_mps_classify_separate_workspace_bytes(two, 0, 8, 1) == 0
    assert lib.tn_mps_classify_separate_workspace_bytes(two, 65, 8, 1) == 0
    assert lib.tn_mps_classify_separate_workspace_bytes(two, 2, -1, 1) == 0
    px = ctypes.c_void_p(0x5000)
    ft, lam = ctypes.c_void_p(0x6000), ctypes.c_void_p(0x7000)
    # MPS of different lengths
    assert lib.tn_mps_classify_separate(mixed, 2, px, 8, 0, 0, ft, lam, None, 0, None) == 2
    # missing outputs
    assert lib.tn_mps_classify_separate(two, 2, px, 8, 0, 0, None, lam, None, 0, None) == 1
    # no workspace
    assert lib.tn_mps_classify_separate(two, 2, px, 8, 0, 0, ft, lam, None, 0, None) == 6
    # backward: checkpoints every >= 1 site required
    table = (ctypes.c_void_p * (2 * n))(*[0x9000] * (2 * n))
    assert lib.tn_mps_classify_separate_backward(two, 2, px, 8, 0, 0, ft, table, None, 0, None) == 1


def test_staged_plan_validation_without_gpu(libpath):
    """tn_staged_plan_create checks, on the host before any CUDA call, that
    every tensor lies in its buffer and that the buffers are laid out in spec
    order; the failure-path check wants a 256-byte aligned counter."""
    lib, tn = _bound(libpath)

    def desc(shape, addr):
        t = tn.TnTensor()
        t.data, t.rank = addr, len(shape)
        for i, n in enumerate(shape):
            t.shape[i] = n
        return t
    base_in, base_out = 0x100000, 0x900000
    # two 8 x 8 by 8 x 8 specs: operands at base_in + 0, 256, 512, 768 bytes
    def specs(order):
        arr = (tn.TnContractSpec * 2)()
        for i, k in enumerate(order):
            arr[i].A = desc((8, 8), base_in + 512 * k)
            arr[i].B = desc((8, 8), base_in + 512 * k + 256)
            arr[i].C = desc((8, 8), base_out + 256 * k)
            arr[i].nshared = 1
            arr[i].legsA[0], arr[i].legsB[0] = 1, 0
        return arr
    h = ctypes.c_void_p()
    vin, vout = ctypes.c_void_p(base_in), ctypes.c_void_p(base_out)
    assert lib.tn_staged_plan_create(specs([0, 1]), 2, 0, vin, 1024, vout, 512, 0, ctypes.byref(h)) == 1  # chunks
    assert lib.tn_staged_plan_create(specs([0, 1]), 2, 0, vin, 1000, vout, 512, 2, ctypes.byref(h)) == 1  # outside
    assert lib.tn_staged_plan_create(specs([0, 1]), 2, 0, vin, 1024, vout, 500, 2, ctypes.byref(h)) == 1  # outside
    assert lib.tn_staged_plan_create(specs([1, 0]), 2, 0, vin, 1024, vout, 512, 2, ctypes.byref(h)) == 1  # order
    assert not h.value
    assert lib.tn_check_grid_barrier_timeout(10_000_000, ctypes.c_void_p(0x1002), None) == 1
    assert lib.tn_check_grid_barrier_timeout(10_000_000, None, None) == 1


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x3"])
def test_workload_plan_counts_the_algorithmic_work(libpath, prec):
    """The bench's headline divides the plan's flops and bytes by the step
    time: for the 2048-spec workload they are sum 2 M N K (about 2.0 TFLOP)
    and sum 4 (|A| + |B| + |C|) bytes (about 31.9 GB), counted here from the
    spec shapes alone, in every precision (planning runs on the host)."""
    from paper_1905_01330_gb300 import synth
    lib, tn = _bound(libpath)
    specs = synth.contraction_specs(2048, seed=2)
    arr = (tn.TnContractSpec * len(specs))()
    flops = nbytes = 0.0
    addr = 1 << 20
    for i, (sha, la, shb, lb) in enumerate(specs):
        M, N, K = synth.spec_sizes((sha, la, shb, lb))
        flops += 2.0 * M * N * K
        nbytes += 4.0 * (M * K + K * N + M * N)
        shc = [n for j, n in enumerate(sha) if j not in la] + [n for j, n in enumerate(shb) if j not in lb]
        for t, sh in ((arr[i].A, sha), (arr[i].B, shb), (arr[i].C, shc)):
            t.data, t.rank = addr, len(sh)
            for j, n in enumerate(sh):
                t.shape[j] = n
            addr += 256 * ((4 * int(np.prod(sh)) + 255) // 256)
        arr[i].nshared = len(la)
        for j in range(len(la)):
            arr[i].legsA[j], arr[i].legsB[j] = la[j], lb[j]
    h = ctypes.c_void_p()
    assert lib.tn_group_plan_create(arr, len(specs), tn.PREC[prec], ctypes.byref(h)) == 0
    try:
        assert lib.tn_group_plan_flops(h) == pytest.approx(flops, rel=1e-12)
        assert lib.tn_group_plan_bytes(h) == pytest.approx(nbytes, rel=1e-12)
        assert 1.9e12 < flops < 2.1e12 and 31e9 < nbytes < 33e9
    finally:
        lib.tn_group_plan_destroy(h)
