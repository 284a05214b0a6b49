"""GPU parity of the grouped two-launch path (pack + tcgen05 GEMM on packed
bf16 blocks) against the FP64 oracle, with the error model and bounds of
test_contract_gpu.check. Grouped BF16 / BF16X3 plans take this path; the
shapes below exercise what is particular to it: the operand with fewer rows
on the MMA's column side (swapped roles, column stores), narrow column tiles
(16..112), single-row operands, shared-index tails that are not a multiple of
64, split k ranges with atomically accumulated results, the outer product
(K = 1), gathers from permuted and strided views, and long k with the
BF16X3 accumulator promotion."""
import numpy as np
import pytest

from paper_1905_01330_gb300 import synth
from test_contract_gpu import check, rand

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tn():
    from paper_1905_01330_gb300 import build, tn as tnmod
    build.build()
    tnmod.load()
    return tnmod


def run_group(tn, cases, prec, seed0):
    """cases: (A, la, B, lb) as host arrays, or (At, la, Bt, lb, A_host, B_host)
    for device views; one plan over all, every result checked."""
    specs, host = [], []
    for i, c in enumerate(cases):
        if len(c) == 4:
            A, la, B, lb = c
            At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        else:
            At, la, Bt, lb, A, B = c
        C = torch.full(tn.result_shape(At, la, Bt, lb), float("nan"), device="cuda")
        specs.append((At, list(la), Bt, list(lb), C))
        host.append((A, la, B, lb))
    plan = tn.GroupPlan(specs, prec=prec)
    assert plan.launches >= 2
    plan.run()
    torch.cuda.synchronize()
    assert tn.sync_status() == 0
    for (A, la, B, lb), sp in zip(host, specs):
        check(sp[4], A, la, B, lb, prec)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_packed_shapes(tn, prec):
    cases = [
        (rand(1, (4096,)), [0], rand(2, (4096, 200)), [0]),      # M = 1, swapped, split k
        (rand(3, (300, 4096)), [1], rand(4, (4096,)), [0]),      # N = 1
        (rand(5, (100, 72)), [1], rand(6, (72, 300)), [0]),      # swapped, K tail 8, 112-wide columns
        (rand(7, (300, 5000)), [1], rand(8, (20, 5000)), [1]),   # 32-wide columns, 3 k ranges
        (rand(9, (50, 3)), [], rand(10, (7, 130)), []),          # outer product (K = 1)
        (rand(11, (130, 20000)), [1], rand(12, (20000, 130)), [0]),  # long k: promotion, 10 k ranges
        (rand(13, (256, 256)), [1], rand(14, (256, 384)), [0]),  # whole tiles only
        (rand(15, (8, 9, 10)), [1], rand(16, (9, 11)), [0]),     # ragged everything
    ]
    run_group(tn, cases, prec, 0)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_packed_permuted_and_strided(tn, prec):
    A = rand(21, (16, 24, 8, 5))
    B = rand(22, (8, 7, 24, 16))
    At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Ap = At.permute(3, 1, 0, 2)                     # non-contiguous view, unit stride on a free leg
    Anp = np.ascontiguousarray(A.transpose(3, 1, 0, 2))
    Bs = Bt[:, ::2]                                 # strided slice: no unit-stride leg run of 4
    Bsnp = np.ascontiguousarray(B[:, ::2])
    cases = [
        (A, [2, 0, 1], B, [0, 3, 2]),
        (Ap, [1, 2], Bt, [2, 3], Anp, B),
        (At, [2], Bs, [0], A, Bsnp),
        (rand(23, (48, 64, 32)), [0, 2], rand(24, (32, 9, 48)), [2, 0]),  # k legs in reverse order
        (rand(25, (64, 40)), [0], rand(26, (64, 40)), [0]),               # both operands m/n-fast
    ]
    run_group(tn, cases, prec, 0)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
@pytest.mark.parametrize("seed", range(6))
def test_packed_random_specs(tn, prec, seed):
    st = synth.Stream(4000 + seed)
    cases = []
    for i in range(12):
        sha, la, shb, lb = synth.contraction_spec(st, dims=(3, 8, 13, 24, 48, 64), cap=1 << 17)
        cases.append((rand(7000 + 100 * seed + 2 * i, sha), la, rand(7001 + 100 * seed + 2 * i, shb), lb))
    run_group(tn, cases, prec, seed)


def mixed_cases():
    return [
        (rand(31, (4096,)), [0], rand(32, (4096, 200)), [0]),      # thin
        (rand(33, (300, 5000)), [1], rand(34, (20, 5000)), [1]),   # thin, split k
        (rand(35, (100, 72)), [1], rand(36, (72, 300)), [0]),      # thin, swapped
        (rand(37, (640, 4608)), [1], rand(38, (4608, 520)), [0]),  # 20 tiles, 72 slabs
        (rand(39, (256, 96)), [1], rand(40, (96, 384)), [0]),      # short k
        (rand(43, (130, 2, 64)), [1, 2], rand(44, (2, 64, 264)), [0, 1]),  # short k, ragged columns
        (rand(41, (8, 9, 10)), [1], rand(42, (9, 11)), [0]),       # ragged
    ]


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_every_schedule_keeps_parity(tn, prec):
    cases = mixed_cases()
    specs = []
    for A, la, B, lb in cases:
        At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        specs.append((At, la, Bt, lb, torch.empty(tn.result_shape(At, la, Bt, lb), device="cuda")))
    plan = tn.GroupPlan(specs, prec=prec)
    schedules = [(128, 1, 0), (64, 1, 1), (128, 0, 1), (64, 0, 0)]
    if prec == "bf16":
        # 256-wide tiles: Q from two 128-row blocks, a partial second block
        # (520 = 2 x 256 + 8, 264 = 256 + 8 rows), a single block (384 = 256 + 128)
        schedules += [(256, 1, 0), (256, 0, 1)]
    else:
        with pytest.raises(tn.TnError):
            plan.set_schedule("long_k", 256, True, False)
    for width, long_k, store16 in schedules:
        for cls in plan.SCHEDULE_CLASSES:
            plan.set_schedule(cls, width, long_k, store16)
        assert plan.schedule() == {c: (width, long_k, store16) for c in plan.SCHEDULE_CLASSES}
        for sp in specs:
            sp[4].fill_(float("nan"))
        plan.run()
        torch.cuda.synchronize()
        assert tn.sync_status() == 0
        for (A, la, B, lb), sp in zip(cases, specs):
            check(sp[4], A, la, B, lb, prec)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
def test_autotune_picks_a_schedule_and_caches_it(tn, prec):
    cases = mixed_cases()
    specs = []
    for A, la, B, lb in cases:
        At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        specs.append((At, la, Bt, lb, torch.empty(tn.result_shape(At, la, Bt, lb), device="cuda")))
    plan = tn.GroupPlan(specs, prec=prec)
    sched = plan.autotune()
    assert tn.sync_status() == 0
    widths = (64, 128, 256) if prec == "bf16" else (64, 128)   # 256-wide tiles are BF16 only
    assert all(w in widths and lk in (0, 1) and s16 in (0, 1) for w, lk, s16 in sched.values())
    for sp in specs:
        sp[4].fill_(float("nan"))
    plan.run()
    torch.cuda.synchronize()
    for (A, la, B, lb), sp in zip(cases, specs):
        check(sp[4], A, la, B, lb, prec)
    # a new plan over the same shapes starts from the cached choice
    again = tn.GroupPlan(specs, prec=prec)
    assert again.schedule() == sched


def test_fused_gemm_access_patterns(tn):
    """BF16 contractions whose narrower operand has at most 64 rows take a
    fused GEMM (the wider operand rounded to bf16 inside it, never packed):
    the TMA one when the wider operand's layout allows whole boxes, else the
    one whose converters copy through offset tables. Cases cover the
    converters' paths: the wider operand unit-stride along k (16-byte
    copies), along its rows (16-byte copies of 4 rows), with no unit stride,
    at an address that is not 16-byte aligned (4-byte fallback), on either
    side (A, or B with the roles swapped), row and k tails, K < 8, many units
    per CTA, and split k ranges; the aligned ones take the TMA GEMM."""
    base = torch.from_numpy(rand(60, (1 + 700 * 96,))).cuda()
    Au = base[1:].view(700, 96)                          # 4-byte aligned only
    Aunp = Au.cpu().numpy()
    Bfull = torch.from_numpy(rand(61, (40, 600))).cuda()
    Bx = Bfull[:, ::2]                                   # (40, 300), strides (600, 2): no unit stride
    cases = [
        (rand(50, (1000, 192)), [1], rand(51, (192, 40)), [0]),         # k unit stride, P = A
        (rand(66, (2000, 100)), [1], rand(67, (100, 30)), [0]),         # ... no 16-byte TMA box (50 wide)
        (rand(52, (72, 900)), [0], rand(53, (72, 24)), [0]),            # rows unit stride (k outer)
        (Au, [1], rand(54, (96, 33)), [0], Aunp, None),                  # misaligned rows: 4-byte copies
        (rand(55, (24, 77)), [1], rand(56, (3000, 77)), [1]),           # swapped: P = B, k tail 13
        (rand(57, (5, 4000)), [0], rand(58, (5, 16)), [0]),             # K = 5
        (rand(59, (20000, 64)), [1], rand(62, (64, 60)), [0]),          # 157 units: CTAs run several
        (rand(63, (300, 6000)), [1], rand(64, (6000, 50)), [0]),        # 3 tiles: split k ranges
        (rand(65, (40, 8)), [0], Bx, [0], None, None),                  # swapped, P without unit stride
    ]
    specs, host = [], []
    for c in cases:
        A, la, B, lb = c[:4]
        At = A if torch.is_tensor(A) else torch.from_numpy(A).cuda()
        Btt = B if torch.is_tensor(B) else torch.from_numpy(B).cuda()
        Ah = c[4] if len(c) > 4 and c[4] is not None else (At.cpu().numpy() if torch.is_tensor(A) else A)
        Bh = c[5] if len(c) > 5 and c[5] is not None else (Btt.cpu().numpy() if torch.is_tensor(B) else B)
        specs.append((At, list(la), Btt, list(lb), torch.empty(tn.result_shape(At, la, Btt, lb), device="cuda")))
        host.append((np.ascontiguousarray(Ah), la, np.ascontiguousarray(Bh), lb))
    plan = tn.GroupPlan(specs, prec="bf16")
    assert "gemm_fused" in plan.launch_names() and "gemm_tma" in plan.launch_names()
    for rep in range(2):   # twice: the second run reuses stale shared memory and staging
        for sp in specs:
            sp[4].fill_(float("nan"))
        plan.run()
        torch.cuda.synchronize()
        assert tn.sync_status() == 0
        for (A, la, B, lb), sp in zip(host, specs):
            check(sp[4], A, la, B, lb, "bf16")


def test_staged_plan_from_pinned_host(tn):
    """StagedGroupPlan: operands in one device buffer and results in another
    (spec order), fed from and drained to pinned host buffers chunk by chunk
    on three streams; every result checked after two runs (the second with
    new operand values in the host buffer)."""
    st = synth.Stream(77)
    # the two large specs first: chunks of equal weight are then [big], [thin], [20 small]
    shapes = [((640, 4608), [1], (4608, 520), [0]), ((4096,), [0], (4096, 200), [0])]
    shapes += [synth.contraction_spec(st, dims=(3, 8, 13, 24, 48, 64), cap=1 << 17) for _ in range(20)]

    def layout(sizes):
        offs, n = [], 0
        for k in sizes:
            offs.append(n)
            n += (k + 63) // 64 * 64
        return offs, n
    in_sizes = [int(np.prod(sh)) for sa, _, sb, _ in shapes for sh in (sa, sb)]
    outs = [tuple(sa[p] for p in range(len(sa)) if p not in la) + tuple(sb[p] for p in range(len(sb)) if p not in lb)
            for sa, la, sb, lb in shapes]
    in_offs, n_in = layout(in_sizes)
    out_offs, n_out = layout([int(np.prod(o)) for o in outs])
    dev_in, dev_out = torch.empty(n_in, device="cuda"), torch.empty(n_out, device="cuda")
    specs = []
    for i, (sa, la, sb, lb) in enumerate(shapes):
        A = dev_in[in_offs[2 * i]:in_offs[2 * i] + in_sizes[2 * i]].view(sa)
        B = dev_in[in_offs[2 * i + 1]:in_offs[2 * i + 1] + in_sizes[2 * i + 1]].view(sb)
        C = dev_out[out_offs[i]:out_offs[i] + int(np.prod(outs[i]))].view(outs[i])
        specs.append((A, list(la), B, list(lb), C))
    staged = tn.StagedGroupPlan(specs, dev_in, dev_out, chunks=3, prec="bf16")
    assert staged.chunks == 3
    host_in = torch.empty(n_in, dtype=torch.float32, pin_memory=True)
    host_out = torch.empty(n_out, dtype=torch.float32, pin_memory=True)
    graph = None
    for seed in (1, 2, 3):
        host_in.copy_(torch.from_numpy(np.random.default_rng(seed).standard_normal(n_in).astype(np.float32)))
        host_out.fill_(float("nan"))
        if seed < 3:
            staged.run(host_in, host_out)
        else:
            # the run only launches and copies: it replays from a CUDA graph
            # (its library streams fork from and join the capturing stream)
            graph = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            torch.cuda.synchronize()
            with torch.cuda.graph(graph, stream=side):
                staged.run(host_in, host_out, stream=side)
            host_out.fill_(float("nan"))
            graph.replay()
        torch.cuda.synchronize()
        assert tn.sync_status() == 0
        hi = host_in.numpy()
        for i, (sa, la, sb, lb) in enumerate(shapes):
            A = hi[in_offs[2 * i]:in_offs[2 * i] + in_sizes[2 * i]].reshape(sa)
            B = hi[in_offs[2 * i + 1]:in_offs[2 * i + 1] + in_sizes[2 * i + 1]].reshape(sb)
            C = host_out[out_offs[i]:out_offs[i] + int(np.prod(outs[i]))].view(outs[i])
            check(C, A, la, B, lb, "bf16")


def test_tma_gemm_box_layouts(tn):
    """The fused TMA GEMM: each tile of the wider operand P is one box of its
    tensor map, the box's dimensions P's legs (whole legs from the fastest,
    then a divisor of the next), staged row-major along k (P unit-stride
    along its last shared leg) or along the rows (unit stride on its last
    free leg), the map's strides in an order that is not the memory order
    when free and shared legs interleave. Cases: boxes of 125, 100 and 96
    rows (tiles of fewer than 128 rows, one odd), 36-, 40- and 48-wide slabs (Q packed
    in slabs of that width), boxes spanning two and three legs, a rank-5
    operand over all five dimensions of the map, P = B, a single-row Q,
    split k ranges with atomically accumulated results, and many units per
    CTA; P with few rows and a long k, whose boxes each cover several slabs
    (the staged tile holds them as k-blocks of ceil8(rows) rows, Q's slot
    their consecutive packed blocks). All in one plan, which then has only
    the TMA GEMM; run twice over NaN-filled results (the second run reuses
    stale staging)."""
    cases = [
        (rand(70, (1000, 192)), [1], rand(71, (192, 40)), [0]),          # 125-row boxes, k 3 x 64
        (rand(72, (72, 900)), [0], rand(73, (72, 24)), [0]),             # rows unit stride: 100 x 36 boxes
        (rand(74, (48, 24, 32)), [2, 0], rand(75, (32, 8, 48)), [0, 2]), # k box over two legs, strides out of order
        (rand(76, (24, 48, 40)), [2], rand(77, (40, 16)), [0]),          # row box: 48 x 2 of (24, 48)
        (rand(78, (64, 8, 24)), [0], rand(79, (64, 32)), [0]),           # rows fastest over two legs: 24 x 4
        (rand(80, (16, 96)), [1], rand(81, (96, 2048)), [0]),            # P = B, rows fastest, 48-wide slabs
        (rand(82, (100, 6000)), [1], rand(83, (6000, 50)), [0]),         # 100 slabs of 60: split k ranges
        (rand(84, (4096,)), [0], rand(85, (4096, 200)), [0]),            # Q of one row
        (rand(86, (8, 16, 8, 24, 8)), [4, 1], rand(87, (16, 8, 12)), [1, 0]),  # rank 5: five map dims
        (rand(88, (20000, 64)), [1], rand(89, (64, 60)), [0]),           # 160 tiles: CTAs run several
        # few rows of P: one box covers several slabs, stacked as k-blocks
        (rand(90, (32, 96, 64)), [1, 2], rand(91, (96, 64, 16)), [0, 1]),  # 32 rows, 4 slabs over two k legs
        (rand(92, (8, 4096)), [1], rand(93, (24, 4096)), [1]),           # P = B, 24 rows, 4 slabs per box
        (rand(94, (16, 65536)), [1], rand(95, (65536,)), [0]),           # a matrix-vector product, split k
        (rand(96, (4, 8, 2048)), [2], rand(97, (2048, 8)), [0]),         # rows over two legs
        (rand(98, (20, 8192)), [1], rand(99, (8192, 3)), [0]),           # 20 rows: k-blocks 24 rows apart
    ]
    specs = []
    for A, la, B, lb in cases:
        At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        specs.append((At, list(la), Bt, list(lb), torch.empty(tn.result_shape(At, la, Bt, lb), device="cuda")))
    plan = tn.GroupPlan(specs, prec="bf16")
    assert [n for n in plan.launch_names() if n not in ("zero", "pack")] == ["gemm_tma"]
    for rep in range(2):
        for sp in specs:
            sp[4].fill_(float("nan"))
        plan.run()
        torch.cuda.synchronize()
        assert tn.sync_status() == 0
        for (A, la, B, lb), sp in zip(cases, specs):
            check(sp[4], A, la, B, lb, "bf16")
