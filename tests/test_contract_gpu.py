"""GPU parity of tn_contract and the grouped launch against the FP64 oracle.

Error model (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3.5):
rounding the operands and accumulating gives |C - C*| <= c |A||B| elementwise.
Each result is checked three ways:
  componentwise |C - C*| <= c * (|A||B|), with
      fp32   c = K * 2^-23          (float32 FMA, any summation order)
      bf16   c = 2^-7               (two bf16 roundings of 2^-9 each, plus accumulation)
      bf16x3 c = 2^-15 + K * 2^-23  (dropped lo*lo and rounded lo, ~2^-16, plus accumulation)
  normwise against the terms, ||C - C*||_F / || |A||B| ||_F <= t_abs:
      fp32 2^-20, bf16 2^-8, bf16x3 2^-16
  normwise against the result, ||C - C*||_F / ||C*||_F <= t_rel (1e-5, 1e-2,
      5e-5), applied when the result is well conditioned, i.e. when
      kappa = || |A||B| ||_F / ||C*||_F <= 32; a sum that cancels (large kappa)
      is judged by the two bounds above.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1905_01330_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NORM_TOL = {"fp32": 1e-5, "bf16": 1e-2, "bf16x3": 5e-5}
ABS_TOL = {"fp32": 2.0 ** -20, "bf16": 2.0 ** -8, "bf16x3": 2.0 ** -16}
KAPPA_MAX = 32.0


def comp_coef(prec, K):
    if prec == "fp32":
        return max(K, 1) * 2.0 ** -23
    if prec == "bf16":
        return 2.0 ** -7
    return 2.0 ** -15 + max(K, 1) * 2.0 ** -23


@pytest.fixture(scope="module")
def tn():
    from paper_1905_01330_gb300 import build, tn as tnmod
    build.build()
    tnmod.load()
    return tnmod


def check(C_gpu, A, la, B, lb, prec):
    ref = oracle.tensordot(A, la, B, lb)
    absref = oracle.tensordot(np.abs(A), la, np.abs(B), lb)
    got = C_gpu.double().cpu().numpy()
    assert got.shape == ref.shape
    K = int(np.prod([A.shape[p] for p in la])) if la else 1
    nrm, anrm = np.linalg.norm(ref), np.linalg.norm(absref)
    err = np.linalg.norm(got - ref)
    if anrm > 0:
        assert err / anrm <= ABS_TOL[prec], (err / anrm)
    if nrm > 0 and anrm / nrm <= KAPPA_MAX:
        assert err / nrm <= NORM_TOL[prec], (err / nrm)
    bound = comp_coef(prec, K) * absref + 1e-30
    bad = np.abs(got - ref) > bound
    assert not bad.any(), "componentwise bound violated at %d of %d elements" % (bad.sum(), bad.size)


def rand(seed, shape):
    return synth.normal_f32(seed, tuple(shape))


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x3"])
@pytest.mark.parametrize("seed", range(10))
def test_random_specs_parity(tn, prec, seed):
    # dims mixing multiples of 8 with ragged ones so tiles are partial
    st = synth.Stream(1000 + seed)
    sha, la, shb, lb = synth.contraction_spec(st, dims=(3, 8, 13, 24, 48), cap=1 << 17)
    A = rand(2000 + seed, sha)
    B = rand(3000 + seed, shb)
    C = tn.contract(torch.from_numpy(A).cuda(), la, torch.from_numpy(B).cuda(), lb, prec=prec)
    torch.cuda.synchronize()
    assert tn.sync_status() == 0
    check(C, A, la, B, lb, prec)


@pytest.mark.parametrize("prec", ["bf16", "bf16x3"])
@pytest.mark.parametrize("seed", range(4))
def test_random_specs_single_pass_kernel(tn, prec, seed):
    # tn_contract without scratch: the single-pass kernel that gathers and
    # converts operand tiles inside the GEMM CTA
    st = synth.Stream(1500 + seed)
    sha, la, shb, lb = synth.contraction_spec(st, dims=(3, 8, 13, 24, 48), cap=1 << 17)
    A = rand(2500 + seed, sha)
    B = rand(3500 + seed, shb)
    C = tn.contract(torch.from_numpy(A).cuda(), la, torch.from_numpy(B).cuda(), lb, prec=prec, packed=False)
    torch.cuda.synchronize()
    assert tn.sync_status() == 0
    check(C, A, la, B, lb, prec)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x3"])
def test_multi_tile_matmul_with_ragged_tail(tn, prec):
    A = rand(11, (300, 200))
    B = rand(12, (200, 270))
    C = tn.contract(torch.from_numpy(A).cuda(), [1], torch.from_numpy(B).cuda(), [0], prec=prec)
    check(C, A, [1], B, [0], prec)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x3"])
def test_permuted_legs_and_strided_views(tn, prec):
    A = rand(21, (16, 24, 8, 5))
    B = rand(22, (8, 7, 24, 16))
    At = torch.from_numpy(A).cuda()
    Bt = torch.from_numpy(B).cuda()
    la, lb = [2, 0, 1], [0, 3, 2]
    check(tn.contract(At, la, Bt, lb, prec=prec), A, la, B, lb, prec)
    # a non-contiguous view (permuted axes) is read in place through its strides
    Ap = At.permute(3, 1, 0, 2)
    Anp = np.ascontiguousarray(A.transpose(3, 1, 0, 2))
    check(tn.contract(Ap, [1, 2], Bt, [2, 3], prec=prec), Anp, [1, 2], B, [2, 3], prec)


def test_small_first_operand_fp32(tn):
    """FP32 contractions with a first operand of at most 16 rows and 16 shared
    indices against a long second one take the one-thread-per-column kernel:
    the MPO step of an energy sweep (W[w, w', s, s'] with T1[w, a', s, b] over
    w and s), a permuted view, K = 1 and the 16 x 16 limit."""
    cases = [
        (rand(81, (3, 3, 2, 2)), [0, 2], rand(82, (3, 96, 2, 80)), [0, 2]),   # MPO step
        (rand(83, (16, 16)), [1], rand(84, (16, 5000)), [0]),                  # at the limit
        (rand(85, (4, 1)), [1], rand(86, (1, 9000)), [0]),                     # K = 1
        (rand(87, (2, 7, 2)), [1, 2], rand(88, (40, 7, 2, 130)), [1, 2]),      # N over two legs
    ]
    for A, la, B, lb in cases:
        At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        C = tn.contract(At, la, Bt, lb, prec="fp32")
        torch.cuda.synchronize()
        check(C, A, la, B, lb, "fp32")
    # a permuted (non-contiguous) second operand
    B = rand(89, (64, 6, 128))
    Bt = torch.from_numpy(B).cuda().permute(2, 1, 0)
    A = rand(90, (5, 6))
    C = tn.contract(torch.from_numpy(A).cuda(), [1], Bt, [1], prec="fp32")
    check(C, A, [1], np.ascontiguousarray(B.transpose(2, 1, 0)), [1], "fp32")


def test_small_first_operand_fp32_grouped(tn):
    """An FP32 grouped plan whose contractions all have a small first operand
    (the MPO steps of a batch of environment sweeps, uneven environments)
    runs the grouped one-thread-per-column kernel."""
    cases = [(rand(91 + i, (3, 3, 2, 2)), [0, 2], rand(101 + i, (3, 16 * (i + 1), 2, 24 * (i + 2))), [0, 2])
             for i in range(5)]
    specs = []
    for A, la, B, lb in cases:
        At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        specs.append((At, la, Bt, lb, torch.full(tn.result_shape(At, la, Bt, lb), float("nan"), device="cuda")))
    plan = tn.GroupPlan(specs, prec="fp32")
    plan.run()
    torch.cuda.synchronize()
    assert tn.sync_status() == 0
    for (A, la, B, lb), sp in zip(cases, specs):
        check(sp[4], A, la, B, lb, "fp32")


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x3"])
def test_degenerate_shapes(tn, prec):
    # inner product (rank-0 result), mat-vec (N = 1), vec-mat (M = 1), outer product (K = 1)
    cases = [((37,), [0], (37,), [0]),
             ((40, 37), [1], (37,), [0]),
             ((37,), [0], (37, 9), [0]),
             ((2, 3), [], (4, 5, 6), []),
             ((5, 6, 7), [0, 1, 2], (7, 5, 6), [1, 2, 0])]
    for i, (sa, la, sb, lb) in enumerate(cases):
        A, B = rand(40 + i, sa), rand(50 + i, sb)
        C = tn.contract(torch.from_numpy(A).cuda(), la, torch.from_numpy(B).cuda(), lb, prec=prec)
        check(C, A, la, B, lb, prec)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x3"])
def test_maximum_rank(tn, prec):
    # rank 8 (the most a tensor may have): a rank-8 operand with four shared
    # legs in scattered positions, and a rank-8 result
    cases = [((2, 3, 2, 3, 2, 3, 2, 2), [1, 3, 5, 7], (3, 4, 3, 3, 2), [0, 2, 3, 4]),
             ((3, 4, 5, 6, 7), [2], (5, 2, 3, 2, 2), [0]),
             ((2, 2, 2, 2, 2, 2, 2, 9), [7, 0, 3], (2, 9, 2), [1, 2, 0])]
    for i, (sa, la, sb, lb) in enumerate(cases):
        A, B = rand(130 + i, sa), rand(140 + i, sb)
        At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        C = tn.contract(At, la, Bt, lb, prec=prec)
        assert C.dim() == len(sa) + len(sb) - 2 * len(la)
        check(C, A, la, B, lb, prec)
        if prec != "fp32":   # and the single-pass kernel (no scratch)
            check(tn.contract(At, la, Bt, lb, prec=prec, packed=False), A, la, B, lb, prec)


def test_paper_examples_on_gpu(tn):
    # ones(2) . ones(2) = 2 (Sec. III.B.4); ncon example equals matmul (App. B)
    o = torch.ones(2, device="cuda")
    assert float(tn.contract(o, [0], o, [0], prec="fp32").cpu()) == 2.0
    assert float(tn.contract(o, [0], o, [0], prec="bf16").cpu()) == 2.0
    a = torch.from_numpy(rand(61, (2, 2))).cuda()
    b = torch.from_numpy(rand(62, (2, 2))).cuda()
    c = tn.contract(a, [1], b, [0], prec="fp32")
    assert torch.linalg.norm((a.double() @ b.double()) - c.double()).item() < 1e-6


def test_empty_and_zero_size(tn):
    A = torch.zeros((0, 4), device="cuda")
    B = torch.from_numpy(rand(71, (4, 3))).cuda()
    assert tn.contract(A, [1], B, [0]).shape == (0, 3)
    A2 = torch.zeros((3, 0), device="cuda")
    B2 = torch.zeros((0, 5), device="cuda")
    C2 = tn.contract(A2, [1], B2, [0], prec="bf16")
    assert C2.shape == (3, 5) and torch.count_nonzero(C2).item() == 0


def test_errors_are_reported(tn):
    A = torch.zeros((3, 4), device="cuda")
    B = torch.zeros((5, 6), device="cuda")
    with pytest.raises(tn.TnError) as e:
        tn.contract(A, [1], B, [0])
    assert e.value.code == 2  # TN_ERR_SHAPE
    with pytest.raises(tn.TnError) as e:
        tn.contract(A, [0, 0], torch.zeros((3, 3), device="cuda"), [0, 1])
    assert e.value.code == 1  # TN_ERR_ARG


@pytest.mark.parametrize("prec", ["fp32", "bf16", "bf16x3"])
def test_grouped_small_specs(tn, prec):
    specs, host = [], []
    st = synth.Stream(77)
    for i in range(40):
        sha, la, shb, lb = synth.contraction_spec(st, dims=(3, 8, 16, 24), cap=1 << 15)
        A, B = rand(5000 + i, sha), rand(6000 + i, shb)
        At, Bt = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        C = torch.empty(tn.result_shape(At, la, Bt, lb), device="cuda")
        specs.append((At, list(la), Bt, list(lb), C))
        host.append((A, la, B, lb))
    plan = tn.GroupPlan(specs, prec=prec)
    plan.run()
    torch.cuda.synchronize()
    assert tn.sync_status() == 0
    for (A, la, B, lb), sp in zip(host, specs):
        check(sp[4], A, la, B, lb, prec)


def sampled_elements(A, la, B, lb, C, idx_list):
    """Oracle values of chosen result elements, one at a time: fix the free
    indices of A and B and contract what is left over all shared legs."""
    fa = [p for p in range(A.ndim) if p not in la]
    fb = [p for p in range(B.ndim) if p not in lb]
    out = []
    for idx in idx_list:
        ia, ib = idx[:len(fa)], idx[len(fa):]
        sa = [slice(None)] * A.ndim
        for p, v in zip(fa, ia):
            sa[p] = v
        sb = [slice(None)] * B.ndim
        for p, v in zip(fb, ib):
            sb[p] = v
        a, b = A[tuple(sa)], B[tuple(sb)]
        # remaining legs of a are the shared legs in A's order; pair them with b's
        ra = sorted(la)
        rb_pos = sorted(lb)
        legs_b = [rb_pos.index(lb[la.index(p)]) for p in ra]
        out.append(float(oracle.tensordot(a, list(range(len(ra))), b, legs_b)))
    return np.array(out)


def test_full_size_grouped_sampled(tn):
    """The bench workload (2048 specs, 2^24-element cap) in the bench's launch
    configuration; sampled result elements against the oracle."""
    specs_h = synth.contraction_specs(2048, seed=2)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2)
    specs = []
    for sha, la, shb, lb in specs_h:
        At = torch.randn(sha, device="cuda", generator=gen)
        Bt = torch.randn(shb, device="cuda", generator=gen)
        C = torch.empty(tn.result_shape(At, la, Bt, lb), device="cuda")
        specs.append((At, list(la), Bt, list(lb), C))
    rng = synth.Stream(9)
    sizes = [2 * np.prod(synth.spec_sizes(s)) for s in specs_h]
    order = np.argsort(sizes)[::-1]
    chosen = list(order[:3]) + [int(order[len(order) // 2]), int(order[-1])] + [rng.below(2048) for _ in range(3)]
    for prec in ("bf16", "bf16x3", "fp32"):
        plan = tn.GroupPlan(specs, prec=prec)
        plan.run()
        torch.cuda.synchronize()
        assert tn.sync_status() == 0
        for si in chosen:
            At, la, Bt, lb, C = specs[si]
            A, B = At.cpu().numpy(), Bt.cpu().numpy()
            Cc = C.cpu().numpy()
            idxs = [tuple(rng.below(n) for n in C.shape) for _ in range(16)]
            ref = sampled_elements(A, la, B, lb, Cc, idxs)
            absA, absB = np.abs(A), np.abs(B)
            aref = sampled_elements(absA, la, absB, lb, Cc, idxs)
            got = np.array([Cc[i] for i in idxs], dtype=np.float64)
            K = int(np.prod([A.shape[p] for p in la]))
            assert np.all(np.abs(got - ref) <= comp_coef(prec, K) * aref + 1e-30), (prec, si)
        del plan


def test_grouped_plan_on_pinned_host_operands(tn):
    """A plan whose operands and results are pinned host tensors (read and
    written by the kernels through unified addressing; the workspace on the
    GPU) gives the device plan's results."""
    specs_h = synth.contraction_specs(12, seed=5, dims=(8, 16, 24), cap=1 << 14)
    dev_specs, host_specs = [], []
    for i, (sa, la, sb, lb) in enumerate(specs_h):
        A = torch.from_numpy(synth.normal_f32(300 + i, sa))
        B = torch.from_numpy(synth.normal_f32(400 + i, sb))
        shape = tn.result_shape(A, la, B, lb)
        host_specs.append((A.pin_memory(), list(la), B.pin_memory(), list(lb),
                           torch.full(shape, float("nan")).pin_memory()))
        dev_specs.append((A.cuda(), list(la), B.cuda(), list(lb), torch.empty(shape, device="cuda")))
    for prec in ("bf16", "fp32"):
        pd = tn.GroupPlan(dev_specs, prec=prec)
        ph = tn.GroupPlan(host_specs, prec=prec, device=torch.device("cuda"))
        pd.run()
        ph.run()
        torch.cuda.synchronize()
        assert tn.sync_status() == 0
        for (_, _, _, _, Cd), (_, _, _, _, Ch) in zip(dev_specs, host_specs):
            ref = Cd.cpu()
            assert torch.isfinite(Ch).all()
            assert (Ch - ref).abs().max().item() <= 1e-5 * max(1.0, ref.abs().max().item()), prec
