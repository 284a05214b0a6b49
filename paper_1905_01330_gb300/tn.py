"""Python binding of libtn.so (include/tn.h): argument marshalling only.

PyTorch provides device memory and streams; every step of the computation
runs in the library's CUDA kernels. There is no fallback: if libtn.so is not
built, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

TN_MAX_RANK = 8
PREC = {"fp32": 0, "bf16": 1, "bf16x3": 2}
STATUS = {0: "TN_OK", 1: "TN_ERR_ARG", 2: "TN_ERR_SHAPE", 3: "TN_ERR_UNSUPPORTED", 4: "TN_ERR_CUDA",
          5: "TN_ERR_TIMEOUT", 6: "TN_ERR_WORKSPACE"}


class TnError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__("%s: %s (%d)" % (what, STATUS.get(code, "?"), code))
        self.code = code


class TnTensor(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("rank", ctypes.c_int32), ("dtype", ctypes.c_int32),
                ("shape", ctypes.c_int64 * TN_MAX_RANK), ("stride", ctypes.c_int64 * TN_MAX_RANK)]


class TnContractSpec(ctypes.Structure):
    _fields_ = [("A", TnTensor), ("B", TnTensor), ("C", TnTensor), ("nshared", ctypes.c_int32),
                ("legsA", ctypes.c_int32 * TN_MAX_RANK), ("legsB", ctypes.c_int32 * TN_MAX_RANK)]


class TnChain(ctypes.Structure):
    """tn_mps / tn_mpo: n cores, physical dim d, host bond array, host table of device pointers."""
    _fields_ = [("n", ctypes.c_int32), ("d", ctypes.c_int32), ("bond", ctypes.POINTER(ctypes.c_int64)),
                ("cores", ctypes.POINTER(ctypes.c_void_p))]


class TnNconStep(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int32), ("b", ctypes.c_int32), ("nshared", ctypes.c_int32),
                ("rank", ctypes.c_int32), ("legs_a", ctypes.c_int32 * TN_MAX_RANK),
                ("legs_b", ctypes.c_int32 * TN_MAX_RANK), ("shape", ctypes.c_int64 * TN_MAX_RANK)]


def chain_desc(cores, phys_axis: int = 1):
    """(TnChain, keepalive) for a list of contiguous float32 CUDA tensors; bonds
    are the first axis of each core plus the last core's second bond axis."""
    for c in cores:
        if c.dtype != torch.float32 or not c.is_cuda or not c.is_contiguous():
            raise TypeError("MPS/MPO cores must be contiguous float32 CUDA tensors")
    n = len(cores)
    right_axis = 2 if cores[-1].dim() == 3 else 1
    bonds = [c.shape[0] for c in cores] + [cores[-1].shape[right_axis]]
    bond_arr = (ctypes.c_int64 * (n + 1))(*bonds)
    ptr_arr = (ctypes.c_void_p * n)(*[c.data_ptr() for c in cores])
    ch = TnChain()
    ch.n = n
    ch.d = cores[0].shape[phys_axis]
    ch.bond = ctypes.cast(bond_arr, ctypes.POINTER(ctypes.c_int64))
    ch.cores = ctypes.cast(ptr_arr, ctypes.POINTER(ctypes.c_void_p))
    return ch, (bond_arr, ptr_arr, cores)


_lib = None
_EXPORTS = None


def exported_symbols():
    """Names of the entry points declared in include/tn.h that the binding uses."""
    return list(_signatures().keys())


def _signatures():
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    tp = ctypes.POINTER(TnTensor)
    ip = ctypes.POINTER(ctypes.c_int)
    return {
        "tn_tensor_init": (i32, [tp, vp, i32, ctypes.POINTER(i64)]),
        "tn_contract": (i32, [tp, ip, tp, ip, i32, tp, i32, vp]),
        "tn_contract_workspace_bytes": (ctypes.c_size_t, [tp, ip, tp, ip, i32, tp, i32]),
        "tn_contract_ws": (i32, [tp, ip, tp, ip, i32, tp, i32, vp, ctypes.c_size_t, vp]),
        "tn_group_plan_create": (i32, [ctypes.POINTER(TnContractSpec), i32, i32, ctypes.POINTER(vp)]),
        "tn_group_plan_workspace_bytes": (ctypes.c_size_t, [vp]),
        "tn_group_plan_upload": (i32, [vp, vp, ctypes.c_size_t, vp]),
        "tn_group_plan_run": (i32, [vp, vp, ctypes.c_size_t, vp]),
        "tn_group_plan_destroy": (None, [vp]),
        "tn_group_plan_flops": (ctypes.c_double, [vp]),
        "tn_group_plan_bytes": (ctypes.c_double, [vp]),
        "tn_group_plan_launches": (i32, [vp]),
        "tn_group_plan_run_launch": (i32, [vp, vp, ctypes.c_size_t, i32, vp]),
        "tn_group_plan_launch_name": (ctypes.c_char_p, [vp, i32]),
        "tn_group_plan_launch_bytes": (ctypes.c_double, [vp, i32]),
        "tn_group_plan_autotune": (i32, [vp, vp, ctypes.c_size_t, vp]),
        "tn_group_plan_schedule": (i32, [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]),
        "tn_group_plan_set_schedule": (i32, [vp, i32, i32, i32, i32]),
        "tn_staged_plan_create": (i32, [ctypes.POINTER(TnContractSpec), i32, i32, vp, ctypes.c_size_t, vp,
                                        ctypes.c_size_t, i32, ctypes.POINTER(vp)]),
        "tn_staged_plan_chunks": (i32, [vp]),
        "tn_staged_plan_flops": (ctypes.c_double, [vp]),
        "tn_staged_plan_set_schedule": (i32, [vp, i32, i32, i32, i32]),
        "tn_staged_plan_workspace_bytes": (ctypes.c_size_t, [vp]),
        "tn_staged_plan_upload": (i32, [vp, vp, ctypes.c_size_t, vp]),
        "tn_staged_plan_run": (i32, [vp, vp, ctypes.c_size_t, vp, vp, vp]),
        "tn_staged_plan_destroy": (None, [vp]),
        "tn_chunk_bounds": (i32, [ctypes.POINTER(ctypes.c_double), i32, i32, ctypes.POINTER(i32),
                                  ctypes.POINTER(i32)]),
        "tn_mps_inner_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(TnChain), ctypes.POINTER(TnChain)]),
        "tn_mps_inner": (i32, [ctypes.POINTER(TnChain), ctypes.POINTER(TnChain), i32, vp, ctypes.c_size_t, vp, vp]),
        "tn_mps_expect_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(TnChain), ctypes.POINTER(TnChain)]),
        "tn_mps_expect_grouped_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(TnChain), i32,
                                                                    ctypes.POINTER(TnChain), i32]),
        "tn_mps_expect_grouped": (i32, [ctypes.POINTER(TnChain), i32, ctypes.POINTER(TnChain), i32, vp,
                                        ctypes.c_size_t, vp, vp]),
        "tn_mps_expect_grouped_plan": (i32, [ctypes.POINTER(TnChain), i32, ctypes.POINTER(TnChain), i32, vp,
                                             ctypes.c_size_t, ctypes.POINTER(vp), vp]),
        "tn_mps_expect_grouped_run": (i32, [vp, vp, vp]),
        "tn_mps_expect_grouped_destroy": (None, [vp]),
        "tn_mps_expect": (i32, [ctypes.POINTER(TnChain), ctypes.POINTER(TnChain), i32, vp, ctypes.c_size_t, vp, vp]),
        "tn_mps_classify_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(TnChain), i32, i32, i32, i32]),
        "tn_mps_classify": (i32, [ctypes.POINTER(TnChain), i32, i32, vp, i32, i32, i32, vp, vp, vp,
                                  ctypes.c_size_t, vp]),
        "tn_mps_classify_backward": (i32, [ctypes.POINTER(TnChain), i32, i32, vp, i32, i32, i32, vp,
                                           ctypes.POINTER(ctypes.c_void_p), vp, ctypes.c_size_t, vp]),
        "tn_mps_classify_loss": (i32, [vp, vp, i32, i32, vp, vp, vp]),
        "tn_split_node_workspace_bytes": (ctypes.c_size_t, [tp, ip, i32, ip, i32]),
        "tn_split_node": (i32, [tp, ip, i32, ip, i32, i64, ctypes.c_double, i32, vp, vp, vp, vp,
                                ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int32), vp, ctypes.c_size_t, vp]),
        "tn_split_truncation": (i64, [ctypes.POINTER(ctypes.c_float), i64, i64, ctypes.c_double]),
        "tn_ncon_plan": (i32, [i32, ip, ctypes.POINTER(i64), ip, ip, i32, ip, i32, ctypes.POINTER(TnNconStep), i32,
                               ip, ip, ip]),
        "tn_mps_classify_separate_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(TnChain), i32, i32, i32]),
        "tn_mps_classify_separate": (i32, [ctypes.POINTER(TnChain), i32, vp, i32, i32, i32, vp, vp, vp,
                                           ctypes.c_size_t, vp]),
        "tn_mps_classify_separate_backward": (i32, [ctypes.POINTER(TnChain), i32, vp, i32, i32, i32, vp,
                                                    ctypes.POINTER(ctypes.c_void_p), vp, ctypes.c_size_t, vp]),
        "tn_check_wait_timeout": (i32, [ctypes.c_uint64, vp]),
        "tn_check_grid_barrier_timeout": (i32, [ctypes.c_uint64, vp, vp]),
        "tn_sync_status": (i32, [vp]),
        "tn_status_string": (ctypes.c_char_p, [i32]),
    }


def library_path() -> str:
    return _build.LIB


def load(require_gpu: bool = True):
    """Loads libtn.so (built by build.build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libtn.so is not built (run paper_1905_01330_gb300.build.build()); "
                           "there is no CPU fallback")
    if require_gpu and not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: libtn.so runs on the GPU only")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _signatures().items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(code: int, what: str):
    if code != 0:
        raise TnError(code, what)


def tensor_desc(t: torch.Tensor) -> TnTensor:
    if t.dtype != torch.float32:
        raise TypeError("libtn contracts float32 tensors")
    if t.dim() > TN_MAX_RANK:
        raise ValueError("rank > 8")
    d = TnTensor()
    d.data = t.data_ptr() if t.numel() > 0 else None
    d.rank = t.dim()
    d.dtype = 0
    for i, (n, s) in enumerate(zip(t.shape, t.stride())):
        d.shape[i] = n
        d.stride[i] = s
    return d


def result_shape(A: torch.Tensor, legsA, B: torch.Tensor, legsB):
    return [A.shape[p] for p in range(A.dim()) if p not in legsA] + \
           [B.shape[p] for p in range(B.dim()) if p not in legsB]


def contract(A: torch.Tensor, legsA, B: torch.Tensor, legsB, prec: str = "bf16",
             out: torch.Tensor | None = None, stream=None, packed: bool = True) -> torch.Tensor:
    """tensordot of A and B over legsA[j] <-> legsB[j]. BF16 / BF16X3 run as
    pack + tcgen05 GEMM on a scratch workspace (tn_contract_ws); packed=False
    (or FP32) runs tn_contract's single-pass kernels."""
    lib = load()
    legsA, legsB = list(legsA), list(legsB)
    if len(legsA) != len(legsB):
        raise ValueError("legsA and legsB differ in length")
    if out is None:
        shape = result_shape(A, legsA, B, legsB)
        out = torch.empty(shape, dtype=torch.float32, device=A.device)
    da, db, dc = tensor_desc(A), tensor_desc(B), tensor_desc(out)
    k = len(legsA)
    la = (ctypes.c_int * max(k, 1))(*legsA)
    lb = (ctypes.c_int * max(k, 1))(*legsB)
    if packed and prec != "fp32":
        nbytes = lib.tn_contract_workspace_bytes(ctypes.byref(da), la, ctypes.byref(db), lb, k, ctypes.byref(dc),
                                                 PREC[prec])
        ws = _workspace(nbytes, A.device) if nbytes > 0 else None
        _check(lib.tn_contract_ws(ctypes.byref(da), la, ctypes.byref(db), lb, k, ctypes.byref(dc), PREC[prec],
                                  ctypes.c_void_p(ws.data_ptr() if ws is not None else None),
                                  ws.numel() if ws is not None else 0, _stream(stream)), "tn_contract_ws")
        out._tn_keep = ws
        return out
    _check(lib.tn_contract(ctypes.byref(da), la, ctypes.byref(db), lb, k, ctypes.byref(dc),
                           PREC[prec], _stream(stream)), "tn_contract")
    return out


def sync_status(stream=None) -> int:
    return load().tn_sync_status(_stream(stream))


def check_wait_timeout(limit_ns: int = 20_000_000, stream=None) -> None:
    """Launches the failure-path check kernel (tn_check_wait_timeout)."""
    _check(load().tn_check_wait_timeout(limit_ns, _stream(stream)), "tn_check_wait_timeout")


def check_grid_barrier_timeout(limit_ns: int = 20_000_000, stream=None) -> None:
    """Launches the device-wide barrier's failure-path check (tn_check_grid_barrier_timeout)."""
    counter = torch.zeros(64, dtype=torch.int32, device="cuda")
    _check(load().tn_check_grid_barrier_timeout(limit_ns, ctypes.c_void_p(counter.data_ptr()), _stream(stream)),
           "tn_check_grid_barrier_timeout")


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def ncon_plan(shapes, network, con_order=None, out_order=None, lib=None):
    """tn_ncon_plan on host shapes and labels: (steps, out_perm) -- steps as
    (a, b, legs_a, legs_b, result shape), b = -1 for a trace."""
    lib = lib or load()
    n = len(shapes)
    if len(network) != n:
        raise TnError(1, "ncon: one label list per tensor")
    ranks = (ctypes.c_int * n)(*[len(sh) for sh in shapes])
    flat_dims = [int(d) for sh in shapes for d in sh]
    flat_labels = [int(x) for labels in network for x in labels]
    if any(len(labels) != len(sh) for labels, sh in zip(network, shapes)):
        raise TnError(1, "ncon: one label per leg")
    dims = (ctypes.c_int64 * max(len(flat_dims), 1))(*flat_dims)
    labs = (ctypes.c_int * max(len(flat_labels), 1))(*flat_labels)
    co = list(con_order) if con_order is not None else []
    oo = list(out_order) if out_order is not None else []
    coa = (ctypes.c_int * max(len(co), 1))(*co)
    ooa = (ctypes.c_int * max(len(oo), 1))(*oo)
    cnt, perm, orank = ctypes.c_int(0), (ctypes.c_int * TN_MAX_RANK)(), ctypes.c_int(0)
    _check(lib.tn_ncon_plan(n, ranks, dims, labs, coa, len(co), ooa, len(oo), None, 0, ctypes.byref(cnt), perm,
                            ctypes.byref(orank)), "tn_ncon_plan")
    steps = (TnNconStep * max(cnt.value, 1))()
    _check(lib.tn_ncon_plan(n, ranks, dims, labs, coa, len(co), ooa, len(oo), steps, cnt.value, ctypes.byref(cnt),
                            perm, ctypes.byref(orank)), "tn_ncon_plan")
    out = []
    for st in steps[:cnt.value]:
        k = st.nshared
        out.append((st.a, st.b, list(st.legs_a[:k]), list(st.legs_b[:k]), list(st.shape[:st.rank])))
    return out, list(perm[:orank.value])


def ncon(tensors, network, con_order=None, out_order=None, prec: str = "fp32", stream=None):
    """ncon (Appendix B): evaluates a labelled network by the steps tn_ncon_plan
    gives, each a tn_contract call (a trace contracts the traced legs with the
    identity matrix); returns the result with its legs in out order (a
    permuted view of the last step's result)."""
    lib = load()
    steps, perm = ncon_plan([list(t.shape) for t in tensors], network, con_order, out_order, lib)
    ops = list(tensors)
    for a, b, la, lb, shape in steps:
        A = ops[a]
        if b < 0:
            d = A.shape[la[0]]
            eye = torch.from_numpy(np.eye(d, dtype=np.float32)).to(A.device)
            R = contract(A, [la[0], lb[0]], eye, [0, 1], prec=prec, stream=stream)
        else:
            R = contract(A, la, ops[b], lb, prec=prec, stream=stream)
        assert list(R.shape) == shape
        ops.append(R)
    return ops[-1].permute(perm) if perm else ops[-1]


class NconPlan:
    """ncon planned once for fixed tensors (Appendix B): the steps of
    tn_ncon_plan with their results allocated and every tn_contract /
    tn_contract_ws argument built here, so run() is one C call per step and
    can be captured in a CUDA graph (capture()/replay()). The tensors must stay
    alive and in place; their values may change between runs."""

    def __init__(self, tensors, network, con_order=None, out_order=None, prec: str = "fp32"):
        self.lib = lib = load()
        self.prec = PREC[prec]
        steps, self.perm = ncon_plan([list(t.shape) for t in tensors], network, con_order, out_order, lib)
        dev = tensors[0].device
        ops = list(tensors)
        self._keep = []
        self.calls = []
        for a, b, la, lb, shape in steps:
            A = ops[a]
            if b < 0:
                d = A.shape[la[0]]
                B = torch.from_numpy(np.eye(d, dtype=np.float32)).to(dev)
                la, lb = [la[0], lb[0]], [0, 1]
            else:
                B = ops[b]
            C = torch.empty(shape, dtype=torch.float32, device=dev)
            da, db, dc = tensor_desc(A), tensor_desc(B), tensor_desc(C)
            k = len(la)
            ia = (ctypes.c_int * max(k, 1))(*la)
            ib = (ctypes.c_int * max(k, 1))(*lb)
            ws = None
            if self.prec != PREC["fp32"]:
                nb = lib.tn_contract_workspace_bytes(ctypes.byref(da), ia, ctypes.byref(db), ib, k,
                                                     ctypes.byref(dc), self.prec)
                ws = _workspace(nb, dev) if nb > 0 else None
            self._keep += [A, B, C, da, db, dc, ia, ib, ws]
            self.calls.append((ctypes.byref(da), ia, ctypes.byref(db), ib, k, ctypes.byref(dc), ws))
            ops.append(C)
        self.result = ops[-1].permute(self.perm) if self.perm else ops[-1]
        self.graph = None

    def run(self, stream=None):
        """Runs every step on `stream` (default: the current stream); returns the result view."""
        st = _stream(stream)
        for da, ia, db, ib, k, dc, ws in self.calls:
            if ws is not None:
                _check(self.lib.tn_contract_ws(da, ia, db, ib, k, dc, self.prec, ctypes.c_void_p(ws.data_ptr()),
                                               ws.numel(), st), "tn_contract_ws")
            else:
                _check(self.lib.tn_contract(da, ia, db, ib, k, dc, self.prec, st), "tn_contract")
        return self.result

    def capture(self):
        """Records run() in a CUDA graph (after one eager run on a side stream)."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.run()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self

    def replay(self):
        self.graph.replay()
        return self.result


def split_node(A: torch.Tensor, left_legs, right_legs, max_singular_values: int | None = None,
               max_truncation_err: float | None = None, full_svd: bool = False, stream=None,
               info: dict | None = None):
    """Splits node A by the SVD of its matrix view (tn_split_node): rows over
    left_legs, columns over right_legs. Returns (u_s, s_vh, dropped) -- U sqrt(S)
    of shape left dims + (k,), sqrt(S) V^T of shape (k,) + right dims, and the
    dropped singular values -- or, with full_svd, (u, s, vh, dropped) with s
    the k kept singular values (the diagonal of the singular-value node).
    Synchronises the stream (k decides the output shapes). info, if given,
    receives the Jacobi sweep count."""
    lib = load()
    left, right = [int(p) for p in left_legs], [int(p) for p in right_legs]
    ad = tensor_desc(A)
    la = (ctypes.c_int * max(len(left), 1))(*left)
    ra = (ctypes.c_int * max(len(right), 1))(*right)
    ws_bytes = lib.tn_split_node_workspace_bytes(ctypes.byref(ad), la, len(left), ra, len(right))
    if ws_bytes == 0:
        raise TnError(1, "tn_split_node: legs must partition the node's legs")
    ldims = [A.shape[p] for p in left]
    rdims = [A.shape[p] for p in right]
    M = int(np.prod(ldims)) if ldims else 1
    N = int(np.prod(rdims)) if rdims else 1
    r = min(M, N)
    dev = A.device
    U = torch.empty(max(M * r, 1), dtype=torch.float32, device=dev)
    Vt = torch.empty(max(r * N, 1), dtype=torch.float32, device=dev)
    S = torch.empty(max(r, 1), dtype=torch.float32, device=dev)
    D = torch.empty(max(r, 1), dtype=torch.float32, device=dev)
    ws = _workspace(ws_bytes, dev)
    kept = ctypes.c_int64(0)
    sweeps = ctypes.c_int32(0)
    _check(lib.tn_split_node(ctypes.byref(ad), la, len(left), ra, len(right),
                             int(max_singular_values) if max_singular_values is not None else 0,
                             float(max_truncation_err) if max_truncation_err is not None else -1.0,
                             0 if full_svd else 1, U.data_ptr(), S.data_ptr(), Vt.data_ptr(), D.data_ptr(),
                             ctypes.byref(kept), ctypes.byref(sweeps), ws.data_ptr(), ws.numel(),
                             _stream(stream)), "tn_split_node")
    k = kept.value
    if info is not None:
        info["sweeps"] = sweeps.value
    u = U[:M * k].view(ldims + [k])
    vh = Vt[:k * N].view([k] + rdims)
    dropped = D[:r - k]
    if full_svd:
        return u, S[:k], vh, dropped
    return u, vh, dropped


def mps_inner(bra, ket, prec: str = "fp32", stream=None, out: torch.Tensor | None = None):
    """<bra|ket> of two MPS (lists of (D, d, D') cores) as a float64 CUDA tensor
    [value, log_scale]: <bra|ket> = value * exp(log_scale) (tn_mps_inner)."""
    lib = load()
    cb, kb = chain_desc(bra)
    ck, kk = chain_desc(ket)
    dev = bra[0].device
    ws = _workspace(lib.tn_mps_inner_workspace_bytes(ctypes.byref(cb), ctypes.byref(ck)), dev)
    res = out if out is not None else torch.empty(2, dtype=torch.float64, device=dev)
    _check(lib.tn_mps_inner(ctypes.byref(cb), ctypes.byref(ck), PREC[prec], ctypes.c_void_p(ws.data_ptr()),
                            ws.numel(), ctypes.c_void_p(res.data_ptr()), _stream(stream)), "tn_mps_inner")
    res._tn_keep = (ws, kb, kk)
    return res


def mps_expect(psi, mpo, prec: str = "fp32", stream=None, out: torch.Tensor | None = None):
    """<psi|H|psi> and <psi|psi> (tn_mps_expect) as a float64 CUDA tensor
    [e_value, e_log_scale, n_value, n_log_scale]. mpo cores are (w, w', d, d)."""
    lib = load()
    cp, kp = chain_desc(psi)
    ch, kh = chain_desc(mpo, phys_axis=2)
    dev = psi[0].device
    ws = _workspace(lib.tn_mps_expect_workspace_bytes(ctypes.byref(cp), ctypes.byref(ch)), dev)
    res = out if out is not None else torch.empty(4, dtype=torch.float64, device=dev)
    _check(lib.tn_mps_expect(ctypes.byref(cp), ctypes.byref(ch), PREC[prec], ctypes.c_void_p(ws.data_ptr()),
                             ws.numel(), ctypes.c_void_p(res.data_ptr()), _stream(stream)), "tn_mps_expect")
    res._tn_keep = (ws, kp, kh)
    return res


class ExpectGroupedPlan:
    """tn_mps_expect_grouped planned once (tn_mps_expect_grouped_plan): the
    host layout and its uploaded tables are kept, and run() only launches.
    The states' and the MPO's tensors are read at every run (values changed
    in place are picked up); they must stay allocated."""

    def __init__(self, psis, mpo, prec: str = "fp32", stream=None):
        lib = load()
        count = len(psis)
        arr = (TnChain * count)()
        keep = []
        for k, cores in enumerate(psis):
            c, kc = chain_desc(cores)
            arr[k] = c
            keep.append(kc)
        ch, kh = chain_desc(mpo, phys_axis=2)
        self.count = count
        self.device = psis[0][0].device
        nbytes = lib.tn_mps_expect_grouped_workspace_bytes(arr, count, ctypes.byref(ch), PREC[prec])
        if nbytes == 0:
            raise TnError(1, "tn_mps_expect_grouped_workspace_bytes (invalid chains or MPO)")
        self.ws = _workspace(nbytes, self.device)
        handle = ctypes.c_void_p()
        _check(lib.tn_mps_expect_grouped_plan(arr, count, ctypes.byref(ch), PREC[prec],
                                              ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(),
                                              ctypes.byref(handle), _stream(stream)), "tn_mps_expect_grouped_plan")
        self.handle = handle
        self._keep = (arr, keep, ch, kh, psis, mpo)

    def run(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """[count, 4] float64 {e_value, e_log_scale, n_value, n_log_scale} per state."""
        res = out if out is not None else torch.empty(self.count, 4, dtype=torch.float64, device=self.device)
        _check(load().tn_mps_expect_grouped_run(self.handle, ctypes.c_void_p(res.data_ptr()), _stream(stream)),
               "tn_mps_expect_grouped_run")
        return res

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.tn_mps_expect_grouped_destroy(self.handle)
            self.handle = None


def mps_expect_grouped(psis, mpo, prec: str = "fp32", stream=None, out: torch.Tensor | None = None):
    """tn_mps_expect for a batch of MPS (a list of core lists, bond dims may
    differ) sharing one MPO, as grouped launches (tn_mps_expect_grouped).
    Returns a float64 CUDA tensor [count, 4] of {e_value, e_log_scale,
    n_value, n_log_scale} per state."""
    lib = load()
    count = len(psis)
    arr = (TnChain * count)()
    keep = []
    for k, cores in enumerate(psis):
        c, kc = chain_desc(cores)
        arr[k] = c
        keep.append(kc)
    ch, kh = chain_desc(mpo, phys_axis=2)
    dev = psis[0][0].device
    nbytes = lib.tn_mps_expect_grouped_workspace_bytes(arr, count, ctypes.byref(ch), PREC[prec])
    if nbytes == 0:
        raise TnError(1, "tn_mps_expect_grouped_workspace_bytes (invalid chains or MPO)")
    ws = _workspace(nbytes, dev)
    res = out if out is not None else torch.empty(count, 4, dtype=torch.float64, device=dev)
    _check(lib.tn_mps_expect_grouped(arr, count, ctypes.byref(ch), PREC[prec], ctypes.c_void_p(ws.data_ptr()),
                                     ws.numel(), ctypes.c_void_p(res.data_ptr()), _stream(stream)),
           "tn_mps_expect_grouped")
    res._tn_keep = (ws, keep, kh)
    return res


class GroupPlan:
    """A grouped contraction (tn_group_plan_*): specs = [(A, legsA, B, legsB, C), ...]."""

    def __init__(self, specs, prec: str = "bf16", stream=None, device=None):
        lib = load()
        arr = (TnContractSpec * max(len(specs), 1))()
        for i, (A, la, B, lb, C) in enumerate(specs):
            arr[i].A = tensor_desc(A)
            arr[i].B = tensor_desc(B)
            arr[i].C = tensor_desc(C)
            arr[i].nshared = len(la)
            for j in range(len(la)):
                arr[i].legsA[j] = la[j]
                arr[i].legsB[j] = lb[j]
        self._keep = specs
        h = ctypes.c_void_p()
        _check(lib.tn_group_plan_create(arr, len(specs), PREC[prec], ctypes.byref(h)), "tn_group_plan_create")
        self._h = h
        self.prec = prec
        nbytes = lib.tn_group_plan_workspace_bytes(h)
        # the workspace lives on the GPU; the operands and results may also be
        # pinned host tensors (device-accessible through unified addressing)
        dev = device if device is not None else (specs[0][0].device if specs and specs[0][0].is_cuda
                                                 else torch.device("cuda"))
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        self.ws_bytes = self.workspace.numel()
        self.flops = lib.tn_group_plan_flops(h)
        self.bytes = lib.tn_group_plan_bytes(h)
        self.launches = lib.tn_group_plan_launches(h)
        _check(lib.tn_group_plan_upload(h, ctypes.c_void_p(self.workspace.data_ptr()), self.ws_bytes,
                                        _stream(stream)), "tn_group_plan_upload")

    def run(self, stream=None):
        _check(load().tn_group_plan_run(self._h, ctypes.c_void_p(self.workspace.data_ptr()), self.ws_bytes,
                                        _stream(stream)), "tn_group_plan_run")

    def autotune(self, stream=None):
        """Times the candidate GEMM schedules on the device and keeps the
        fastest (tn_group_plan_autotune); returns self.schedule()."""
        _check(load().tn_group_plan_autotune(self._h, ctypes.c_void_p(self.workspace.data_ptr()), self.ws_bytes,
                                             _stream(stream)), "tn_group_plan_autotune")
        self.launches = load().tn_group_plan_launches(self._h)
        return self.schedule()

    SCHEDULE_CLASSES = ("thin", "short_k", "long_k")

    def set_schedule(self, cls: str, tile_width: int, long_k: bool, store16: bool, stream=None):
        """Sets the GEMM schedule of one class by hand and uploads the plan again."""
        lib = load()
        _check(lib.tn_group_plan_set_schedule(self._h, self.SCHEDULE_CLASSES.index(cls), tile_width,
                                              1 if long_k else 0, 1 if store16 else 0),
               "tn_group_plan_set_schedule")
        _check(lib.tn_group_plan_upload(self._h, ctypes.c_void_p(self.workspace.data_ptr()), self.ws_bytes,
                                        _stream(stream)), "tn_group_plan_upload")
        self.launches = lib.tn_group_plan_launches(self._h)

    def schedule(self):
        """{class: (tile_width, long_k, store16)} for the classes thin, short_k, long_k."""
        lib = load()
        out = {}
        for c, name in enumerate(self.SCHEDULE_CLASSES):
            w, lk, s16 = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
            _check(lib.tn_group_plan_schedule(self._h, c, ctypes.byref(w), ctypes.byref(lk), ctypes.byref(s16)),
                   "tn_group_plan_schedule")
            out[name] = (w.value, lk.value, s16.value)
        return out

    def launch_names(self):
        lib = load()
        return [lib.tn_group_plan_launch_name(self._h, i).decode() for i in range(self.launches)]

    def launch_bytes(self):
        """Algorithmic bytes of each launch (tn_group_plan_launch_bytes)."""
        lib = load()
        return [lib.tn_group_plan_launch_bytes(self._h, i) for i in range(self.launches)]

    def run_launch(self, index: int, stream=None):
        """Launch `index` of the run's sequence alone (tn_group_plan_run_launch)."""
        _check(load().tn_group_plan_run_launch(self._h, ctypes.c_void_p(self.workspace.data_ptr()), self.ws_bytes,
                                               index, _stream(stream)), "tn_group_plan_run_launch")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.tn_group_plan_destroy(h)
            self._h = None


# ---------------------------------------------------------------------------
# MPS classifier (Sec. IV.A)
# ---------------------------------------------------------------------------

def chunk_bounds(weights, chunks: int):
    """Cuts a sequence of items with the given weights into at most `chunks`
    runs of consecutive items of about equal total weight (tn_chunk_bounds,
    host code in the library): returns the run boundaries [0, ..., len(weights)]."""
    lib = load(require_gpu=False)
    n = len(weights)
    w = (ctypes.c_double * max(n, 1))(*[float(x) for x in weights])
    out = (ctypes.c_int32 * (chunks + 1))()
    m = ctypes.c_int32()
    _check(lib.tn_chunk_bounds(w, n, chunks, out, ctypes.byref(m)), "tn_chunk_bounds")
    return [out[i] for i in range(m.value)]


def _spec_array(specs):
    arr = (TnContractSpec * max(len(specs), 1))()
    for i, (A, la, B, lb, C) in enumerate(specs):
        arr[i].A = tensor_desc(A)
        arr[i].B = tensor_desc(B)
        arr[i].C = tensor_desc(C)
        arr[i].nshared = len(la)
        for j in range(len(la)):
            arr[i].legsA[j] = la[j]
            arr[i].legsB[j] = lb[j]
    return arr


class StagedGroupPlan:
    """A grouped contraction fed from pinned host memory and drained back to it
    in chunks (tn_staged_plan_*). The specs' operands must fill one device
    buffer `dev_in` and their results another, `dev_out`, in spec order (each
    chunk of consecutive specs then owns one contiguous range of each).
    run(host_in, host_out): the library copies chunk c's operands host ->
    device on one of its streams while chunk c-1 is contracted on a second and
    chunk c-2's results go device -> host on a third; the caller's stream
    waits for the last copy. host_in / host_out are pinned tensors laid out
    like dev_in / dev_out."""

    def __init__(self, specs, dev_in: torch.Tensor, dev_out: torch.Tensor, chunks: int = 8, prec: str = "bf16",
                 schedule=None, stream=None):
        if dev_in.dim() != 1 or dev_out.dim() != 1:
            raise ValueError("dev_in and dev_out must be 1-D buffers")
        lib = load()
        arr = _spec_array(specs)
        h = ctypes.c_void_p()
        _check(lib.tn_staged_plan_create(arr, len(specs), PREC[prec], ctypes.c_void_p(dev_in.data_ptr()),
                                         dev_in.numel() * dev_in.element_size(),
                                         ctypes.c_void_p(dev_out.data_ptr()),
                                         dev_out.numel() * dev_out.element_size(), chunks, ctypes.byref(h)),
               "tn_staged_plan_create")
        self._h = h
        self._keep = (specs, dev_in, dev_out)
        self.dev_in, self.dev_out = dev_in, dev_out
        self.chunks = lib.tn_staged_plan_chunks(h)
        self.flops = lib.tn_staged_plan_flops(h)
        if schedule:
            for cls, (w, lk, s16) in schedule.items():
                _check(lib.tn_staged_plan_set_schedule(h, GroupPlan.SCHEDULE_CLASSES.index(cls), w, int(bool(lk)),
                                                       int(bool(s16))), "tn_staged_plan_set_schedule")
        nbytes = lib.tn_staged_plan_workspace_bytes(h)
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev_in.device)
        self.ws_bytes = self.workspace.numel()
        _check(lib.tn_staged_plan_upload(h, ctypes.c_void_p(self.workspace.data_ptr()), self.ws_bytes,
                                         _stream(stream)), "tn_staged_plan_upload")

    def run(self, host_in: torch.Tensor, host_out: torch.Tensor, stream=None):
        if host_in.numel() * host_in.element_size() < self.dev_in.numel() * self.dev_in.element_size() or \
                host_out.numel() * host_out.element_size() < self.dev_out.numel() * self.dev_out.element_size():
            raise ValueError("host buffers must be laid out like dev_in / dev_out")
        _check(load().tn_staged_plan_run(self._h, ctypes.c_void_p(self.workspace.data_ptr()), self.ws_bytes,
                                         ctypes.c_void_p(host_in.data_ptr()), ctypes.c_void_p(host_out.data_ptr()),
                                         _stream(stream)), "tn_staged_plan_run")

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.tn_staged_plan_destroy(self._h)
            self._h = None


def classifier_workspace(cores, label_site: int, n_labels: int, batch: int, ckpt_every: int) -> torch.Tensor:
    lib = load()
    ch, keep = chain_desc_classifier(cores, label_site)
    nbytes = lib.tn_mps_classify_workspace_bytes(ctypes.byref(ch), label_site, n_labels, batch, ckpt_every)
    return _workspace(nbytes, cores[0].device)


def chain_desc_classifier(cores, label_site: int):
    """tn_mps of a classifier MPS: the label core (D, 2, L, D') keeps its bonds."""
    for c in cores:
        if c.dtype != torch.float32 or not c.is_cuda or not c.is_contiguous():
            raise TypeError("classifier cores must be contiguous float32 CUDA tensors")
    n = len(cores)
    bonds = [c.shape[0] for c in cores] + [cores[-1].shape[-1]]
    bond_arr = (ctypes.c_int64 * (n + 1))(*bonds)
    ptr_arr = (ctypes.c_void_p * n)(*[c.data_ptr() for c in cores])
    ch = TnChain()
    ch.n = n
    ch.d = cores[0].shape[1]
    ch.bond = ctypes.cast(bond_arr, ctypes.POINTER(ctypes.c_int64))
    ch.cores = ctypes.cast(ptr_arr, ctypes.POINTER(ctypes.c_void_p))
    return ch, (bond_arr, ptr_arr, cores)


def mps_classify(cores, label_site: int, pixels: torch.Tensor, prec: str = "fp32", ckpt_every: int = 1,
                 workspace: torch.Tensor | None = None, stream=None):
    """(ftilde [B, L] float32, log_scale [B] float64, workspace): scores = ftilde * exp(log_scale)."""
    lib = load()
    L = cores[label_site].shape[2]
    B = pixels.shape[0]
    if pixels.dtype != torch.float32 or not pixels.is_contiguous():
        raise TypeError("pixels must be a contiguous float32 CUDA tensor [batch, n]")
    ch, keep = chain_desc_classifier(cores, label_site)
    if workspace is None:
        workspace = classifier_workspace(cores, label_site, L, B, ckpt_every)
    ft = torch.empty((B, L), dtype=torch.float32, device=pixels.device)
    lam = torch.empty((B,), dtype=torch.float64, device=pixels.device)
    _check(lib.tn_mps_classify(ctypes.byref(ch), label_site, L, ctypes.c_void_p(pixels.data_ptr()), B, PREC[prec],
                               ckpt_every, ctypes.c_void_p(ft.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                               ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream(stream)),
           "tn_mps_classify")
    return ft, lam, workspace


def mps_classify_backward(cores, label_site: int, pixels: torch.Tensor, dftilde: torch.Tensor,
                          workspace: torch.Tensor, prec: str = "fp32", ckpt_every: int = 1, stream=None):
    """Core gradients (list shaped like cores) from dLoss/dftilde; needs the forward's workspace."""
    lib = load()
    L = cores[label_site].shape[2]
    B = pixels.shape[0]
    ch, keep = chain_desc_classifier(cores, label_site)
    dft = dftilde.contiguous().float()
    grads = [torch.empty_like(c) for c in cores]
    table = (ctypes.c_void_p * len(grads))(*[g.data_ptr() for g in grads])
    _check(lib.tn_mps_classify_backward(ctypes.byref(ch), label_site, L, ctypes.c_void_p(pixels.data_ptr()), B,
                                        PREC[prec], ckpt_every, ctypes.c_void_p(dft.data_ptr()), table,
                                        ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream(stream)),
           "tn_mps_classify_backward")
    return grads


def _separate_chains(mps_list):
    arr = (TnChain * len(mps_list))()
    keep = []
    for l, cores in enumerate(mps_list):
        ch, k = chain_desc_classifier(cores, len(cores) // 2)
        arr[l] = ch
        keep.append(k)
    return arr, keep


def classifier_separate_workspace(mps_list, batch: int, ckpt_every: int) -> torch.Tensor:
    lib = load()
    arr, keep = _separate_chains(mps_list)
    nbytes = lib.tn_mps_classify_separate_workspace_bytes(arr, len(mps_list), batch, ckpt_every)
    if nbytes == 0:
        raise TnError(1, "tn_mps_classify_separate_workspace_bytes")
    return _workspace(nbytes, mps_list[0][0].device)


def mps_classify_separate(mps_list, pixels: torch.Tensor, prec: str = "fp32", ckpt_every: int = 1,
                          workspace: torch.Tensor | None = None, stream=None):
    """One MPS per label (tn_mps_classify_separate): (ftilde [B, L] float32,
    log_scale [B] float64, workspace), scores = ftilde * exp(log_scale)."""
    lib = load()
    B, L = pixels.shape[0], len(mps_list)
    if pixels.dtype != torch.float32 or not pixels.is_contiguous():
        raise TypeError("pixels must be a contiguous float32 CUDA tensor [batch, n]")
    arr, keep = _separate_chains(mps_list)
    if workspace is None:
        workspace = classifier_separate_workspace(mps_list, B, ckpt_every)
    ft = torch.empty((B, L), dtype=torch.float32, device=pixels.device)
    lam = torch.empty((B,), dtype=torch.float64, device=pixels.device)
    _check(lib.tn_mps_classify_separate(arr, L, ctypes.c_void_p(pixels.data_ptr()), B, PREC[prec], ckpt_every,
                                        ctypes.c_void_p(ft.data_ptr()), ctypes.c_void_p(lam.data_ptr()),
                                        ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream(stream)),
           "tn_mps_classify_separate")
    return ft, lam, workspace


def mps_classify_separate_backward(mps_list, pixels: torch.Tensor, dftilde: torch.Tensor, workspace: torch.Tensor,
                                   prec: str = "fp32", ckpt_every: int = 1, stream=None):
    """Core gradients of every MPS (a list per MPS, shaped like its cores) from
    dLoss/dftilde [B, L]; needs the forward's workspace and ckpt_every."""
    lib = load()
    B, L = pixels.shape[0], len(mps_list)
    arr, keep = _separate_chains(mps_list)
    dft = dftilde.contiguous().float()
    grads = [[torch.empty_like(c) for c in cores] for cores in mps_list]
    flat = [g for gl in grads for g in gl]
    table = (ctypes.c_void_p * len(flat))(*[g.data_ptr() for g in flat])
    _check(lib.tn_mps_classify_separate_backward(arr, L, ctypes.c_void_p(pixels.data_ptr()), B, PREC[prec],
                                                 ckpt_every, ctypes.c_void_p(dft.data_ptr()), table,
                                                 ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                                 _stream(stream)), "tn_mps_classify_separate_backward")
    return grads


def mps_classify_loss(ftilde: torch.Tensor, labels: torch.Tensor, stream=None):
    """(loss float64 scalar tensor, dLoss/dftilde) of mean CE(softmax(f/||f||), y) (tn_mps_classify_loss)."""
    lib = load()
    B, L = ftilde.shape
    ft = ftilde.contiguous()
    y = labels.to(torch.int64).contiguous()
    loss = torch.empty((), dtype=torch.float64, device=ft.device)
    dft = torch.empty_like(ft)
    _check(lib.tn_mps_classify_loss(ctypes.c_void_p(ft.data_ptr()), ctypes.c_void_p(y.data_ptr()), B, L,
                                    ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(dft.data_ptr()),
                                    _stream(stream)), "tn_mps_classify_loss")
    return loss, dft


class MPSClassifierFn(torch.autograd.Function):
    """ftilde, log_scale = MPSClassifierFn.apply(pixels, label_site, prec, ckpt_every, *cores).

    The backward is the library's hand-written adjoint (tn_mps_classify_backward)
    with checkpointed sweep vectors. log_scale is returned without a gradient:
    losses must depend on the scores only through f / ||f|| (as the
    normalised cross-entropy of the classifier does)."""

    @staticmethod
    def forward(ctx, pixels, label_site, prec, ckpt_every, *cores):
        ft, lam, ws = mps_classify(list(cores), label_site, pixels, prec=prec, ckpt_every=ckpt_every)
        ctx.save_for_backward(pixels, *cores)
        ctx.ws = ws
        ctx.meta = (label_site, prec, ckpt_every)
        ctx.mark_non_differentiable(lam)
        return ft, lam

    @staticmethod
    def backward(ctx, dft, dlam):
        pixels, *cores = ctx.saved_tensors
        label_site, prec, ckpt_every = ctx.meta
        grads = mps_classify_backward(cores, label_site, pixels, dft, ctx.ws, prec=prec, ckpt_every=ckpt_every)
        ctx.ws = None
        return (None, None, None, None, *grads)
