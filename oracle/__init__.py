"""FP64 CPU oracle for the tensor-network contraction path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
use this package. The GPU library neither imports nor links it, and the two
share no code; they share only the seeded inputs of
``paper_1905_01330_gb300.synth``.

The arithmetic lives in ``oracle.c`` (plain nested loops in float64, OpenMP
over independent outputs); this module builds it with gcc and marshals numpy
arrays through ctypes. Three modules build on it: ``split.py`` (node
splitting, its decomposition step numpy's LAPACK SVD), ``ncon.py`` (ncon over
tensordot and trace) and ``classifier_separate.py`` (one MPS per label over
the classifier sweep).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)
_dpp = ctypes.POINTER(_dp)


def build(force: bool = False) -> str:
    """Compiles oracle.c into _build/liboracle.so (gcc, -O2, OpenMP)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= max(
            os.path.getmtime(src), os.path.getmtime(hdr)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.or_tensordot.argtypes = [_dp, ctypes.c_int, _i64p, _ip, _dp, ctypes.c_int, _i64p, _ip,
                                   ctypes.c_int, _dp]
        L.or_trace.argtypes = [_dp, ctypes.c_int, _i64p, ctypes.c_int, ctypes.c_int, _dp]
        L.or_mps_inner.argtypes = [ctypes.c_int, ctypes.c_int, _i64p, _dpp, _i64p, _dpp, _dp, _dp]
        L.or_mps_state.argtypes = [ctypes.c_int, ctypes.c_int, _i64p, _dpp, _dp]
        L.or_mpo_expect.argtypes = [ctypes.c_int, ctypes.c_int, _i64p, _dpp, _i64p, _dpp, _dp, _dp]
        L.or_tfim_energy_dense.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp]
        L.or_tfim_energy_dense.restype = ctypes.c_double
        L.or_classify.argtypes = [ctypes.c_int, _i64p, _dpp, ctypes.c_int, ctypes.c_int, _dp,
                                  ctypes.c_int, _dp, _dp]
        L.or_classify_grad.argtypes = [ctypes.c_int, _i64p, _dpp, ctypes.c_int, ctypes.c_int, _dp,
                                       ctypes.c_int, _i64p, _dp, _dpp]
        L.or_classify_loss.argtypes = [ctypes.c_int, _i64p, _dpp, ctypes.c_int, ctypes.c_int, _dp,
                                       ctypes.c_int, _i64p, _dp]
    return _lib


def _f64(a) -> np.ndarray:
    return np.array(a, dtype=np.float64, order="C", copy=True)  # keeps rank 0


def _ptr(a: np.ndarray, t=_dp):
    return a.ctypes.data_as(t)


def _i64(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.int64))


def _i32(v) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32))


def _ptrs(arrs):
    return (_dp * len(arrs))(*[_ptr(a) for a in arrs])


def tensordot(A, legsA, B, legsB) -> np.ndarray:
    """C[free A legs, free B legs] = sum over shared legs (legsA[j] <-> legsB[j])."""
    A, B = _f64(A), _f64(B)
    la, lb = list(legsA), list(legsB)
    if len(la) != len(lb):
        raise ValueError("legsA and legsB differ in length")
    shape = [A.shape[p] for p in range(A.ndim) if p not in la] + \
            [B.shape[p] for p in range(B.ndim) if p not in lb]
    C = np.zeros(shape, dtype=np.float64)
    sha, shb = _i64(A.shape if A.ndim else [1]), _i64(B.shape if B.ndim else [1])
    rc = lib().or_tensordot(_ptr(A), A.ndim, _ptr(sha, _i64p), _ptr(_i32(la or [0]), _ip),
                            _ptr(B), B.ndim, _ptr(shb, _i64p), _ptr(_i32(lb or [0]), _ip),
                            len(la), _ptr(C))
    if rc != 0:
        raise ValueError("invalid contraction")
    return C


def trace(A, l1: int, l2: int) -> np.ndarray:
    A = _f64(A)
    shape = [A.shape[p] for p in range(A.ndim) if p not in (l1, l2)]
    out = np.zeros(shape, dtype=np.float64)
    rc = lib().or_trace(_ptr(A), A.ndim, _ptr(_i64(A.shape), _i64p), l1, l2, _ptr(out))
    if rc != 0:
        raise ValueError("invalid trace")
    return out


def _bonds(cores):
    return _i64([c.shape[0] for c in cores] + [cores[-1].shape[-1]])


def mps_inner(bra, ket):
    """(value, log_scale) with <bra|ket> = value * exp(log_scale)."""
    bra = [_f64(c) for c in bra]
    ket = [_f64(c) for c in ket]
    v, lg = ctypes.c_double(), ctypes.c_double()
    bb, bk = _bonds(bra), _bonds(ket)
    rc = lib().or_mps_inner(len(bra), bra[0].shape[1], _ptr(bb, _i64p), _ptrs(bra),
                            _ptr(bk, _i64p), _ptrs(ket), ctypes.byref(v), ctypes.byref(lg))
    if rc != 0:
        raise ValueError("invalid MPS")
    return v.value, lg.value


def mps_state(cores) -> np.ndarray:
    cores = [_f64(c) for c in cores]
    d = cores[0].shape[1]
    psi = np.zeros(d ** len(cores), dtype=np.float64)
    rc = lib().or_mps_state(len(cores), d, _ptr(_bonds(cores), _i64p), _ptrs(cores), _ptr(psi))
    if rc != 0:
        raise ValueError("invalid MPS")
    return psi


def mpo_expect(cores, W):
    """(value, log_scale) with <psi|H|psi> = value * exp(log_scale)."""
    cores = [_f64(c) for c in cores]
    W = [_f64(w) for w in W]
    wb = _i64([w.shape[0] for w in W] + [W[-1].shape[1]])
    v, lg = ctypes.c_double(), ctypes.c_double()
    rc = lib().or_mpo_expect(len(cores), cores[0].shape[1], _ptr(_bonds(cores), _i64p), _ptrs(cores),
                             _ptr(wb, _i64p), _ptrs(W), ctypes.byref(v), ctypes.byref(lg))
    if rc != 0:
        raise ValueError("invalid MPS/MPO")
    return v.value, lg.value


def tfim_energy_dense(n: int, J: float, h: float, psi) -> float:
    psi = _f64(psi)
    return lib().or_tfim_energy_dense(n, J, h, _ptr(psi))


def _cls_bonds(cores, label_site):
    return _i64([c.shape[0] for c in cores] + [cores[-1].shape[-1]])


def classify(cores, label_site: int, pixels):
    """(ftilde [B, L], lam [B]) with scores = ftilde * exp(lam[:, None])."""
    cores = [_f64(c) for c in cores]
    px = _f64(pixels)
    B, n = px.shape
    L = cores[label_site].shape[2]
    ft = np.zeros((B, L))
    lam = np.zeros(B)
    rc = lib().or_classify(n, _ptr(_cls_bonds(cores, label_site), _i64p), _ptrs(cores), label_site, L,
                           _ptr(px), B, _ptr(ft), _ptr(lam))
    if rc != 0:
        raise ValueError("invalid classifier")
    return ft, lam


def classify_loss(cores, label_site: int, pixels, labels) -> float:
    cores = [_f64(c) for c in cores]
    px = _f64(pixels)
    B, n = px.shape
    L = cores[label_site].shape[2]
    y = _i64(labels)
    out = ctypes.c_double()
    rc = lib().or_classify_loss(n, _ptr(_cls_bonds(cores, label_site), _i64p), _ptrs(cores), label_site,
                                L, _ptr(px), B, _ptr(y, _i64p), ctypes.byref(out))
    if rc != 0:
        raise ValueError("invalid classifier")
    return out.value


def classify_grad(cores, label_site: int, pixels, labels):
    """(loss, [dcore per site]) for loss = mean_b CE(softmax(f_b/||f_b||), y_b)."""
    cores = [_f64(c) for c in cores]
    px = _f64(pixels)
    B, n = px.shape
    L = cores[label_site].shape[2]
    y = _i64(labels)
    d = [np.zeros_like(c) for c in cores]
    out = ctypes.c_double()
    rc = lib().or_classify_grad(n, _ptr(_cls_bonds(cores, label_site), _i64p), _ptrs(cores), label_site,
                                L, _ptr(px), B, _ptr(y, _i64p), ctypes.byref(out), _ptrs(d))
    if rc != 0:
        raise ValueError("invalid classifier")
    return out.value, d


from .split import matrix_view, split_node, svd, truncation_count  # noqa: E402  (node splitting, numpy)
from .ncon import ncon  # noqa: E402  (ncon over tensordot / trace)
from .classifier_separate import classify_separate, classify_separate_loss  # noqa: E402
