"""Energy sweeps against the FP64 oracle at the workload's bond dimensions.

The oracle's values (tests/golden/energy_oracle.txt, written by
tests/golden/make_energy_oracle.py, which calls only oracle/) cover the
transverse-field Ising energy of left-canonical MPS at chi = 256 (the whole
N = 100 chain), chi = 512 and 1024 on the deterministic subset chains of 20
full-bond sites (N = 38 and 40: the same per-site contraction shapes as the
N = 100 chain), and the first four states of the 64-MPS batch (N = 100, bonds
64, 512, 416, 416). The inputs are regenerated here from the same seeds; a
fingerprint of the float32 cores checks that they are the stored ones (up to
the last-bit differences another host's LAPACK may leave in a few entries).

<psi|H|psi> is a sum of terms of both signs, so its error is bounded
relative to ||H|| <psi|psi>, ||H|| <= J (N - 1) + h N, with the per-sweep
tolerances of the other sweep tests: float32 1e-5; split BF16x3
2 * 2^-16 * sqrt(c); bf16 2 * 2^-8 * sqrt(c), c = 2N contractions.
<psi|psi> is a sum of squares: the term the split drops (lo * lo, at most
2^-18 of a product) and the rounding of each operand enter it as quadratic
forms of one sign, so those errors add up over the c contractions instead of
walking: its bound adds c * 2^-18 (BF16x3) or c * 2^-16 (bf16) to the walk.
"""
import math
import os

import numpy as np
import pytest

from paper_1905_01330_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
UNIT = {"fp32": None, "bf16x3": 2.0 ** -16, "bf16": 2.0 ** -8}


def tol(prec, n):
    return 1e-5 if prec == "fp32" else 2.0 * UNIT[prec] * math.sqrt(2 * n)


def norm_tol(prec, n):
    bias = {"fp32": 0.0, "bf16x3": 2.0 ** -18, "bf16": 2.0 ** -16}[prec]
    return tol(prec, n) + 2 * n * bias


def golden():
    rows = {}
    with open(os.path.join(HERE, "golden", "energy_oracle.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, chi, n, seed, e, le, v, lv, s, q = line.split()
            rows[k] = dict(chi=int(chi), n=int(n), seed=int(seed), energy=float(e) * math.exp(float(le)),
                           norm=float(v) * math.exp(float(lv)), sum=float(s), sumsq=float(q))
    return rows


@pytest.fixture(scope="module")
def tn():
    from paper_1905_01330_gb300 import build, tn as tnmod
    build.build()
    tnmod.load()
    return tnmod


def inputs(row):
    cores = synth.left_canonical_mps(row["n"], 2, row["chi"], seed=row["seed"])
    s = sum(float(np.sum(c, dtype=np.float64)) for c in cores)
    q = sum(float(np.sum(c.astype(np.float64) ** 2)) for c in cores)
    assert abs(s - row["sum"]) <= 1e-6 * max(1.0, abs(row["sum"])), "regenerated cores differ"
    assert abs(q - row["sumsq"]) <= 1e-9 * row["sumsq"], "regenerated cores differ"
    return [torch.from_numpy(c).cuda() for c in cores]


def check(r, row, prec, what):
    r = np.asarray(r, dtype=np.float64)
    n = row["n"]
    h_norm = 1.0 * (n - 1) + 1.0 * n
    energy, norm = r[0] * math.exp(r[1]), r[2] * math.exp(r[3])
    assert abs(energy - row["energy"]) <= tol(prec, n) * h_norm * row["norm"], (what, prec, energy, row["energy"])
    assert abs(norm - row["norm"]) <= norm_tol(prec, n) * row["norm"], (what, prec, norm, row["norm"])


@pytest.mark.parametrize("key", ["chain_chi256_n100", "chain_chi512_n38", "chain_chi1024_n40"])
def test_energy_against_oracle_at_workload_bonds(tn, key):
    row = golden()[key]
    cores = inputs(row)
    W = [torch.from_numpy(w).cuda() for w in synth.tfim_mpo(row["n"])]
    for prec in ("fp32", "bf16x3", "bf16"):
        r = tn.mps_expect(cores, W, prec=prec)
        assert tn.sync_status() == 0
        check(r.cpu().numpy(), row, prec, key)


def test_grouped_energy_against_oracle_batch_states(tn):
    g = golden()
    rows = [g[k] for k in sorted(g) if k.startswith("batch")]
    assert [r["chi"] for r in rows] == synth.uneven_chis(64, seed=50)[:4]
    states = [inputs(r) for r in rows]
    W = [torch.from_numpy(w).cuda() for w in synth.tfim_mpo(100)]
    for prec in ("fp32", "bf16x3", "bf16"):
        r = tn.mps_expect_grouped(states, W, prec=prec).cpu().numpy()
        assert tn.sync_status() == 0
        for k, row in enumerate(rows):
            check(r[k], row, prec, "batch%d" % k)
