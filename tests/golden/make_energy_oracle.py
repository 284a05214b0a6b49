"""Writes tests/golden/energy_oracle.txt: FP64 oracle values of the transverse-
field Ising energy <psi|H|psi> and norm <psi|psi> (oracle.mpo_expect and
oracle.mps_inner) for left-canonical MPS at the large bond dimensions of the
energy workload, where the oracle's nested loops take minutes per chain
(too long to rerun inside a GPU test).

Cases (open chain, d = 2, J = h = 1, bonds D_i = min(chi, 2^i, 2^(N-i))):
  * chi = 256, N = 100, seed 5: the whole workload chain;
  * chi = 512, N = 38 and chi = 1024, N = 40, seed 5: the deterministic subset
    of the N = 100 chains, 20 sites at the full bond dimension between the two
    ramps (the same per-site shapes as the N = 100 chain);
  * the first four states of the 64-MPS batch (bonds from uneven_chis(64, 50),
    seeds 500 + k), N = 100.

Inputs come from paper_1905_01330_gb300.synth (seeded SplitMix64 normals and a
float64 QR rounded to float32 once). Each line also records a fingerprint of
those float32 cores (sum and sum of squares in float64), so a test can check
that its regenerated inputs are the same ones up to the last-bit rounding
differences a host's LAPACK may introduce. Only oracle/ computes the values.

  python tests/golden/make_energy_oracle.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1905_01330_gb300 import synth  # noqa: E402


def cases():
    out = [("chain", 256, 100, 5), ("chain", 512, 38, 5), ("chain", 1024, 40, 5)]
    chis = synth.uneven_chis(64, seed=50)
    for k in range(4):
        out.append(("batch%d" % k, chis[k], 100, 500 + k))
    return out


def fingerprint(cores):
    s = sum(float(np.sum(c, dtype=np.float64)) for c in cores)
    q = sum(float(np.sum(c.astype(np.float64) ** 2)) for c in cores)
    return s, q


def main():
    path = os.path.join(HERE, "energy_oracle.txt")
    lines = ["# FP64 oracle (oracle.mpo_expect, oracle.mps_inner) of the TFIM energy of",
             "# left-canonical MPS; written by make_energy_oracle.py (see its docstring).",
             "# key chi N seed energy_value energy_log_scale norm_value norm_log_scale core_sum core_sumsq"]
    for name, chi, n, seed in cases():
        t0 = time.time()
        cores = synth.left_canonical_mps(n, 2, chi, seed=seed)
        W = synth.tfim_mpo(n)
        e, le = oracle.mpo_expect(cores, W)
        v, lv = oracle.mps_inner(cores, cores)
        s, q = fingerprint(cores)
        key = "%s_chi%d_n%d" % (name, chi, n)
        lines.append("%s %d %d %d %.17g %.17g %.17g %.17g %.17g %.17g" % (key, chi, n, seed, e, le, v, lv, s, q))
        print(lines[-1], "(%.0f s)" % (time.time() - t0), flush=True)
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
