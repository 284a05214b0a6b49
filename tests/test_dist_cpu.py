"""The multi-rank path on CPU: two gloo ranks through the bench's process-group
helpers (weak scaling, one all-reduce of the slowest time), and the reference
arm of bench.py launched with torch.distributed.run on two ranks (rank 0 alone
prints the line, the other exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    from paper_1905_01330_gb300 import dist as tndist
    tndist.init("gloo")
    r, w, local = tndist.env()
    ms = 10.0 + 5.0 * r                      # rank 1 is the slower one
    slowest = tndist.max_over_ranks(ms)
    tndist.barrier()
    value = tndist.weak_scaling_value(2.0e12, slowest, w)
    out[r] = (r, w, local, slowest, value, tndist.data_seed(2, r))
    tndist.finish()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    world, port = 2, free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r, (rr, w, local, slowest, value, seed) in res.items():
        assert (rr, w, local) == (r, 2, r)
        assert slowest == 15.0                          # max over ranks
        assert value == pytest.approx(2 * 2.0e12 / 15e-3)  # whole-job throughput, weak scaling
    assert res[0][5] != res[1][5]                       # each rank draws its own operands


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    from paper_1905_01330_gb300 import dist as tndist
    if "RANK" not in os.environ:
        assert tndist.env() == (0, 1, 0)
    assert tndist.max_over_ranks(3.5) == 3.5


def test_reference_arm_under_torchrun_two_ranks():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1                               # rank 0 only
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
