"""Host logic without a GPU: the chunking of the staged plan (tn_chunk_bounds), the bench's
JSON line of the reference arm (the FP64 oracle on the host cores) and its clock record."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_1905_01330_gb300 import build
    return build.build()


@pytest.mark.parametrize("weights,chunks,bounds", [
    ([1] * 8, 4, [0, 2, 4, 6, 8]),
    ([1] * 7, 3, [0, 2, 5, 7]),
    ([10, 1, 1, 1], 3, [0, 1, 2, 4]),       # a heavy first item ends a run by itself
    ([1, 1, 1, 10], 3, [0, 3, 4]),          # a heavy last item: fewer runs
    ([5.68e6, 8.2e5] + [4e4] * 20, 3, [0, 1, 2, 22]),   # the staged-plan GPU test's specs
    ([5], 8, [0, 1]),
    ([], 4, [0, 0]),
])
def test_chunk_bounds(built, weights, chunks, bounds):
    from paper_1905_01330_gb300.tn import chunk_bounds
    got = chunk_bounds(weights, chunks)  # tn_chunk_bounds, host code of libtn.so
    assert got == bounds
    assert all(a < b for a, b in zip(got, got[1:])) or not weights


def test_chunk_bounds_properties_on_random_weights(built):
    """On random weights (zeros and heavy items included): the bounds start at
    0, end at n, rise strictly, give at most `chunks` runs, and no run of more
    than one item exceeds the ideal share by more than twice the largest item
    (each cut lands within one item of its ideal place)."""
    import random
    from paper_1905_01330_gb300.tn import chunk_bounds
    rnd = random.Random(5)
    for _ in range(300):
        n = rnd.randint(1, 60)
        w = [rnd.choice([0.0, rnd.random(), 10 * rnd.random(), 1000 * rnd.random()]) for _ in range(n)]
        chunks = rnd.randint(1, 12)
        b = chunk_bounds(w, chunks)
        assert b[0] == 0 and b[-1] == n
        assert all(x < y for x, y in zip(b, b[1:]))
        assert len(b) - 1 <= chunks
        share, big = sum(w) / chunks, max(w)
        for lo, hi in zip(b, b[1:]):
            if hi - lo > 1:
                assert sum(w[lo:hi]) <= share + 2 * big + 1e-9, (w, chunks, b)


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["dtype"] == "f64"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_clock_sampler_keeps_samples_of_the_timed_region(tmp_path, monkeypatch):
    """The bench's clock record: samples taken between start() and stop()
    only, with the throttle reasons parsed from nvidia-smi's CSV. A stand-in
    nvidia-smi on PATH prints one CSV line every 50 ms."""
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\nwhile true; do\n"
                    "  echo '0, 2070, 2070, 512.3, 0x4, Not Active, Not Active, Not Active, Active'\n"
                    "  sleep 0.05\ndone\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    sys.path.insert(0, ROOT)
    try:
        import bench
    finally:
        sys.path.remove(ROOT)
    import time
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.4)
    c = s.stop()
    assert c is not None
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"]
    assert 3 <= c["samples"] <= 12
    # without nvidia-smi there is no record (and no error)
    monkeypatch.setenv("PATH", str(tmp_path / "none"))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop() is None
