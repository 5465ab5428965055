"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps the
JSON-line contract: one line with the metric, the unit and the configuration
of the GPU arm, `impl: reference`, a `cpu_baseline` describing this run and an
`e2e` entry with no host-device traffic.  CPU only (small workload)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=600, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out
    return json.loads(lines[0])


def test_reference_arm_json_line():
    import bench
    d = _run("--impl", "reference", "--workload", "small", "--steps", "2", "--warmup", "3")
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    for key in ("value", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling", "vs_baseline",
                "dtype", "data", "config"):
        assert key in d, key
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"] == "small"
    # value: the full iteration's rate extrapolated from the sample; ms_per_step: the
    # sample's measured wall time (so K steps fit in the run's own clock)
    assert d["value"] > 0 and abs(d["value"] * d["ms_per_full_iteration"] / 1000.0 - 1.0) < 1e-6
    assert 0 < d["ms_per_step"] * d["steps"] <= 1000.0 * d["wall_s"] * 1.001
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"] and cb["cores"] >= 1
    assert cb["sample"]
    st = cb["single_thread"]  # one BLAS thread (null only where no OpenBLAS is loaded)
    assert st is None or (st["cores"] == 1 and st["value"] > 0)
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_batch_tile_spec():
    """--batch-tile pins one tile for both half-steps or one per half-step."""
    import bench
    assert bench.parse_batch_tile("192,3,2") == [(-1, (192, 3, 2))]
    assert bench.parse_batch_tile("256,3,2,2/192,3,2,1") == [(0, (256, 3, 2, 2)), (1, (192, 3, 2, 1))]
    for bad in ("192,3", "1,2,3,4,5", "1,2,3/1,2,3/1,2,3", "a,b,c"):
        with pytest.raises(ValueError):
            bench.parse_batch_tile(bad)
