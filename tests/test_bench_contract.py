"""The benchmark's reference arm (the CPU oracle timed on the host's cores) prints one JSON line
with the fields of the benchmark contract, and the serving stream's request generator behaves;
neither needs a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=900, check=True)
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in d, key
    assert d["unit"] == "GB/s" and d["value"] > 0 and d["steps"] == 1
    assert d["warmup"] >= 3  # at least three warm-up steps, whatever is asked
    assert d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["config"]["n"] == 6000000 and d["config"]["nnz"] == 29880000
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "GB/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_request_stream_preload_and_order():
    """The serving stream's generator: with preload every request exists before the first
    get (no waits counted), requests come back in order with the cell counts of the stream's
    sizes, the streamed form gives the same requests, and several threads building the box
    assembler at once do not collide."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    sizes = np.array([1.2e4, 2.5e4, 1.0e4, 1.8e4])
    pre = bench.RequestStream(sizes, 4, preload=True)
    got = [pre.get(i) for i in range(len(sizes))]
    pre.close()
    assert pre.wait_s == 0.0
    assert [g[0] for g in got] == list(range(len(sizes)))
    for g, c in zip(got, sizes):
        assert abs(g[1] - c) / c < 0.2  # a box of about the target cell count
    st = bench.RequestStream(sizes, 2, ahead=2)
    for i in range(len(sizes)):
        r = st.get(i)
        assert r[1] == got[i][1] and np.array_equal(r[3], got[i][3])
        assert np.array_equal(r[5], got[i][5])
    st.close()
    assert bench.preload_fits(np.array([1e4] * 4))
    assert not bench.preload_fits(np.array([1e15]))
