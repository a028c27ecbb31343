"""bench.py's reference arm runs the oracle on the host cores, so its JSON
line can be checked without a GPU: one line with the contract's keys, the
same metric and workload names as the GPU arm, zero transfer bytes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "rmat10-exact-plain", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "BC GTEPS (sources*m/s)" and d["unit"] == "GTEPS"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 0 and d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "rmat10-exact-plain"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_bytes_models_follow_their_stated_formulas():
    """The two bytes models of the roofline, on made-up counters, equal the
    formulas the benchmark line states (so a reader can redo them by hand)."""
    sys.path.insert(0, ROOT)
    import bench
    E, I, O, D, R = 10, 100, 200, 1000, 50
    st = dict(frontier_entries=E, scanned_in_edges=I, scanned_out_edges=O, dag_pairs=D,
              reached_pairs=R, kernel_kind=2, mask_words=4)
    for b in (4, 8):
        assert bench.method_bytes_model(st, b) == 8 * E + 4 * (I + O) + 32 * (I + O) + \
            (16 + b) * D + (16 + b) * R
        assert bench.bytes_model(st, b) == 124 * E + 36 * (I + O) + (8 + b) * D + (16 + b) * R
    plain = dict(st, kernel_kind=1)
    assert bench.method_bytes_model(plain, 8) == 8 * (I + O) + 32 * D + 88 * E
    assert bench.bytes_model(plain, 8) == 92 * E + 8 * (I + O) + 16 * D


def test_traffic_reported_only_for_the_kernel_it_was_measured_on(monkeypatch):
    """roofline.traffic comes from the committed ncu summary only while its
    kernel hash matches the current kernel sources."""
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
        rec = json.load(fh)
    entry = rec["rmat20-sampled4096"]
    assert len(bench.kernel_source_sha()) == 16
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: entry["kernel_sha"])
    assert bench.ncu_traffic("rmat20-sampled4096") == entry["dram_bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
    assert bench.ncu_traffic("rmat20-sampled4096") is None
    assert bench.ncu_traffic("no-such-workload") is None
