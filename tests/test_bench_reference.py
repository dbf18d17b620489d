"""The benchmark's reference arm (the serial oracle on the host) prints the contract's JSON line,
checked on a small grid so that it runs in a second on CPU; and the bench's host-side helpers."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--side", "16",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == "RCM GTEPS" and d["unit"] == "GTEPS"
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["n"] == 16 ** 3


def test_bench_launch_options_and_traffic_record():
    """--launch parses key=value pairs or JSON into engine options; the recorded DRAM traffic is
    reported only for the kernel sources it was captured from."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_1610_08128_gb300 import rcm

    assert bench.parse_launch("executor=1,narrow_threshold=512") == {"executor": 1, "narrow_threshold": 512}
    assert bench.parse_launch('{"expand_mode": 3}') == {"expand_mode": 3}
    assert bench.parse_launch("") == {}
    a, b = rcm.rcm_options(), rcm.rcm_options()
    a.narrow_threshold, a.expand_mode, a.nnz = 512, 3, 99
    bench.ctypes_copy(a, b)
    assert (b.narrow_threshold, b.expand_mode, b.nnz) == (512, 3, 99)
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["k_rcm_single"]["grid192"]
    assert rec["dram_bytes_per_launch"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    if rec["sources"] == bench.kernel_sources_hash():
        assert bench.recorded_traffic("k_rcm_single", "grid192") == rec["dram_bytes_per_launch"]
    assert bench.recorded_traffic("k_rcm_single", "grid7") is None


def test_fifo_replay_of_the_served_baseline():
    """The FIFO baseline of the served line: the trace replayed in real time, one request at a time
    in arrival order (a request waits for its arrival and for the one before it)."""
    import time

    sys.path.insert(0, ROOT)
    import bench

    starts = []

    def call(gi):
        starts.append((time.perf_counter(), gi))
        time.sleep(0.05)

    t0 = time.perf_counter()
    rate, lat = bench.fifo_replay([0.0, 0.01, 0.02, 0.3], [3, 1, 2, 0], call)
    assert [gi for _, gi in starts] == [3, 1, 2, 0]
    rel = [t - t0 for t, _ in starts]
    # the first three queue behind each other; the last waits for its arrival (the server is idle)
    assert rel[1] >= 0.05 and rel[2] >= 0.10 and rel[3] >= 0.3
    assert lat[0] >= 0.05 and lat[2] >= 0.13 and 0.05 <= lat[3] < 0.2
    assert abs(rate - 4 / (rel[3] + 0.05)) < 0.5
    assert bench.fifo_replay([], [], call) == (0.0, [])
    assert bench.pct([3.0, 1.0, 2.0], 0.5) == 2.0 and bench.pct([], 0.5) is None
