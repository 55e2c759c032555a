"""Host-side logic of bench.py that the GPU numbers rest on: the whole-job rate, the traffic
lookup keyed by the kernel's source hash, the clock record, and the argument defaults."""
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_whole_job_rate_is_weak_scaling(bench):
    # 4 ranks each doing 1e6 units, slowest rank 2 ms -> 2e9 units/s for the job
    assert bench.whole_job_rate(1e6, 4, 2.0) == pytest.approx(2e9)
    assert bench.reduce_over_ranks(3.5, None) == 3.5


def test_traffic_is_dropped_when_the_kernel_source_changes(bench):
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        d = json.load(f)
    for kernel, e in d.items():
        current = e["source_hash"] == bench.source_hash(*e["files"])
        assert bench.load_traffic(kernel, e["files"]) == (e["bytes_per_launch"] if current else None), kernel
    # a different source: same kernel name, other files -> no traffic figure
    k, e = next(iter(d.items()))
    assert bench.load_traffic(k, ["bench.py"]) is None
    assert bench.load_traffic("no_such_kernel", e["files"]) is None


def test_committed_traffic_matches_the_current_kernels(bench):
    """The DRAM traffic the bench reports was captured on the kernel sources in the tree: a kernel
    edited without a new capture fails here instead of reporting traffic: null."""
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        d = json.load(f)
    for kernel, e in d.items():
        assert e["source_hash"] == bench.source_hash(*e["files"]), kernel
        assert os.path.exists(os.path.join(ROOT, e["profile"])), kernel


def test_clock_record_flags_throttling(bench, tmp_path):
    cs = bench.ClockSampler(0)
    path = tmp_path / "clocks.csv"
    rows = ["0, 2070, 2070, 700.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 1500, 2070, 950.0, 0x8, Active, Not Active, Not Active, Not Active"]
    path.write_text("\n".join(rows) + "\n")

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs.proc, cs.path = Done(), str(path)
    rec = cs.stop()
    assert rec["samples"] == 3 and rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert rec["sm_mhz"] == 2070.0 and rec["power_w_max"] == 950.0


def test_defaults_are_one_gpu_and_a_short_run(bench):
    a = bench.parse_args([])
    assert a.gpus == 1 and a.warmup >= 3 and a.workload == "glyphs" and a.impl == "shm"
    assert a.dtype_id == 0 and a.layout_id == 0
