"""Host-side logic of bench.py that the GPU numbers rest on: the whole-job rate, the traffic
lookup keyed by the kernel's source hash, the clock record, the argument defaults, and the event
ordering of the glyph field's end-to-end copy pipeline."""
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


class _Graph:
    """Stream-ordered operations with event dependencies, as the bench's pipeline issues them."""

    def __init__(self):
        self.ops, self.edges, self.last, self.records = [], {}, {}, {}
        self.current = None

    def add(self, stream, what):
        i = len(self.ops)
        self.ops.append((stream, what))
        self.edges[i] = set()
        if stream in self.last:
            self.edges[self.last[stream]].add(i)
        self.last[stream] = i
        return i

    def after(self, x, y):
        """True if op x is ordered after op y."""
        seen, todo = set(), [y]
        while todo:
            n = todo.pop()
            for m in self.edges[n]:
                if m == x:
                    return True
                if m not in seen:
                    seen.add(m)
                    todo.append(m)
        return False


def test_e2e_pipeline_orders_every_chunk_buffer(bench):
    """The glyph field's end-to-end step, replayed with recording streams and events over two
    steps: a chunk's bake and query follow its host-to-device copy; its outputs go back after its
    query; and in the next step its directions are overwritten only after the previous query read
    them, its outputs only after the previous device-to-host copy read them."""
    import contextlib
    g = _Graph()

    class Stream:
        def __init__(self, name):
            self.name = name

        def wait_event(self, ev):
            i = g.add(self.name, ("wait", ev.name))
            g.edges[g.records[(ev.name, ev.version)]].add(i)

    class Event:
        def __init__(self, name):
            self.name, self.version = name, 0

        def record(self, stream):
            self.version += 1
            g.records[(self.name, self.version)] = g.add(stream.name, ("record", self.name))

    class View:
        def __init__(self, name, lo, hi):
            self.name, self.lo, self.hi = name, lo, hi

        def copy_(self, src, non_blocking=False):
            g.add(g.current, ("copy", self.name, src.name, self.lo))

    class Tensor:
        def __init__(self, name):
            self.name = name

        def __getitem__(self, sl):
            return View(self.name, sl.start, sl.stop)

    class Cuda:
        @staticmethod
        @contextlib.contextmanager
        def stream(s):
            prev, g.current = g.current, s.name
            yield
            g.current = prev

    class Torch:
        cuda = Cuda

    class Lib:
        @staticmethod
        def build_lut(lut, src, ws=None, stream=None):
            g.add(stream.name, ("bake", lut))

        @staticmethod
        def query(lut, dirs, seg=None, out=None, stream=None):
            g.add(stream.name, ("query", lut))

    C = 4
    w = bench.GlyphField.__new__(bench.GlyphField)
    w.torch, w.S, w.per = Torch, Lib, 2
    w.e2e_h2d, w.e2e_d2h, w.e2e_streams = Stream("h2d"), Stream("d2h"), [Stream("kernels")]
    w.e2e_chunks = [(c, None, None, 3 * c, 3 * c + 3) for c in range(C)]
    w.e2e_ws = [None]
    w.dirs, w.dirs_host, w.coeffs, w.c_pinned = Tensor("dirs"), Tensor("dirs_host"), Tensor("coeffs"), Tensor("c_host")
    w.out = {k: Tensor("out_" + k) for k in ("R", "grad", "normal")}
    w.e2e_ev_in, w.e2e_ev_q, w.e2e_ev_out = ([Event(f"{n}{c}") for c in range(C)] for n in ("in", "q", "out"))
    w.e2e_used = [False] * C
    host_out = {k: Tensor("host_" + k) for k in ("R", "grad", "normal")}
    for _ in range(2):
        w.e2e_step_pipeline(host_out)

    def find(kind, step, match):
        """The step-th op of this kind whose fields match ({position: value})."""
        hits = [i for i, (s, what) in enumerate(g.ops) if what[0] == kind and
                all(what[j] == v for j, v in match.items())]
        return hits[step]

    for c in range(C):
        q0 = 3 * c * w.per
        for step in range(2):
            h2d = find("copy", step, {1: "dirs", 3: q0})
            bake, query = find("bake", step, {1: c}), find("query", step, {1: c})
            back = [find("copy", step, {1: "host_" + k, 3: q0}) for k in ("R", "grad", "normal")]
            assert g.after(bake, h2d) and g.after(query, bake)
            assert all(g.after(b, query) for b in back)
            if step == 1:
                assert g.after(h2d, find("query", 0, {1: c}))  # directions read by the last query
                assert all(g.after(query, find("copy", 0, {1: "host_" + k, 3: q0}))
                           for k in ("R", "grad", "normal"))  # outputs read by the last copy back
