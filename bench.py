#!/usr/bin/env python3
"""Benchmark of the Spherical Hermite Map hot path (arXiv 2602.20063) on one GB300 per rank.

Default workload (the configuration the headline metric is quoted on): a batched glyph field of
16,384 real-SH glyphs, L = 8, N = 32 per face (padded 34^2), 4,096 uniform query directions per
glyph (2^26 queries).  One step = the whole hot path over one batch: the SH -> table bake as one
[G x K] x [K x 4T] contraction, then the query (direction -> face/uv -> 2x2 fetch -> Hermite value
and chart gradient -> S^2 gradient -> normal) of all 2^26 directions.  The per-(N, L) SH basis is
a constant of the configuration and is prepared before timing.

Other workloads (``--workload``): planet (procedural fBm planet, N = 2048, 2^28 random queries),
impostors (512 bump objects of uneven N ray cast at 1920x1080), fit (fwd + bwd of 1,024 glyphs at
N = 64 against direct-SH targets), single (one L = 4 glyph at N = 10, 65,536 queries).

Prints ONE JSON line.  ``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload instead (rank 0 only; other ranks exit without work).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hermite value+grad queries/s, % of HBM roofline; fwd+bwd vs plain at fixed error"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}


# ----------------------------------------------------------------------------------- environment
def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    d = dict(FALLBACK_PEAKS)
    d["_source"] = "fallback"
    return d


def fp32_simt_peak_tflops(peaks, sms=152):
    # 128 FP32 lanes per SM x 2 flop per FMA x max SM clock
    return sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        loaded = sorted(sm)[len(sm) // 2:] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit()) if rows else None}


class KernelTimer:
    """CUDA events between launches on one stream; per-name totals over the timed steps."""

    def __init__(self, stream):
        import torch
        self.torch = torch
        self.stream = stream
        self.marks = []
        self.active = False

    def mark(self, name):
        if not self.active:
            return
        e = self.torch.cuda.Event(enable_timing=True)
        e.record(self.stream)
        self.marks.append((name, e))

    def totals(self):
        out = {}
        for (name, e0), (_, e1) in zip(self.marks[:-1], self.marks[1:]):
            if name == "_end":
                continue
            out.setdefault(name, [0.0, 0])
            out[name][0] += e0.elapsed_time(e1)
            out[name][1] += 1
        return out


def source_hash(*files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic(kernel, files):
    """DRAM bytes per launch from a committed ncu capture, if it was taken on the current source."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel)
    if not e or e.get("source_hash") != source_hash(*files):
        return None
    return e.get("bytes_per_launch")


# ----------------------------------------------------------------------------------- workloads
class GlyphField:
    name = "glyphs"
    unit = "queries/s"

    def __init__(self, args, rank):
        self.G, self.L, self.N, self.per = args.glyphs, 8, 32, args.per_glyph
        self.Q = self.G * self.per
        self.dtype, self.layout = args.dtype_id, args.layout_id
        self.seed = 20063 + 1 + 1000 * rank
        self.config = {"workload": f"glyph field: {self.G} real-SH glyphs, L=8, N=32 (+1 gutter), "
                                   f"{self.per} uniform queries per glyph ({self.Q} total), "
                                   f"{['f32', 'f16', 'bf16'][self.dtype]} {['texel', 'cell'][self.layout]} records; "
                                   "step = SH bake contraction + query",
                       "glyphs": self.G, "L": self.L, "N": self.N, "queries_per_step": self.Q,
                       "l2": "inputs larger than L2 (table 1.82 GB, directions 805 MB)"}

    def setup(self, S, torch):
        import shm_inputs as I
        dev = "cuda"
        self.S, self.torch = S, torch
        self.c_host = I.sh_coeffs(self.G, self.L, self.seed).astype(np.float32)
        self.coeffs = torch.from_numpy(self.c_host).to(dev)
        self.basis = S.sh_basis(self.N, self.L)
        self.lut = S.alloc_lut(self.G, self.N, self.dtype, self.layout)
        self.dirs = torch.empty((self.Q, 3), dtype=torch.float32, device=dev)
        self.dirs_host = torch.empty((self.Q, 3), dtype=torch.float32).pin_memory()
        for s0, d in I.directions_chunked(self.Q, self.seed + 7):
            self.dirs_host[s0:s0 + len(d)] = torch.from_numpy(d)
        self.dirs.copy_(self.dirs_host)
        self.seg = torch.from_numpy(I.query_glyphs_csr(self.G, self.per)).to(dev)
        self.out = {k: torch.empty(s, dtype=torch.float32, device=dev)
                    for k, s in (("R", (self.Q,)), ("grad", (self.Q, 3)), ("normal", (self.Q, 3)))}
        self.src = S.Source(kind=S.SHM_SRC_SH, L=self.L, coeffs=self.coeffs, basis=self.basis)
        self.launches_per_step = 2

    def step(self, timer):
        timer.mark("sh_build_gemm")
        self.S.build_lut(self.lut, self.src)
        timer.mark("query_fwd")
        self.S.query(self.lut, self.dirs, seg=self.seg, out=self.out)
        timer.mark("_end")

    def units_per_step(self):
        return self.Q

    def e2e_step(self, host_out):
        """Public API from pinned host buffers: H2D directions + coefficients, bake, query, D2H outputs."""
        self.dirs.copy_(self.dirs_host, non_blocking=True)
        self.coeffs.copy_(self.c_pinned, non_blocking=True)
        self.S.build_lut(self.lut, self.src)
        self.S.query(self.lut, self.dirs, seg=self.seg, out=self.out)
        for k in ("R", "grad", "normal"):
            host_out[k].copy_(self.out[k], non_blocking=True)

    def e2e_setup(self):
        torch = self.torch
        self.c_pinned = torch.from_numpy(self.c_host).pin_memory()
        host_out = {k: torch.empty(v.shape, dtype=torch.float32).pin_memory() for k, v in self.out.items()}
        h2d = self.dirs.numel() * 4 + self.coeffs.numel() * 4
        d2h = sum(v.numel() * 4 for v in self.out.values())
        return host_out, h2d, d2h

    def roofline_terms(self, peaks, kernel_ms, sms):
        T = 6 * (self.N + 2) ** 2
        rec = self.S.record_bytes(self.dtype, self.layout)
        lut_bytes = self.G * self.S.records_per_glyph(self.N, self.layout) * rec
        K = (self.L + 1) ** 2
        q_alg = lut_bytes + self.Q * (12 + 28)
        terms = {
            "query_fwd": {"bound": "hbm", "algorithmic": q_alg, "unit": "GB/s", "peak": peaks["hbm_gbs"],
                          "per_unit": f"{q_alg / self.Q:.1f} B/query = table bytes once ({lut_bytes / self.Q:.1f} B/q) "
                                      "+ 12 B direction + 28 B outputs (compulsory traffic)",
                          "files": ["paper_2602_20063_gb300/csrc/shm_query.cu",
                                    "paper_2602_20063_gb300/csrc/shm_device.cuh"]},
            "sh_build_gemm": {"bound": "alu", "algorithmic": 2.0 * self.G * K * 4 * T, "unit": "TFLOP/s",
                              "peak": fp32_simt_peak_tflops(peaks, sms),
                              "per_unit": f"2 K = {2 * K} flop per stored scalar, {4 * T} scalars per glyph",
                              "files": ["paper_2602_20063_gb300/csrc/shm_build.cu"]},
        }
        return terms

    def extras(self, S, torch, steps):
        """fwd+bwd vs fwd on the same queries, and 16-bit storage vs f32 (error and speed)."""
        ex = {}
        st = torch.cuda.current_stream()
        dl = S.like_lut(self.lut, dtype=S.SHM_F32, layout=S.SHM_LAYOUT_TEXEL, zero=True)
        g = torch.Generator(device="cuda").manual_seed(5)
        gR = torch.randn(self.Q, device="cuda", generator=g)
        gG = torch.randn((self.Q, 3), device="cuda", generator=g)
        gN = torch.randn((self.Q, 3), device="cuda", generator=g)

        def timeit(fn, n):
            for _ in range(2):
                fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(n):
                fn()
            e1.record(st)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / n

        n = max(3, min(steps, 10))
        fwd = timeit(lambda: S.query(self.lut, self.dirs, seg=self.seg, out=self.out), n)
        bwd = timeit(lambda: S.query_backward(self.lut, self.dirs, dl, gR=gR, ggrad=gG, gnormal=gN, seg=self.seg,
                                              want_ddirs=True), n)
        ex["fwd_bwd"] = {"fwd_ms": round(fwd, 4), "bwd_ms": round(bwd, 4), "fwd_plus_bwd_over_fwd": round((fwd + bwd) / fwd, 3),
                         "note": "backward = recompute + 4 float4 atomics per query into a float32 texel table + d/ddirs"}
        ref = {k: v.clone() for k, v in self.out.items()}
        for name, dt in (("bf16", S.SHM_BF16), ("f16", S.SHM_F16)):
            r0 = torch.full((self.G,), 0.7, dtype=torch.float32, device="cuda")
            L16 = S.like_lut(self.lut, dtype=dt, r0=r0)
            S.pack_lut(self.lut, L16)
            o16 = {k: torch.empty_like(v) for k, v in self.out.items()}
            ms = timeit(lambda: S.query(L16, self.dirs, seg=self.seg, out=o16), n)
            eR = float((o16["R"] - ref["R"]).abs().max() / ref["R"].abs().max())
            eG = float((o16["grad"] - ref["grad"]).abs().max() / ref["grad"].norm(dim=1).max())
            ex[name] = {"query_ms": round(ms, 4), "queries_per_s": self.Q / (ms * 1e-3),
                        "speedup_vs_f32": round(fwd / ms, 3),
                        "max_err_R_rel_vs_f32": eR, "max_err_grad_rel_vs_f32": eG,
                        "note": "value offset r0 = 0.7 per glyph; error vs the same queries on f32 storage"}
            del L16, o16
        del dl
        return ex

    # ---------------------------------------------------------------- oracle sample (CPU)
    def oracle_task_args(self, n_glyphs, start=0):
        return [("glyphs", g, self.c_host[g].astype(np.float64), self.N, self.L, self.per, self.seed + 7)
                for g in range(start, start + n_glyphs)]


def _oracle_glyph_task(args):
    """One glyph of the glyph-field workload on the oracle: FP64 bake + its queries."""
    kind, g, c, N, L, per, dseed = args
    import oracle as O
    import shm_inputs as I
    lut = O.bake_sh(N, L, c)
    pool, off, Ns = O.make_pool([lut])
    d = I.directions_range(g * per, per, dseed)
    O.query(pool, off, Ns, d, nthreads=1)
    return per


def oracle_sample(work, budget_s, procs):
    """Run the oracle on whole glyphs in a spawn pool until ~budget_s; returns (queries/s, sample)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        t0 = time.perf_counter()
        pool.map(_oracle_glyph_task, work.oracle_task_args(procs))  # calibrate (includes worker start)
        t1 = time.perf_counter()
        per_round = max(t1 - t0, 1e-3)
        rounds = max(1, int(budget_s / per_round))
        n = procs * rounds
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_glyph_task, work.oracle_task_args(n, start=procs)))
        dt = time.perf_counter() - t0
    return done / dt, f"{n} glyphs (FP64 bake of each + its {work.per} queries), {procs} processes, {dt:.1f} s"


WORKLOADS = {"glyphs": GlyphField}


# ----------------------------------------------------------------------------------- arms
def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    work = WORKLOADS[args.workload](args, 0)
    procs = os.cpu_count() or 1
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    times, units = [], []
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_glyph_task, work.oracle_task_args(procs))
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            u = sum(pool.map(_oracle_glyph_task, work.oracle_task_args(procs, start=procs * (k + 1))))
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                times.append(dt)
                units.append(u)
    value = sum(units) / sum(times)
    sample = f"each step: {procs} glyphs (FP64 bake + {work.per} queries each), {procs} processes"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": work.unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": work.config,
            "cpu_baseline": {"value": value, "unit": work.unit, "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": work.unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_gpu(args):
    rank, world, local = env_rank()
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    peaks = load_peaks()
    work = WORKLOADS[args.workload](args, rank)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # before the first GPU call, in spawned processes
        v, sample = oracle_sample(work, args.cpu_budget, os.cpu_count() or 1)
        cpu = {"value": v, "unit": work.unit, "cores": os.cpu_count() or 1, "kind": "oracle", "sample": sample}

    import paper_2602_20063_gb300 as S
    S.lib()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    work.setup(S, torch)
    stream = torch.cuda.current_stream()
    timer = KernelTimer(stream)
    clocks = ClockSampler(local)
    torch.cuda.synchronize()
    clocks.start()
    for _ in range(args.warmup):
        work.step(timer)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    timer.active = True
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        work.step(timer)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    clk = clocks.stop()
    timer.active = False
    ktot = timer.totals()
    ms_step = ms / args.steps
    value = world * work.units_per_step() / (ms_step * 1e-3)

    # ---- end to end through the public API from pinned host memory
    host_out, h2d, d2h = work.e2e_setup()
    for _ in range(2):
        work.e2e_step(host_out)
    torch.cuda.synchronize()
    n_e2e = max(2, min(args.steps, 5))
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(n_e2e):
        work.e2e_step(host_out)
    a1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = a0.elapsed_time(a1) / n_e2e
    if world > 1:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())

    # ---- roofline of the dominant kernel
    terms = work.roofline_terms(peaks, ktot, sms)
    kernels = {}
    total_k = sum(v[0] for v in ktot.values())
    for name, (tms, cnt) in ktot.items():
        avg = tms / cnt
        t = terms.get(name)
        entry = {"launches": cnt, "avg_ms": round(avg, 5), "share": round(tms / total_k, 4)}
        if t:
            ach = t["algorithmic"] / (avg * 1e-3) / (1e9 if t["unit"] == "GB/s" else 1e12)
            entry.update({"bound": t["bound"], "achieved": ach, "peak": t["peak"], "unit": t["unit"],
                          "frac": ach / t["peak"], "algorithmic_per_launch": t["algorithmic"], "per_unit": t["per_unit"]})
        kernels[name] = entry
    dom = max(ktot, key=lambda k: ktot[k][0])
    dk = kernels[dom]
    roof = {"kernel": dom, "bound": dk.get("bound"), "achieved": dk.get("achieved"), "peak": dk.get("peak"),
            "unit": dk.get("unit"), "frac": dk.get("frac"),
            "traffic": load_traffic(dom, terms[dom]["files"]) if dom in terms else None,
            "peak_source": ("measured" if peaks["_source"] == "measured" else "fallback") +
                           (" hbm_gbs" if dk.get("unit") == "GB/s" else " FP32 SIMT from unit counts x max clock")}
    extras = {} if args.no_extras else work.extras(S, torch, args.steps)
    line = {"metric": METRIC, "value": value, "unit": work.unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": ["f32", "f16", "bf16"][args.dtype_id], "data": "synthetic",
            "config": dict(work.config, parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": world * work.units_per_step() / (e2e_ms * 1e-3), "unit": work.unit,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": work.launches_per_step * args.steps, "clocks": clk, "kernels": kernels,
            "extras": extras}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["shm", "reference"], default="shm")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="glyphs")
    ap.add_argument("--dtype", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--layout", choices=["texel", "cell"], default="texel")
    ap.add_argument("--glyphs", type=int, default=16384)
    ap.add_argument("--per-glyph", type=int, default=4096)
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    args = ap.parse_args()
    args.dtype_id = {"f32": 0, "f16": 1, "bf16": 2}[args.dtype]
    args.layout_id = {"texel": 0, "cell": 1}[args.layout]
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
