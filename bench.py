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
E2E_WARMUP, E2E_REPEATS, E2E_STEPS = 5, 7, 20
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}


# ----------------------------------------------------------------------------------- environment
def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def reduce_over_ranks(value: float, dist, device="cpu") -> float:
    """Max over ranks (the slowest replica sets the whole-job time); identity on one process."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_link_probe(torch, nbytes=512 << 20, reps=3):
    """Plain page-locked host <-> device copies of nbytes each way (torch copies, the copy engines),
    host to device, device to host, and both at once on two streams, timed right after the end-to-end
    windows: the host link's throughput at that moment, next to which the end-to-end figure is read."""
    h = [torch.empty(nbytes, dtype=torch.uint8).pin_memory() for _ in range(2)]
    d = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
    st = [torch.cuda.Stream(), torch.cuda.Stream()]
    main = torch.cuda.current_stream()

    def timed(up, down):
        for s_ in st:
            s_.wait_stream(main)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(main)
        for s_ in st:
            s_.wait_event(e0)
        for _ in range(reps):
            if up:
                with torch.cuda.stream(st[0]):
                    d[0].copy_(h[0], non_blocking=True)
            if down:
                with torch.cuda.stream(st[1]):
                    h[1].copy_(d[1], non_blocking=True)
        for s_ in st:
            main.wait_stream(s_)
        e1.record(main)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    timed(True, True)
    t_up, t_down, t_both = timed(True, False), timed(False, True), timed(True, True)
    return {"h2d_GBps": round(nbytes / (t_up * 1e-3) / 1e9, 1), "d2h_GBps": round(nbytes / (t_down * 1e-3) / 1e9, 1),
            "both_GBps": round(2 * nbytes / (t_both * 1e-3) / 1e9, 1), "bytes_each_way": nbytes}


def whole_job_rate(units_per_rank: float, world: int, ms_max: float) -> float:
    """Units of all ranks (weak scaling: each rank processes the same amount) per second of the slowest."""
    return world * units_per_rank / (ms_max * 1e-3)


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
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

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
                                          "--format=csv,noheader,nounits", "-lms", "100"],
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
class _NoTimer:
    """Stand-in for KernelTimer when a step runs outside the timed region."""

    def mark(self, name):
        pass


class GlyphField:
    name = "glyphs"
    unit = "queries/s"

    def __init__(self, args, rank):
        self.args = args
        self.G, self.L, self.N, self.per = args.glyphs, 8, 32, args.per_glyph
        self.Q = self.G * self.per
        self.dtype, self.layout = args.dtype_id, args.layout_id
        self.engine = args.engine
        self.e2e_chunks_n, self.e2e_streams_n = args.e2e_chunks, args.e2e_streams
        self.e2e_mode_arg = args.e2e_mode
        self.seed = 20063 + 1 + 1000 * rank
        import shm_inputs as I
        self.c_host = I.sh_coeffs(self.G, self.L, self.seed).astype(np.float32)
        self.config = {"workload": f"glyph field: {self.G} real-SH glyphs, L=8, N=32 (+1 gutter), "
                                   f"{self.per} uniform queries per glyph ({self.Q} total), "
                                   f"{['f32', 'f16', 'bf16'][self.dtype]} {['texel', 'cell'][self.layout]} records; "
                                   f"step = SH bake contraction ({self.engine}) + query",
                       "glyphs": self.G, "L": self.L, "N": self.N, "queries_per_step": self.Q,
                       "l2": "inputs larger than L2 (table 1.82 GB, directions 805 MB)"}

    def setup(self, S, torch):
        import shm_inputs as I
        dev = "cuda"
        self.S, self.torch = S, torch
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
        self.ws = S.build_workspace(self.lut, self.src) if self.engine == "tcgen05" else None
        # launch shape of the query picked by the library's tuner on this batch (kept for the run)
        S.build_lut(self.lut, self.src, ws=self.ws)
        self.tuned = S.tune_query(self.lut, self.dirs, seg=self.seg, reps=3)
        self.config["query_launch_shape"] = self.tuned
        # tcgen05 engine: coefficient split + contraction; CUDA-core engine: one contraction kernel
        self.launches_per_step = 3 if self.engine == "tcgen05" else 2

    def step(self, timer):
        timer.mark("sh_build_gemm")
        self.S.build_lut(self.lut, self.src, ws=self.ws)
        timer.mark("query_fwd")
        self.S.query(self.lut, self.dirs, seg=self.seg, out=self.out)
        timer.mark("_end")

    def units_per_step(self):
        return self.Q

    def e2e_step(self, host_out):
        if self.e2e_mode == "zero_copy":
            return self.e2e_step_zero_copy(host_out)
        return self.e2e_step_pipeline(host_out)

    def e2e_step_zero_copy(self, host_out):
        """Public API on page-locked host buffers: the coefficients are copied to the device (5 MB),
        the bake runs, and the query reads the directions from host memory and writes R, grad and
        normal into host memory itself, over the host link, with no staging copies."""
        self.coeffs.copy_(self.c_pinned, non_blocking=True)
        self.S.build_lut(self.lut, self.src, ws=self.ws)
        self.S.query(self.lut, self.dirs_host, seg=self.seg, out=host_out)

    def e2e_step_pipeline(self, host_out):
        """Public API from pinned host buffers, pipelined over glyph chunks: each chunk's directions
        and coefficients go host to device on one copy stream, its bake and query run on the kernel
        stream, its outputs go device to host on a second copy stream.  Per-chunk events order a
        chunk's copies and kernels, and each chunk buffer against the previous step's use of it, so
        both copy directions and the kernels of neighbouring chunks (and steps) overlap."""
        torch, S = self.torch, self.S
        h2d, d2h = self.e2e_h2d, self.e2e_d2h
        for c, (lut_c, src_c, seg_c, g0, g1) in enumerate(self.e2e_chunks):
            q0, q1 = g0 * self.per, g1 * self.per
            if self.e2e_used[c]:
                h2d.wait_event(self.e2e_ev_q[c])  # the last query of this chunk has read its inputs
            with torch.cuda.stream(h2d):
                self.dirs[q0:q1].copy_(self.dirs_host[q0:q1], non_blocking=True)
                self.coeffs[g0:g1].copy_(self.c_pinned[g0:g1], non_blocking=True)
            self.e2e_ev_in[c].record(h2d)
            k = c % len(self.e2e_streams)
            ks = self.e2e_streams[k]
            ks.wait_event(self.e2e_ev_in[c])
            if self.e2e_used[c]:
                ks.wait_event(self.e2e_ev_out[c])  # the last outputs of this chunk are on the host
            S.build_lut(lut_c, src_c, ws=self.e2e_ws[k], stream=ks)
            out_c = {kk: v[q0:q1] for kk, v in self.out.items()}
            S.query(lut_c, self.dirs[q0:q1], seg=seg_c, out=out_c, stream=ks)
            self.e2e_ev_q[c].record(ks)
            d2h.wait_event(self.e2e_ev_q[c])
            with torch.cuda.stream(d2h):
                for kk in ("R", "grad", "normal"):
                    host_out[kk][q0:q1].copy_(out_c[kk], non_blocking=True)
            self.e2e_ev_out[c].record(d2h)
            self.e2e_used[c] = True

    def e2e_begin(self):
        """Start of a timed window: the pipeline's streams wait for the current stream (its start
        event and any earlier work on the buffers)."""
        if self.e2e_mode == "copy_pipeline":
            cur = self.torch.cuda.current_stream()
            for st in [self.e2e_h2d, self.e2e_d2h] + self.e2e_streams:
                st.wait_stream(cur)

    def e2e_end(self):
        """End of a timed window: the current stream waits for every copy and kernel of the pipeline."""
        if self.e2e_mode == "copy_pipeline":
            cur = self.torch.cuda.current_stream()
            for st in [self.e2e_h2d, self.e2e_d2h] + self.e2e_streams:
                cur.wait_stream(st)

    def e2e_setup(self, mode=None):
        self.e2e_mode = mode or self.e2e_mode_arg
        chunks, streams = self.e2e_chunks_n, self.e2e_streams_n
        torch, S = self.torch, self.S
        self.c_pinned = torch.from_numpy(self.c_host).pin_memory()
        host_out = {k: torch.empty(v.shape, dtype=torch.float32).pin_memory() for k, v in self.out.items()}
        h2d = self.dirs.numel() * 4 + self.coeffs.numel() * 4
        d2h = sum(v.numel() * 4 for v in self.out.values())
        if self.e2e_mode == "zero_copy":
            self.e2e_note = "kernels read the directions from and write the outputs to the page-locked host buffers"
            return host_out, h2d, d2h
        self.e2e_note = (f"{chunks} glyph chunks: host-to-device copies on one stream, bake + query on {streams} kernel "
                         "stream(s), device-to-host copies on a second copy stream, ordered by per-chunk events; "
                         "consecutive steps overlap inside a timed window")
        self.e2e_streams = [torch.cuda.Stream() for _ in range(streams)]
        self.e2e_h2d, self.e2e_d2h = torch.cuda.Stream(), torch.cuda.Stream()
        per_glyph = S.records_per_glyph(self.N, self.layout) * S.record_bytes(self.dtype, self.layout)
        elem = self.lut.data.element_size()
        self.e2e_chunks = []
        Gc = (self.G + chunks - 1) // chunks
        for g0 in range(0, self.G, Gc):
            g1 = min(self.G, g0 + Gc)
            lut_c = S.Lut(data=self.lut.data[g0 * per_glyph // elem:g1 * per_glyph // elem], n_glyphs=g1 - g0,
                          dtype=self.dtype, layout=self.layout, N_uniform=self.N)
            src_c = S.Source(kind=S.SHM_SRC_SH, L=self.L, coeffs=self.coeffs[g0:g1], basis=self.basis)
            seg_c = (self.seg[g0:g1 + 1] - self.seg[g0]).contiguous()
            self.e2e_chunks.append((lut_c, src_c, seg_c, g0, g1))
        n = len(self.e2e_chunks)
        self.e2e_ev_in, self.e2e_ev_q, self.e2e_ev_out = ([torch.cuda.Event() for _ in range(n)] for _ in range(3))
        self.e2e_used = [False] * n
        ws_c = self.e2e_chunks[0][1]
        self.e2e_ws = ([S.build_workspace(self.e2e_chunks[0][0], ws_c) for _ in range(streams)]
                       if self.engine == "tcgen05" else [None] * streams)
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
                          "files": ["paper_2602_20063_gb300/csrc/shm_query_staged.cu",
                                    "paper_2602_20063_gb300/csrc/shm_device.cuh"]},
            "sh_build_gemm": ({"bound": "alu", "algorithmic": 2.0 * self.G * K * 4 * T, "unit": "TFLOP/s",
                               "peak": fp32_simt_peak_tflops(peaks, sms),
                               "per_unit": f"2 K = {2 * K} flop per stored scalar, {4 * T} scalars per glyph",
                               "files": ["paper_2602_20063_gb300/csrc/shm_build.cu"]}
                              if self.engine == "simt" else
                              {"bound": "hbm", "algorithmic": lut_bytes + self.G * K * 4 + 4 * T * K * 4,
                               "unit": "GB/s", "peak": peaks["hbm_gbs"],
                               "per_unit": f"{lut_bytes / self.G:.0f} B of table written per glyph + coefficients + basis read "
                                           f"(tensor work 3 x 2 K' x 4T = {3 * 2 * ((K + 7) // 8 * 8) * 4 * T / 1e6:.1f} MFLOP "
                                           "tf32 per glyph, K' = K rounded up to the MMA's K step of 8, is not the binding resource)",
                               "files": ["paper_2602_20063_gb300/csrc/shm_bake_tc.cu"]}),
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
        bwd_det = timeit(lambda: S.query_backward(self.lut, self.dirs, dl, gR=gR, ggrad=gG, gnormal=gN, seg=self.seg,
                                                  want_ddirs=True, deterministic=True), n)
        # the bake's adjoint (dL/dcoeffs from dL/dtable): tensor cores vs the float32 CUDA-core contraction
        dco = torch.empty((self.G, (self.L + 1) ** 2), dtype=torch.float32, device="cuda")
        bake_bwd = timeit(lambda: S.build_lut_backward(dl, self.L, self.basis, out=dco), n)
        bake_bwd_simt = timeit(lambda: S.build_lut_backward(dl, self.L, self.basis, out=dco, cuda_cores=True), n)
        dl_bytes = dl.data.numel() * 4
        ex["bake_bwd"] = {"ms": round(bake_bwd, 4), "cuda_cores_ms": round(bake_bwd_simt, 4),
                          "speedup_vs_cuda_cores": round(bake_bwd_simt / bake_bwd, 3),
                          "achieved_GBps": round(dl_bytes / (bake_bwd * 1e-3) / 1e9, 1),
                          "frac_of_measured_hbm": round(dl_bytes / (bake_bwd * 1e-3) / 1e9 / load_peaks()["hbm_gbs"], 3),
                          "per_unit": f"{dl_bytes / self.G:.0f} B of dL/dtable read per glyph (the basis operands, "
                                      "21 MB, come from L2); 3 x 2 x Kp x 4T tf32 flop per glyph on the tensor cores",
                          "note": "dcoeffs = dL/dtable . basis^T, tcgen05 3xTF32 with a fixed-order cluster reduction "
                                  "(deterministic); cuda_cores: the float32 SIMT contraction with split-K atomics"}
        del dco
        ex["fwd_bwd"] = {"fwd_ms": round(fwd, 4), "bwd_ms": round(bwd, 4), "fwd_plus_bwd_over_fwd": round((fwd + bwd) / fwd, 3),
                         "bwd_deterministic_ms": round(bwd_det, 4), "bake_bwd_ms": round(bake_bwd, 4),
                         "note": "backward = recompute + 4 float4 vector reductions per query (issued by lane pairs, one 32-byte footprint row per pair) into a float32 texel table + d/ddirs; "
                                 "deterministic = per-glyph CTA, chunks sorted by cell, per-cell sums added in a fixed order"}
        del dl
        ex["precision"] = self.precision_extras(S, torch, timeit, n, fwd)
        ex["write_ceiling"] = self.write_ceiling(torch, timeit, n)
        ex["planet"] = planet_leg(self.args, S, torch)
        ex["e2e_modes"] = self.e2e_mode_extras(torch)
        ex["recon"] = self.recon_extras(S, torch, timeit, n, fwd)
        ex["equal_storage"] = self.equal_storage_extras(S, torch)
        ex["cuda_graph"] = self.graph_extras(S, torch, timeit, n)
        return ex

    def e2e_mode_extras(self, torch):
        """End to end (public API, page-locked host buffers) in both forms: kernels reading and
        writing the host buffers directly, and chunked staging copies overlapped with the kernels."""
        res = {}
        keep = self.e2e_mode
        for mode in ("zero_copy", "copy_pipeline"):
            host_out, h2d, d2h = self.e2e_setup(mode)
            self.e2e_begin()
            for _ in range(E2E_WARMUP):
                self.e2e_step(host_out)
            self.e2e_end()
            torch.cuda.synchronize()
            st = torch.cuda.current_stream()
            wins = []
            for _ in range(E2E_REPEATS):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                self.e2e_begin()
                for _ in range(E2E_STEPS):
                    self.e2e_step(host_out)
                self.e2e_end()
                e1.record(st)
                torch.cuda.synchronize()
                wins.append(e0.elapsed_time(e1) / E2E_STEPS)
            ms = statistics.median(wins)
            res[mode] = {"ms_per_step": round(ms, 3), "queries_per_s": self.Q / (ms * 1e-3),
                         "host_link_GBps": round((h2d + d2h) / (ms * 1e-3) / 1e9, 1),
                         "window_ms_per_step": [round(w, 3) for w in wins]}
            if mode == "copy_pipeline":
                res["host_link_ceiling"] = self.host_link_ceiling(torch, host_out)
                res["copy_pipeline"]["frac_of_host_link_ceiling"] = round(
                    res["host_link_ceiling"]["both_ms"] / ms, 3)
            del host_out
        self.e2e_mode = keep
        return res

    def host_link_ceiling(self, torch, host_out):
        """Plain copies of the step's bytes between page-locked host memory and the device: the
        directions host to device, the outputs device to host, each alone and both at once on two
        streams (torch copies, the copy engines)."""
        st = [torch.cuda.Stream(), torch.cuda.Stream()]

        def h2d():
            with torch.cuda.stream(st[0]):
                self.dirs.copy_(self.dirs_host, non_blocking=True)

        def d2h():
            with torch.cuda.stream(st[1]):
                for k in ("R", "grad", "normal"):
                    host_out[k].copy_(self.out[k], non_blocking=True)

        def timed(*fns):
            main = torch.cuda.current_stream()
            for s_ in st:
                s_.wait_stream(main)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(main)
            for s_ in st:
                s_.wait_event(e0)
            for _ in range(3):
                for fn in fns:
                    fn()
            for s_ in st:
                main.wait_stream(s_)
            e1.record(main)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / 3
        bi, bo = self.dirs.numel() * 4, sum(v.numel() * 4 for v in self.out.values())
        t_in, t_out, t_both = timed(h2d), timed(d2h), timed(h2d, d2h)
        return {"h2d_ms": round(t_in, 3), "h2d_GBps": round(bi / (t_in * 1e-3) / 1e9, 1),
                "d2h_ms": round(t_out, 3), "d2h_GBps": round(bo / (t_out * 1e-3) / 1e9, 1),
                "both_ms": round(t_both, 3), "both_GBps": round((bi + bo) / (t_both * 1e-3) / 1e9, 1)}

    def write_ceiling(self, torch, timeit, n):
        """Write-only ceiling for the bake, which reads almost nothing and writes the table: a
        plain device fill (torch's own kernel) of a buffer of the table's size, and the bake's
        time against it."""
        nbytes = self.lut.data.numel() * self.lut.data.element_size()
        buf = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
        ms = timeit(lambda: buf.fill_(1.0), n)
        gbs = nbytes / (ms * 1e-3) / 1e9
        bake = timeit(lambda: self.S.build_lut(self.lut, self.src, ws=self.ws), n)
        del buf
        return {"fill_ms": round(ms, 4), "fill_GBps": round(gbs, 1),
                "fill_frac_of_measured_copy": round(gbs / load_peaks()["hbm_gbs"], 3),
                "bake_ms": round(bake, 4), "bake_over_fill_time": round(bake / ms, 3),
                "note": f"torch fill_ of {nbytes / 1e9:.2f} GB (the glyph table's size), write-only traffic"}

    def graph_extras(self, S, torch, timeit, n):
        """The step (bake + query) captured once in a CUDA graph and replayed, against eager launches."""
        eager = timeit(lambda: self.step(_NoTimer()), n)
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            self.step(_NoTimer())  # warm the capture stream
        torch.cuda.current_stream().wait_stream(side)
        with torch.cuda.graph(graph):
            self.step(_NoTimer())
        replay = timeit(graph.replay, n)
        return {"eager_ms": round(eager, 4), "graph_replay_ms": round(replay, 4),
                "queries_per_s_graph": self.Q / (replay * 1e-3),
                "launches_per_step": self.launches_per_step}

    def recon_extras(self, S, torch, timeit, n, hermite_ms):
        """Value-only baselines (§4.2, §4.5) on the same glyphs, directions and segments: a value
        table per glyph (two-texel gutter) and the same query skeleton; time per method and value
        PSNR against direct SH evaluation on the first 64 glyphs' queries."""
        vlut = S.alloc_lut(self.G, self.N, S.SHM_F32, S.SHM_LAYOUT_VALUE)
        S.build_lut(vlut, S.Source(kind=S.SHM_SRC_SH, L=self.L, coeffs=self.coeffs))
        nq = 64 * self.per
        Rt, _, _ = S.sh_eval(self.L, self.coeffs[:64].contiguous(), self.dirs[:nq].contiguous(),
                             seg=self.seg[:65].contiguous())
        peak = Rt.abs().max()

        def psnr(R):
            mse = ((R[:nq].double() - Rt.double()) ** 2).mean()
            return round(float(20 * torch.log10(peak.double() / mse.sqrt())), 2)

        S.query(self.lut, self.dirs, seg=self.seg, out=self.out)
        res = {"hermite": {"query_ms": round(hermite_ms, 4), "value_psnr_db": psnr(self.out["R"]),
                           "footprint": "4 records x 4 channels"}}
        o = {k: torch.empty_like(v) for k, v in self.out.items()}
        names = {S.SHM_RECON_NEAREST: "nearest", S.SHM_RECON_BILINEAR: "bilinear_fd",
                 S.SHM_RECON_BICUBIC: "bicubic_catmull_rom", S.SHM_RECON_FAST_BICUBIC: "fast_bicubic_bspline_fd"}
        taps = {S.SHM_RECON_NEAREST: "1 scalar", S.SHM_RECON_BILINEAR: "5 bilinear lookups (12 scalars)",
                S.SHM_RECON_BICUBIC: "16 scalars", S.SHM_RECON_FAST_BICUBIC: "5 x 16 taps (36 scalars)"}
        for m, nm in names.items():
            ms = timeit(lambda: S.query_recon(vlut, m, self.dirs, seg=self.seg, out=o), n)
            res[nm] = {"query_ms": round(ms, 4), "hermite_speedup": round(ms / hermite_ms, 3),
                       "value_psnr_db": psnr(o["R"]), "footprint": taps[m]}
        res["note"] = ("same kernel skeleton and I/O for every method; value table f32 with a two-texel gutter "
                       f"({vlut.data.numel() * 4 / 1e9:.2f} GB) vs Hermite f32 texel records "
                       f"({self.lut.data.numel() * self.lut.data.element_size() / 1e9:.2f} GB); PSNR peak = max|r_true| "
                       f"over {nq} queries of the first 64 glyphs")
        del vlut, o
        return res

    # ---------------------------------------------------------------- oracle sample (CPU)
    def oracle_measure(self, budget_s, procs, pool=None):
        return _glyph_oracle_measure(self, budget_s, procs, pool)

    def precision_glyphs(self):
        """64 glyphs spread over the field; all their queries form the precision sample."""
        return np.unique(np.linspace(0, self.G - 1, 64).round().astype(np.int64))

    def oracle_truth(self, procs):
        """Float64 direct SH (the oracle, spawned processes) at every query of the precision glyphs, on
        the float32 coefficients the device bakes from: {R, grad, normal} float64."""
        import shm_inputs as I
        gs = self.precision_glyphs()
        coeffs = self.c_host[gs].astype(np.float64)
        tasks = []
        for k, g in enumerate(gs):
            d = I.directions_range(int(g) * self.per, self.per, self.seed + 7)
            tasks.append((self.L, coeffs, d, np.full(self.per, k, dtype=np.int32)))
        with _PoolScope(None, procs) as pool:
            res = pool.map(_oracle_truth_task, tasks)
        return {"R": np.concatenate([r[0] for r in res]), "grad": np.concatenate([r[1] for r in res]),
                "normal": np.concatenate([r[2] for r in res])}

    def equal_storage_extras(self, S, torch):
        """§4.5's equal-storage comparison, rendered (§4.4 renders with the analytic normal): glyph 0 of
        the field (L = 8) ray cast at 512 x 512 with its Hermite table at N and with the value-only
        baselines at 2N (the same bytes: 4 (N+2)^2 = (2N+4)^2 scalars per face), against a reference
        render from a Hermite table at N = 128 (value error ~1e-9, below float32 rounding); fixed camera,
        Blinn-Phong ambient 0.1, k_d 0.7, k_s 0.3, shininess 64, light (1, 1, 1)."""
        W = H = 512
        c = self.coeffs[0:1].contiguous()
        eye = np.array([0.55, 0.65, 3.0])
        fwd = -eye / np.linalg.norm(eye)
        right = np.cross(fwd, [0.0, 1.0, 0.0])
        right /= np.linalg.norm(right)
        up = np.cross(right, fwd)
        cam = S.make_camera(eye, fwd, right, up, 40.0, W, H)

        bracket = {}

        def render(lut, recon=0):
            # one bounding sphere for every render, so that all march the same samples along a ray
            objs = S.objects_tensor(np.zeros((1, 3)), [1.0], [bracket["rmax"]], [0])
            return S.raycast(lut, objs, 1, cam, S.make_raycast_params(recon=recon))

        def hermite_table(N):
            lut = S.alloc_lut(1, N)
            S.build_lut(lut, S.Source(kind=S.SHM_SRC_SH, L=self.L, coeffs=c, basis=S.sh_basis(N, self.L)))
            return lut

        def hermite(N):
            return render(hermite_table(N))

        def value(N2, method):
            v = S.alloc_lut(1, N2, S.SHM_F32, S.SHM_LAYOUT_VALUE)
            S.build_lut(v, S.Source(kind=S.SHM_SRC_SH, L=self.L, coeffs=c))
            return render(v, method)

        ref_lut = hermite_table(128)
        bracket["rmax"] = 1.25 * float(S.lut_bounds(ref_lut)[0])  # covers every table's overshoot here
        ref = render(ref_lut)
        rI = ref["rgba"][..., 0].double()
        rN = ref["normal"].double()
        rhit = ref["obj_id"] >= 0
        peak = float(rI.max())

        def metrics(o):
            I = o["rgba"][..., 0].double()
            hit = o["obj_id"] >= 0
            both = hit & rhit
            mse = float(((I - rI) ** 2).mean())
            ang = torch.rad2deg(torch.acos((o["normal"].double()[both] * rN[both]).sum(-1).clamp(-1.0, 1.0)))
            return {"shaded_psnr_db": round(10 * math.log10(peak * peak / max(mse, 1e-30)), 2),
                    "normal_mean_deg": round(float(ang.mean()), 4),
                    "normal_p95_deg": round(float(torch.quantile(ang, 0.95)), 4),
                    "silhouette_mismatch_px": int((hit ^ rhit).sum())}
        res = {}
        for N in (8, 16, 32, 64):
            res[f"N{N}"] = {"hermite_N": metrics(hermite(N)),
                            "bilinear_fd_2N": metrics(value(2 * N, S.SHM_RECON_BILINEAR)),
                            "catmull_rom_2N": metrics(value(2 * N, S.SHM_RECON_BICUBIC))}
        res["setup"] = (f"glyph 0 of the field (L = {self.L}), {W} x {H}, camera at {eye.round(2).tolist()} looking at "
                        "the centre, 40 deg vertical field of view; reference: Hermite table at N = 128; every render "
                        "marches the same bounding sphere (1.25 x the reference table's bound); PSNR over the whole "
                        "image (background 0) with peak = the reference's brightest pixel; normal angles over pixels "
                        "both renders hit")
        res["paper_context"] = ("§4.5 (WebGPU renders, its own glyph, camera and lighting): bilinear N = 16 vs Hermite "
                                "N = 8: 21.4 vs 26.4 dB; bilinear N = 32 vs Hermite N = 16: 24.7 vs 45.5 dB")
        return res

    def precision_extras(self, S, torch, timeit, n, fwd_ms):
        """Error of each storage form against float64 direct SH (§4.2 measures error against direct
        SH): the sampled glyphs' tables as baked by the step (f32 texel) and re-encoded (f16 / bf16,
        texel / cell, value offset r0 = the glyph's mean radius c_00 Y_00), queried at all their
        directions; and each form's query time on the whole field."""
        tr = getattr(self, "truth", None)
        if tr is None:
            return None
        gs = torch.from_numpy(self.precision_glyphs()).cuda()
        ng = int(gs.numel())
        rec = self.S.records_per_glyph(self.N, 0) * 4
        sub = S.alloc_lut(ng, self.N)
        sub.data.view(ng, rec).copy_(self.lut.data.view(self.G, rec)[gs])
        d = self.dirs.view(self.G, self.per, 3)[gs].reshape(-1, 3).contiguous()
        seg = torch.arange(ng + 1, dtype=torch.int64, device="cuda") * self.per
        r0 = (self.coeffs[gs, 0] * 0.28209479177387814).contiguous()
        Rt, Gt, Nt = (torch.from_numpy(tr[k]).cuda() for k in ("R", "grad", "normal"))
        maxR, maxG = float(Rt.abs().max()), float(Gt.norm(dim=1).max())
        res = {}
        for name, dt, ly in (("f32_texel", 0, 0), ("f32_cell", 0, 1), ("f16_texel", 1, 0), ("bf16_texel", 2, 0),
                             ("f16_cell", 1, 1), ("bf16_cell", 2, 1)):
            L = sub if (dt, ly) == (0, 0) else S.like_lut(sub, dtype=dt, layout=ly, r0=r0)
            if (dt, ly) != (0, 0):
                S.pack_lut(sub, L)
            o = S.query(L, d, seg=seg)
            eR = (o["R"].double() - Rt).abs()
            eG = (o["grad"].double() - Gt).norm(dim=1)
            cosang = (o["normal"].double() * Nt).sum(1).clamp(-1.0, 1.0)
            ang = torch.rad2deg(torch.acos(cosang))
            entry = {"R_max_rel": float(eR.max()) / maxR, "R_rms_rel": float(eR.pow(2).mean().sqrt()) / maxR,
                     "grad_max_rel": float(eG.max()) / maxG, "grad_rms_rel": float(eG.pow(2).mean().sqrt()) / maxG,
                     "normal_max_deg": float(ang.max()), "normal_mean_deg": float(ang.mean())}
            if (dt, ly) == (0, 0):
                entry["query_ms"] = round(fwd_ms, 4)
            else:
                Lf = S.like_lut(self.lut, dtype=dt, layout=ly,
                                r0=(self.coeffs[:, 0] * 0.28209479177387814).contiguous())
                S.pack_lut(self.lut, Lf)
                of = {k: torch.empty_like(v) for k, v in self.out.items()}
                ms = timeit(lambda: S.query(Lf, self.dirs, seg=self.seg, out=of), n)
                entry["query_ms"] = round(ms, 4)
                entry["speedup_vs_f32_texel"] = round(fwd_ms / ms, 3)
                del Lf, of
            res[name] = entry
        res["sample"] = (f"{ng} glyphs spread over the field x {self.per} queries ({ng * self.per}); truth: the "
                         "oracle's float64 direct SH on the float32 coefficients; R and grad errors relative to "
                         "max|R| and max|grad R| of the sample; normal error as the angle to the true normal")
        return res

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


def _oracle_truth_task(args):
    """Direct float64 SH (no table) at the given queries: the ground truth of the precision extras."""
    L, coeffs, dirs, glyph = args
    import oracle as O
    return O.sh_eval(L, coeffs, dirs, glyph=glyph, nthreads=1)


def oracle_sample(work, budget_s, procs):
    """Time the oracle on a bounded sample of the workload (spawned processes): (rate, description)."""
    return work.oracle_measure(budget_s, procs)


def _spawn_pool(procs):
    import multiprocessing as mp
    return mp.get_context("spawn").Pool(procs)


class _PoolScope:
    """The caller's process pool, or a spawned one closed on exit."""

    def __init__(self, pool, procs):
        self.pool, self.own, self.procs = pool, pool is None, procs

    def __enter__(self):
        if self.own:
            self.pool = _spawn_pool(self.procs)
        return self.pool

    def __exit__(self, *exc):
        if self.own:
            self.pool.close()
            self.pool.join()
        return False


def _glyph_oracle_measure(work, budget_s, procs, pool=None):
    with _PoolScope(pool, procs) as pool:
        pool.map(_oracle_glyph_task, work.oracle_task_args(procs))  # start the workers
        t0 = time.perf_counter()
        pool.map(_oracle_glyph_task, work.oracle_task_args(procs, start=procs))  # calibrate
        per_round = max(time.perf_counter() - t0, 1e-3)
        rounds = max(1, int(budget_s / per_round))
        n = procs * rounds
        t0 = time.perf_counter()
        done = sum(pool.map(_oracle_glyph_task, work.oracle_task_args(n, start=2 * procs)))
        dt = time.perf_counter() - t0
    return done / dt, f"{n} glyphs (FP64 bake of each + its {work.per} queries), {procs} processes, {dt:.1f} s"


class Planet:
    """Procedural planet (§4.10): R = 1 + 0.02 fBm (8 octaves of value noise), N = 2048 per face
    (table 403 MB f32, out of L2).  Step = FD bake of the height field + 2^28 uniform random
    queries + 2^28 screen-coherent queries (4K orbit view, 8x8 pixel tiles)."""
    name = "planet"
    unit = "queries/s"

    def __init__(self, args, rank):
        self.N = 2048
        self.Qr = args.planet_queries
        self.Qc = args.planet_queries
        self.dtype, self.layout = args.dtype_id, args.layout_id
        self.l2g_choice = args.l2_fetch_granularity
        self.random_mode = args.planet_random
        self.band = args.planet_band_bytes
        self.seed = 20063 + 3 + 1000 * rank
        import shm_inputs as I
        self.keys = I.fbm_keys(self.seed)
        self.config = {"workload": f"procedural planet: R = 1 + 0.02 fBm (8 octaves value noise), N = 2048 (+1 gutter), "
                                   f"{['f32', 'f16', 'bf16'][self.dtype]} {['texel', 'cell'][self.layout]} records; "
                                   f"step = FD bake + {self.Qr} random + {self.Qc} screen-coherent (4K orbit) queries",
                       "N": self.N, "queries_per_step": self.Qr + self.Qc,
                       "l2": "inputs larger than L2 (table 403 MB f32, directions 3.2 GB per set)"}

    def setup(self, S, torch):
        import shm_inputs as I
        self.S, self.torch = S, torch
        dev = "cuda"
        self.lut = S.alloc_lut(1, self.N, self.dtype, self.layout, r0=[1.0])
        self.src = S.Source(kind=S.SHM_SRC_FBM, octaves=8, keys=torch.from_numpy(self.keys.view(np.int32)).to(dev),
                            base_freq=2.0, lacunarity=2.0, gain=0.5, amplitude=0.02)
        if self.dtype != 0 or self.layout != 0:
            self.lut32 = S.alloc_lut(1, self.N, 0, 0, r0=[1.0])
        self.dr = torch.empty((self.Qr, 3), dtype=torch.float32, device=dev)
        for s0, d in I.directions_chunked(self.Qr, self.seed + 11):
            self.dr[s0:s0 + len(d)].copy_(torch.from_numpy(d))
        self.dc = torch.from_numpy(I.coherent_sphere_directions(self.Qc, n_frames=128)).to(dev)
        # launch shape of the per-query kernel picked by the library's tuner (random batch)
        self.bake()
        self.tuned = S.tune_query(self.lut, self.dr, reps=2)
        self.config["query_launch_shape"] = self.tuned
        self.out = {k: torch.empty(s, dtype=torch.float32, device=dev)
                    for k, s in (("R", (self.Qr,)), ("grad", (self.Qr, 3)), ("normal", (self.Qr, 3)))}
        if self.random_mode == "binned":
            self.ws = S.query_binned_workspace(self.lut, self.Qr, self.band)
            self.config["random_queries"] = dict(path="binned (shm_query_binned: partition by face and row band, "
                                                      "query in partitioned order, results back in query order)",
                                                 band_bytes=self.band or "default", workspace_bytes=self.ws.numel(),
                                                 **S.query_binned_bins(self.lut, self.band))
        else:
            self.ws = None
            self.config["random_queries"] = {"path": "direct (shm_query in query order)"}
        self.config["l2_fetch_granularity"] = self.pick_l2_granularity(self.l2g_choice)
        self.launches_per_step = ((1 if (self.dtype == 0 and self.layout == 0) else 2) + 1 +
                                  (5 if self.random_mode == "binned" else 1))

    def query_random(self, out, stream=None, dirs=None, ws=None):
        d = self.dr if dirs is None else dirs
        if self.random_mode == "binned":
            self.S.query_binned(self.lut, d, self.ws if ws is None else ws, band_bytes=self.band, out=out,
                                stream=stream)
        else:
            self.S.query(self.lut, d, out=out, stream=stream)

    def pick_l2_granularity(self, choice):
        """The context's L2 fetch granularity for this process (shm_l2_fetch_granularity): "auto"
        times one step at 128 B (the behaviour of a fresh context) and at 64 B and keeps the faster.
        The random query repeated back to back runs 13 % faster at 64 B (more distinct table pieces
        stay in L2 between repetitions); inside the step, after the bake and the coherent queries,
        64 B measured 1-2 % slower."""
        S, torch = self.S, self.torch
        if choice != "auto":
            S.l2_fetch_granularity(int(choice))
            return {"bytes": int(choice), "how": "fixed by --l2-fetch-granularity"}
        st = torch.cuda.current_stream()
        times = {}
        for g in (128, 64):
            S.l2_fetch_granularity(g)
            self.step(_NoTimer())
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(2):
                self.step(_NoTimer())
            e1.record(st)
            torch.cuda.synchronize()
            times[g] = e0.elapsed_time(e1) / 2
        best = min(times, key=times.get)
        S.l2_fetch_granularity(best)
        return {"bytes": best, "how": "auto: one step timed at each", "step_ms": {str(k): round(v, 3) for k, v in times.items()}}

    def bake(self):
        if self.dtype == 0 and self.layout == 0:
            self.S.build_lut(self.lut, self.src)
        else:
            self.S.build_lut(self.lut32, self.src)
            self.S.pack_lut(self.lut32, self.lut)

    def step(self, timer):
        timer.mark("fbm_bake")
        self.bake()
        timer.mark("query_random")
        self.query_random(self.out)
        timer.mark("query_coherent")
        self.S.query(self.lut, self.dc, out=self.out)
        timer.mark("_end")

    def units_per_step(self):
        return self.Qr + self.Qc

    def e2e_setup(self):
        torch = self.torch
        self.hr = self.dr.cpu().pin_memory()
        self.hc = self.dc.cpu().pin_memory()
        host_out = {k: torch.empty(v.shape, dtype=torch.float32).pin_memory() for k, v in self.out.items()}
        h2d = (self.dr.numel() + self.dc.numel()) * 4
        d2h = 2 * sum(v.numel() * 4 for v in self.out.values())
        self.e2e_streams = [torch.cuda.Stream() for _ in range(3)]
        self.e2e_chunks = 8
        self.e2e_steps = 5
        step = (self.Qr + self.e2e_chunks - 1) // self.e2e_chunks
        self.e2e_ws = ([self.S.query_binned_workspace(self.lut, step, self.band) for _ in self.e2e_streams]
                       if self.random_mode == "binned" else [None] * len(self.e2e_streams))
        return host_out, h2d, d2h

    def e2e_step(self, host_out):
        """Public API from page-locked host memory: the bake, then both query sets in chunks that
        rotate over three streams (a chunk's directions copy in, its queries run and its outputs copy
        out while its neighbours do the same), so the host link carries traffic both ways at once.
        Chunk c of both sets shares a stream, so the device output buffer is reused in order."""
        torch = self.torch
        main = torch.cuda.current_stream()
        self.bake()
        for st in self.e2e_streams:
            st.wait_stream(main)
        n = self.Qr
        step = (n + self.e2e_chunks - 1) // self.e2e_chunks
        for kind, d, h in (("random", self.dr, self.hr), ("coherent", self.dc, self.hc)):
            for c, q0 in enumerate(range(0, n, step)):
                q1 = min(n, q0 + step)
                st = self.e2e_streams[c % len(self.e2e_streams)]
                with torch.cuda.stream(st):
                    d[q0:q1].copy_(h[q0:q1], non_blocking=True)
                    o = {k: v[q0:q1] for k, v in self.out.items()}
                    if kind == "random":
                        self.query_random(o, stream=st, dirs=d[q0:q1], ws=self.e2e_ws[c % len(self.e2e_streams)])
                    else:
                        self.S.query(self.lut, d[q0:q1], out=o, stream=st)
                    for k in ("R", "grad", "normal"):
                        host_out[k][q0:q1].copy_(o[k], non_blocking=True)
        for st in self.e2e_streams:
            main.wait_stream(st)

    def roofline_terms(self, peaks, ktot, sms):
        rec = self.S.record_bytes(self.dtype, self.layout) * (1 if self.layout == 1 else 4)
        per_q = rec + 12 + 28
        T = 6 * (self.N + 2) ** 2
        qfiles = ["paper_2602_20063_gb300/csrc/shm_query_kernel.cuh", "paper_2602_20063_gb300/csrc/shm_device.cuh"]
        rfiles = (["paper_2602_20063_gb300/csrc/shm_query_binned.cu", "paper_2602_20063_gb300/csrc/shm_device.cuh",
                   "paper_2602_20063_gb300/csrc/shm_stage.cuh"] if self.random_mode == "binned" else qfiles)
        return {
            "query_random": {"bound": "hbm", "algorithmic": self.Qr * per_q, "unit": "GB/s", "peak": peaks["hbm_gbs"],
                             "per_unit": f"{per_q} B/query: 4 corner records ({rec} B, the paper's 16-scalar "
                                         "accounting) + 12 B direction + 28 B outputs, no reuse assumed"
                                         + ("; timed: the whole binned query (count, scan, partition, query in "
                                            "partitioned order, gradient/normal back in query order)"
                                            if self.random_mode == "binned" else ""),
                             "files": rfiles},
            "query_coherent": {"bound": "hbm", "algorithmic": self.Qc * per_q, "unit": "GB/s", "peak": peaks["hbm_gbs"],
                               "per_unit": f"{per_q} B/query (no-reuse accounting; neighbouring pixels share texels, "
                                           "so L2 serves most table reads)", "files": qfiles},
            "fbm_bake": {"bound": "hbm", "algorithmic": T * 16, "unit": "GB/s", "peak": peaks["hbm_gbs"],
                         "per_unit": "16 B written per texel (8 octaves x 8 PCG3D lattice hashes per sample); the "
                                     "kernel is issue-bound, not DRAM-bound: ncu shows issue slots 88 % and DRAM 5 % busy "
                                     "(profiles/fd_face_fbm_planet.md)",
                         "files": ["paper_2602_20063_gb300/csrc/shm_build.cu"]},
        }

    def extras(self, S, torch, steps):
        """Cell layout and 16-bit storage on the random queries."""
        ex = {}
        st = torch.cuda.current_stream()

        def timeit(fn, n=5):
            fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(n):
                fn()
            e1.record(st)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / n

        base = self.lut if (self.dtype == 0 and self.layout == 0) else self.lut32
        S.build_lut(base, self.src)
        ref = {k: torch.empty_like(v) for k, v in self.out.items()}
        t_ref = timeit(lambda: S.query(base, self.dr, out=ref))
        ws = self.ws if self.ws is not None else S.query_binned_workspace(base, self.Qr, self.band)
        # the cell layout partitions into more bands (bigger rows): size the shared workspace for it
        cell_shape = S.Lut(data=torch.empty(8, device="cuda"), n_glyphs=1, dtype=0, layout=1, N_uniform=self.N)
        wsb = max(ws.numel(), S.query_binned_workspace_bytes(cell_shape, self.Qr, self.band))
        if wsb > ws.numel():
            ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
        t_bin = timeit(lambda: S.query_binned(base, self.dr, ws, band_bytes=self.band, out=ref))
        for name, dt, ly in (("f32_cell", 0, 1), ("bf16_texel", 2, 0), ("f16_texel", 1, 0), ("f16_cell", 1, 1)):
            L2 = S.like_lut(base, dtype=dt, layout=ly)
            S.pack_lut(base, L2)
            o = {k: torch.empty_like(v) for k, v in self.out.items()}
            ms = timeit(lambda: S.query(L2, self.dr, out=o))
            msb = timeit(lambda: S.query_binned(L2, self.dr, ws, band_bytes=self.band, out=o))
            rb = S.record_bytes(dt, ly) * (1 if ly == 1 else 4) + 40
            ex[name] = {"query_random_ms": round(ms, 4), "queries_per_s": self.Qr / (ms * 1e-3),
                        "speedup_vs_f32_texel": round(t_ref / ms, 3),
                        "achieved_GBps_no_reuse": rb * self.Qr / (ms * 1e-3) / 1e9,
                        "binned_query_random_ms": round(msb, 4), "binned_queries_per_s": self.Qr / (msb * 1e-3),
                        "max_err_R_rel_vs_f32": float((o["R"] - ref["R"]).abs().max() / ref["R"].abs().max()),
                        "max_err_grad_rel_vs_f32": float((o["grad"] - ref["grad"]).abs().max()
                                                         / ref["grad"].norm(dim=1).max())}
            del L2, o
        ex["f32_texel_binned"] = {"query_random_ms": round(t_bin, 4), "queries_per_s": self.Qr / (t_bin * 1e-3),
                                  "speedup_vs_direct": round(t_ref / t_bin, 3),
                                  "frac_of_measured_hbm_at_104B": round(104 * self.Qr / (t_bin * 1e-3) / 1e9
                                                                        / load_peaks()["hbm_gbs"], 3)}
        del ws
        # random-gather ceiling: the same traffic pattern (12 B in, one aligned block of the
        # footprint's size gathered from a table of the same size as the query's, 28 B out)
        # without the arithmetic (a bench-only probe, not part of libshm.so)
        import bench_probe
        bench_probe.build()
        probe_out = torch.empty((self.Qr, 7), dtype=torch.float32, device="cuda")
        ceiling = {}
        ex["f32_texel"] = {"query_random_ms": round(t_ref, 4)}
        for blk, dt, ly, tab_name in ((64, 0, 0, "f32_texel"), (64, 0, 1, "f32_cell"), (32, 1, 0, "f16_texel"),
                                      (32, 1, 1, "f16_cell")):
            Lc = base if (dt, ly) == (0, 0) else S.like_lut(base, dtype=dt, layout=ly)
            nb = Lc.data.numel() * Lc.data.element_size()
            ms = timeit(lambda: bench_probe.gather_probe(Lc.data, blk, self.dr, out=probe_out))
            q_ms = ex[tab_name]["query_random_ms"]
            ceiling[f"{blk}B_from_{tab_name}_table"] = {
                "table_MB": round(nb / 1e6, 1), "probe_ms": round(ms, 4), "items_per_s": self.Qr / (ms * 1e-3),
                "GBps_at_block_plus_40B": (blk + 40) * self.Qr / (ms * 1e-3) / 1e9,
                "frac_of_measured_hbm": round((blk + 40) * self.Qr / (ms * 1e-3) / 1e9 / load_peaks()["hbm_gbs"], 3),
                f"query_{tab_name}_over_probe_time": round(q_ms / ms, 3)}
            del Lc
        ceiling["note"] = ("uncorrelated aligned gathers of the footprint's bytes (64 B f32, 32 B 16-bit) from a table "
                           "of the query's table size, per item 12 B read + 28 B written; the query does the same "
                           "traffic (texel layouts: two row pieces instead of one block) plus the chart, Hermite and "
                           "S^2 arithmetic.  Items/s fall with table size (100 MB: 41 G/s, 403 MB: 27 G/s, 1.6 GB: "
                           "20 G/s for 64 B): random 32 B sectors, not streaming bandwidth, set this ceiling")
        ex["random_gather_ceiling"] = ceiling
        # the same probe over table sizes and block sizes (a zero buffer; L2 flushed between runs)
        big = torch.zeros(3 << 30, dtype=torch.uint8, device="cuda")
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

        def timeit_flushed(fn, n=5):
            fn()
            ts = []
            for _ in range(n):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                fn()
                e1.record(st)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return statistics.median(ts)
        sweep = {}
        for mb in (100, 201, 403, 806, 1612, 3221):
            tab = big[: mb * 1000 * 1000 // 64 * 64]
            sweep[f"{mb}MB"] = {f"{blk}B": round(self.Qr / (timeit_flushed(
                lambda: bench_probe.gather_probe(tab, blk, self.dr, out=probe_out)) * 1e-3) / 1e9, 2) for blk in (16, 32, 64)}
        sweep["unit"] = "G items/s (2^28 uniform random items, 12 B read + one aligned block + 28 B written each)"
        ex["random_gather_sweep"] = sweep
        del big, flush
        # the random query repeated back to back under each context L2 fetch granularity, per launch shape
        prev = S.l2_fetch_granularity(-1)
        gran = {}
        for g in (128, 64, 32):
            S.l2_fetch_granularity(g)
            gran[f"{g}B"] = S.tune_query(base, self.dr, reps=3)["times_ms"]
        S.l2_fetch_granularity(prev)
        S.tune_query(base, self.dr, reps=2)
        ex["random_query_back_to_back_by_l2_fetch_granularity"] = {
            "ms_per_launch_shape": gran, "restored_bytes": prev,
            "note": "same batch launched repeatedly: table pieces left in L2 by the previous launch are reused"}
        del probe_out
        # derivative-consistent mip chain (§4.7) of the f32 texel table: 2048 -> 1024 -> ... -> 16
        chain = [base]
        for _ in range(7):
            chain.append(S.mip_like(chain[-1]))

        def build_chain():
            for a, b in zip(chain[:-1], chain[1:]):
                S.build_mip(a, b)
        t1 = timeit(lambda: S.build_mip(chain[0], chain[1]))
        tc = timeit(build_chain)
        lvl1_bytes = 6 * ((self.N + 2) ** 2 + (self.N // 2 + 2) ** 2) * 16
        gbs = lvl1_bytes / (t1 * 1e-3) / 1e9
        ex["mip_chain"] = {"level1_ms": round(t1, 4), "chain_ms_7_levels": round(tc, 4),
                           "level1_achieved_GBps": round(gbs, 1),
                           "level1_frac_of_measured_hbm": round(gbs / load_peaks()["hbm_gbs"], 3),
                           "per_unit": "algorithmic 16 B read per fine texel + 16 B written per coarse texel "
                                       "(interior coarse samples: the mean of their four children's stored values; "
                                       "gutter and margin rings: four fine interpolant queries)"}
        del chain
        return ex

    def oracle_measure(self, budget_s, procs, pool=None):
        """Oracle rate projected to one planet step: per-process FD bake rate (N = 128 faces) and query
        rate (2^14 queries), times the process count, applied to 6 x 2050^2 texels + 2^29 queries."""
        with _PoolScope(pool, procs) as pool:
            res = pool.map(_oracle_planet_task, [a + (128, 16384) for a in self.oracle_task_args(procs)])
        texels, tb, q, tq = (np.array([r[i] for r in res], dtype=np.float64) for i in range(4))
        bake_rate = procs * texels.mean() / tb.mean()
        query_rate = procs * q.mean() / tq.mean()
        T = 6 * (self.N + 2) ** 2
        t_step = T / bake_rate + (self.Qr + self.Qc) / query_rate
        return (self.Qr + self.Qc) / t_step, (f"{procs} processes each: FP64 FD bake of an N=128 planet "
                                              f"({bake_rate:.3g} texels/s aggregate) and 16,384 queries "
                                              f"({query_rate:.3g} q/s aggregate), projected to one step")

    def oracle_task_args(self, n, start=0):
        return [("planet", k, self.keys, self.seed) for k in range(start, start + n)]


def planet_leg(args, S, torch):
    """The procedural planet (§4.10) beside the glyph field: N = 2048 f32 texel table (403 MB, out of
    L2), 2^28 uniform random directions through the binned query and through the direct query, and
    2^28 screen-coherent directions through the direct query; per form the time, queries/s, the
    fraction of the measured HBM bandwidth at the paper's 104 B/query accounting and the DRAM bytes
    per query of the committed ncu capture of that form (null once its kernels changed)."""
    import copy
    a = copy.copy(args)
    a.dtype_id, a.layout_id, a.planet_random, a.l2_fetch_granularity = 0, 0, "binned", "64"
    prev = S.l2_fetch_granularity(-1)
    P = Planet(a, 0)
    P.setup(S, torch)
    st = torch.cuda.current_stream()
    peak = load_peaks()["hbm_gbs"]

    def timeit(fn, n=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    def form(ms, q, kernel):
        files = {"binned": ["paper_2602_20063_gb300/csrc/shm_query_binned.cu",
                            "paper_2602_20063_gb300/csrc/shm_device.cuh", "paper_2602_20063_gb300/csrc/shm_stage.cuh"],
                 "direct": ["paper_2602_20063_gb300/csrc/shm_query_kernel.cuh",
                            "paper_2602_20063_gb300/csrc/shm_device.cuh"]}[kernel[0]]
        tr = load_traffic(kernel[1], files)
        return {"ms": round(ms, 4), "queries_per_s": q / (ms * 1e-3),
                "frac_of_measured_hbm_at_104B": round(104 * q / (ms * 1e-3) / 1e9 / peak, 3),
                "dram_bytes_per_query": round(tr / q, 1) if tr else None}

    bake = timeit(P.bake)
    t_bin = timeit(lambda: P.query_random(P.out))
    t_dir = timeit(lambda: S.query(P.lut, P.dr, out=P.out), 3)
    t_coh = timeit(lambda: S.query(P.lut, P.dc, out=P.out), 3)
    # the random half on 16-bit and cell-layout copies of the same table: speed against f32 texel
    storage = {}
    for name, dt, ly in (("f16_texel", S.SHM_F16, S.SHM_LAYOUT_TEXEL), ("bf16_texel", S.SHM_BF16, S.SHM_LAYOUT_TEXEL),
                         ("f32_cell", S.SHM_F32, S.SHM_LAYOUT_CELL), ("f16_cell", S.SHM_F16, S.SHM_LAYOUT_CELL)):
        t = S.like_lut(P.lut, dtype=dt, layout=ly)
        S.pack_lut(P.lut, t)
        ws = S.query_binned_workspace(t, P.Qr)
        tb = timeit(lambda: S.query_binned(t, P.dr, ws, out=P.out), 3)
        del ws
        td = timeit(lambda: S.query(t, P.dr, out=P.out), 3)
        storage[name] = {"table_MB": round(t.data.numel() * t.data.element_size() / 1e6, 1),
                         "random_binned_ms": round(tb, 4), "binned_speedup_vs_f32_texel": round(t_bin / tb, 3),
                         "random_direct_ms": round(td, 4), "direct_speedup_vs_f32_texel": round(t_dir / td, 3)}
        del t
        torch.cuda.empty_cache()
    res = {"workload": P.config["workload"], "random_queries": P.config["random_queries"],
           "l2_fetch_granularity_bytes": 64, "fbm_bake_ms": round(bake, 4),
           "random_binned": form(t_bin, P.Qr, ("binned", "query_random")),
           "random_direct": form(t_dir, P.Qr, ("direct", "planet_random_direct")),
           "coherent_direct": form(t_coh, P.Qc, ("direct", "query_coherent")),
           "random_storage": storage,
           "step_ms": round(bake + t_bin + t_coh, 4),
           "step_queries_per_s": (P.Qr + P.Qc) / ((bake + t_bin + t_coh) * 1e-3),
           "note": "frac at 104 B/query = the paper's per-query bytes (4 corner records + direction + outputs, no "
                   "reuse) over the measured copy bandwidth; the binned form moves fewer DRAM bytes than that "
                   "(dram_bytes_per_query, from the committed ncu capture) because the table is read about once"}
    del P
    S.l2_fetch_granularity(prev)
    torch.cuda.empty_cache()
    return res


def _oracle_planet_task(args):
    """Oracle sample of the planet step: bake Nb faces (rate per texel) and nq queries."""
    kind, k, keys, seed, Nb, nq = args
    import oracle as O
    import shm_inputs as I
    t0 = time.perf_counter()
    samples = O.sample_grid_fbm(Nb, keys, 2.0, 2.0, 0.5, 0.02)
    lut = O.bake_fd(Nb, samples)
    t1 = time.perf_counter()
    pool, off, Ns = O.make_pool([lut])
    d = I.directions_range(k * nq, nq, seed + 11)
    O.query(pool, off, Ns, d, r0=np.array([1.0]), nthreads=1)
    t2 = time.perf_counter()
    return (6 * (Nb + 2) ** 2, t1 - t0, nq, t2 - t1)


class Impostors:
    """Radial depth-map impostors (§4.9): 512 objects R = 1 + sum of 8-64 Gaussian bumps, N from
    {16, 32, 64, 128}, on an 8x8x8 grid (spacing 3) ray cast at 1920x1080 (45 deg FOV, camera on +z
    at the distance where the grid's bounding sphere fills the view).  Step = FD bake of all objects
    + bounds + persistent tile-binned ray cast with Blinn-Phong shading."""
    name = "impostors"
    unit = "pixels/s"

    def __init__(self, args, rank):
        import shm_inputs as I
        self.n = 512
        self.W, self.H = 1920, 1080
        self.seed = 20063 + 2 + 1000 * rank
        self.counts, self.offs, self.mu, self.amp, self.width = I.bump_params(self.n, self.seed)
        self.Ns = I.uneven_N(self.n, self.seed + 1)
        g = (np.arange(8) - 3.5) * 3.0
        self.centres = np.array([[x, y, z] for x in g for y in g for z in g])
        self.config = {"workload": "radial depth-map impostors: 512 bump objects (8-64 Gaussian bumps), N in "
                                   "{16,32,64,128}, 8x8x8 grid spacing 3, ray cast 1920x1080, f32 texel records; "
                                   "step = FD bake + bounds + persistent ray cast (march 32, bisect 12, Newton 3)",
                       "objects": self.n, "W": self.W, "H": self.H, "pixels_per_step": self.W * self.H,
                       "l2": f"table {int(sum(6 * (n + 2) ** 2 for n in self.Ns) * 16 / 1e6)} MB (L2-resident reuse)"}

    def setup(self, S, torch):
        self.S, self.torch = S, torch
        dev = "cuda"
        self.lut = S.alloc_lut(self.n, [int(n) for n in self.Ns], r0=[1.0] * self.n)
        self.src = S.Source(kind=S.SHM_SRC_BUMPS, bump_offset=torch.from_numpy(self.offs).to(dev),
                            mu=torch.from_numpy(self.mu.astype(np.float32)).to(dev),
                            amp=torch.from_numpy(self.amp.astype(np.float32)).to(dev),
                            width=torch.from_numpy(self.width.astype(np.float32)).to(dev))
        S.build_lut(self.lut, self.src)
        rmax = S.lut_bounds(self.lut).cpu().numpy()
        self.R_scene = math.sqrt(3) * 10.5 + float(rmax.max())
        dist = self.R_scene / math.sin(math.radians(22.5))
        eye = np.array([0.0, 0.0, dist])
        fwd = -eye / np.linalg.norm(eye)
        right = np.cross(fwd, [0.0, 1.0, 0.0])
        right /= np.linalg.norm(right)
        up = np.cross(right, fwd)
        self.cam = S.make_camera(eye, fwd, right, up, 45.0, self.W, self.H)
        self.prm = S.make_raycast_params()
        self.rmax = torch.empty(self.n, dtype=torch.float32, device=dev)
        self.objs = S.objects_tensor(self.centres, np.ones(self.n), rmax, np.arange(self.n))
        self.ws = torch.empty(S.raycast_workspace_bytes(self.n, self.W, self.H), dtype=torch.uint8, device=dev)
        self.out = {"rgba": torch.empty((self.H, self.W, 4), device=dev), "depth": torch.empty((self.H, self.W), device=dev),
                    "normal": torch.empty((self.H, self.W, 3), device=dev),
                    "obj_id": torch.empty((self.H, self.W), dtype=torch.int32, device=dev)}
        self.launches_per_step = 5  # FD bake, bounds, rank, bin, ray cast

    def step(self, timer):
        S = self.S
        timer.mark("fd_bake_bumps")
        S.build_lut(self.lut, self.src)
        timer.mark("bounds")
        r = S.lut_bounds(self.lut)
        self.objs.view(self.torch.float32).view(-1, 6)[:, 4].copy_(r)  # object bounding radius from the new table
        timer.mark("raycast")
        S.raycast(self.lut, self.objs, self.n, self.cam, self.prm, ws=self.ws, out=self.out)
        timer.mark("_end")

    def units_per_step(self):
        return self.W * self.H

    def e2e_setup(self):
        torch = self.torch
        self.h_mu = self.src.mu.cpu().pin_memory()
        self.h_amp = self.src.amp.cpu().pin_memory()
        self.h_w = self.src.width.cpu().pin_memory()
        host_out = {"rgba": torch.empty((self.H, self.W, 4)).pin_memory()}
        # two device colour buffers: a frame's image copies back while the next frame renders
        self.rgba2 = [self.out["rgba"], torch.empty_like(self.out["rgba"])]
        self.copy_stream = torch.cuda.Stream()
        self.copy_done = [None, None]
        self.frame = 0
        h2d = (self.h_mu.numel() + self.h_amp.numel() + self.h_w.numel()) * 4
        d2h = self.W * self.H * 16
        return host_out, h2d, d2h

    def e2e_step(self, host_out):
        """One frame through the public API: the bump parameters come from page-locked host memory,
        the objects are baked and bounded, the frame is ray cast into one of two colour buffers and
        copied back on a second stream while the next frame renders.  A step ends when the previous
        frame's image has landed, so one image copy is timed per step."""
        torch = self.torch
        main = torch.cuda.current_stream()
        b = self.frame % 2
        if self.copy_done[b] is not None:
            main.wait_event(self.copy_done[b])  # this buffer's last image has been read back
        self.src.mu.copy_(self.h_mu, non_blocking=True)
        self.src.amp.copy_(self.h_amp, non_blocking=True)
        self.src.width.copy_(self.h_w, non_blocking=True)
        self.S.build_lut(self.lut, self.src)
        self.objs.view(torch.float32).view(-1, 6)[:, 4].copy_(self.S.lut_bounds(self.lut))
        out = dict(self.out, rgba=self.rgba2[b])
        self.S.raycast(self.lut, self.objs, self.n, self.cam, self.prm, ws=self.ws, out=out)
        self.copy_stream.wait_stream(main)
        with torch.cuda.stream(self.copy_stream):
            host_out["rgba"].copy_(self.rgba2[b], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.copy_stream)
        self.copy_done[b] = ev
        prev = self.copy_done[1 - b]
        if prev is not None:
            main.wait_event(prev)
        self.frame += 1

    def roofline_terms(self, peaks, ktot, sms):
        """The ray cast is bound by instruction issue (SIMT root finding, DRAM ~5 %): its roofline is
        the issue-slot ceiling, SMs x 4 schedulers x one warp instruction per clock at the maximum SM
        clock, against the warp instructions of one k_raycast launch counted by the committed ncu
        capture (same source only; the timed region also holds the rank and bin kernels)."""
        files = ["paper_2602_20063_gb300/csrc/shm_raycast.cu", "paper_2602_20063_gb300/csrc/shm_device.cuh"]
        p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
        e = json.load(open(p)).get("raycast") if os.path.exists(p) else None
        if not e or e.get("source_hash") != source_hash(*files):
            return {}
        ceiling = sms * 4 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # T warp instructions/s
        return {"raycast": {"bound": "alu", "algorithmic": float(e["warp_instructions_per_launch"]),
                            "unit": "T warp-inst/s", "peak": ceiling, "files": files,
                            "per_unit": "warp instructions of the frame's ray cast (9.8 surface queries per pixel)"}}

    def extras(self, S, torch, steps):
        """Surface queries per frame, and the ray cast alone with fixed refinement counts against
        refinement by projected size (§3.1; bisection 8-16, Newton 2-4 as in the paper)."""
        st = torch.cuda.current_stream()

        def timed(prm, n=5):
            S.raycast(self.lut, self.objs, self.n, self.cam, prm, ws=self.ws, out=self.out)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(n):
                S.raycast(self.lut, self.objs, self.n, self.cam, prm, ws=self.ws, out=self.out)
            e1.record(st)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / n, S.raycast_query_count(self.ws)

        ms_fixed, nq = timed(self.prm)
        hit = float((self.out["obj_id"] >= 0).float().mean())
        depth_fixed = self.out["depth"].clone()
        lod = S.make_raycast_params(bisect=16, newton=4, lod=1, bisect_min=8, newton_min=2)
        ms_lod, nq_lod = timed(lod)
        both = torch.isfinite(depth_fixed) & torch.isfinite(self.out["depth"])
        ddepth = float(((self.out["depth"] - depth_fixed).abs() / depth_fixed)[both].max()) if both.any() else 0.0
        return {"surface_queries_per_frame": nq, "hit_fraction": hit,
                "raycast_fixed": {"ms": round(ms_fixed, 4), "surface_queries": nq,
                                  "params": "march 32, bisect 12, Newton 3 for every object"},
                "raycast_lod": {"ms": round(ms_lod, 4), "surface_queries": nq_lod,
                                "params": "march 32, bisect 8-16 (march 2^b >= 128 p), Newton 4 from 64 px else 2",
                                "max_rel_depth_change_vs_fixed": ddepth}}

    def oracle_measure(self, budget_s, procs, pool=None):
        """Oracle rate projected to one impostor step: FP64 FD bake of the 512 objects (spawned
        processes) then the oracle ray cast of random pixels (OpenMP over all cores).  The first call
        bakes every object; later calls (the reference arm's steps) re-bake a budget-sized subset of
        the objects and cast a budget-sized set of pixels, each projected to the whole step."""
        import oracle as O
        args = [(int(self.Ns[o]), self.mu[self.offs[o]:self.offs[o + 1]], self.amp[self.offs[o]:self.offs[o + 1]],
                 self.width[self.offs[o]:self.offs[o + 1]]) for o in range(self.n)]
        first = getattr(self, "_oracle_luts", None) is None
        frac = 1.0
        with _PoolScope(pool, procs) as pool:
            if first:
                t0 = time.perf_counter()
                self._oracle_luts = pool.map(_oracle_bump_bake, args)
                t_bake = time.perf_counter() - t0
                self._oracle_t_bake = t_bake
            else:
                frac = min(1.0, max(procs / self.n, 0.5 * budget_s / max(self._oracle_t_bake, 1e-3)))
                m = max(1, int(round(frac * self.n)))
                t0 = time.perf_counter()
                pool.map(_oracle_bump_bake, args[:m])
                t_bake = (time.perf_counter() - t0) * self.n / m
        luts = self._oracle_luts
        pool_, off, Ns = O.make_pool(luts)
        rmax = np.array([O.lut_bound(l, int(n), 1.0) for l, n in zip(luts, Ns)])
        R_scene = math.sqrt(3) * 10.5 + float(rmax.max())
        dist = R_scene / math.sin(math.radians(22.5))
        eye = np.array([0.0, 0.0, dist])
        fwd = -eye / dist
        right = np.cross(fwd, [0.0, 1.0, 0.0])
        right /= np.linalg.norm(right)
        up = np.cross(right, fwd)
        cam = O.make_camera(eye, fwd, right, up, 45.0, self.W, self.H)
        rng = np.random.default_rng(1)
        npx = max(16, int(256 * frac))
        px = rng.integers(0, self.W, npx).astype(np.int32)
        py = rng.integers(0, self.H, npx).astype(np.int32)
        t0 = time.perf_counter()
        O.raycast(pool_, off, Ns, self.centres, np.ones(self.n), rmax, np.arange(self.n), cam,
                  O.make_raycast_params(), px=px, py=py, r0=np.ones(self.n), nthreads=procs)
        t_ray = (time.perf_counter() - t0) * (self.W * self.H) / npx
        return self.W * self.H / (t_bake + t_ray), (f"FP64 bake of {'all 512' if first else 'a subset of the 512'} objects "
                                                    f"({t_bake:.1f} s projected, {procs} processes) + "
                                                    f"oracle ray cast of {npx} random pixels ({procs} threads) "
                                                    f"projected to 1920x1080")

    def oracle_task_args(self, n, start=0):
        return []


def _oracle_bump_bake(args):
    N, mu, amp, width = args
    import oracle as O
    return O.bake_fd(N, O.sample_grid_bumps(N, mu, amp, width), r0=1.0)


class Fit:
    """Differentiable table fit: 1,024 glyphs at N = 64 (428 MB of float32 table parameters) fitted by
    Adam to direct-SH targets of degree L = 16 (value + normal MSE) at 2^24 directions per step
    (16,384 per glyph, resampled per step from a pool of direction sets whose targets are evaluated
    before timing).  Step = fused forward + loss + adjoint (shm_fit_backward) + Adam."""
    name = "fit"
    unit = "queries/s"

    def __init__(self, args, rank):
        import shm_inputs as I
        self.G, self.N, self.L, self.per = 1024, 64, 16, 16384
        self.Q = self.G * self.per
        self.n_sets = 4
        self.seed = 20063 + 4 + 1000 * rank
        self.coeffs = I.sh_coeffs(self.G, self.L, self.seed).astype(np.float32)
        self.config = {"workload": "differentiable fit: 1024 glyphs, N = 64, f32 table parameters, Adam (lr 1e-2), "
                                   "targets direct SH L = 16, value + normal MSE, 2^24 directions per step; "
                                   "step = fused forward + loss + adjoint + Adam",
                       "glyphs": self.G, "N": self.N, "L_target": self.L, "queries_per_step": self.Q,
                       "l2": "inputs larger than L2 (table + Adam state 1.7 GB, directions 201 MB per set)"}

    def setup(self, S, torch):
        import shm_inputs as I
        self.S, self.torch = S, torch
        dev = "cuda"
        self.lut = S.alloc_lut(self.G, self.N, zero=True)
        self.lut.data.view(self.G, -1, 4)[:, :, 0] = torch.from_numpy(self.coeffs[:, 0] * 0.28209479177387814).to(dev)[:, None]
        self.m = torch.zeros_like(self.lut.data)
        self.v = torch.zeros_like(self.lut.data)
        self.dl = S.like_lut(self.lut, zero=True)
        self.seg = torch.from_numpy(I.query_glyphs_csr(self.G, self.per)).to(dev)
        cdev = torch.from_numpy(self.coeffs).to(dev)
        self.sets = []
        for k in range(self.n_sets):
            d = torch.from_numpy(I.directions(self.Q, self.seed + 100 + k)).to(dev)
            Rt, _, nt = S.sh_eval(self.L, cdev, d, seg=self.seg)
            self.sets.append((d, Rt, nt))
        self.loss = torch.zeros(1, device=dev)
        self.k = 0
        self.out = {k: torch.empty(s, dtype=torch.float32, device=dev)
                    for k, s in (("R", (self.Q,)), ("grad", (self.Q, 3)), ("normal", (self.Q, 3)))}
        self.launches_per_step = 2

    def step(self, timer):
        d, Rt, nt = self.sets[self.k % self.n_sets]
        self.k += 1
        timer.mark("fit_fwd_loss_bwd")
        self.S.fit_backward(self.lut, d, Rt, nt, self.dl, 1.0, 1.0, loss=self.loss, seg=self.seg)
        timer.mark("adam")
        self.S.adam_step(self.lut.data, self.dl.data, self.m, self.v, lr=1e-2, step=self.k)
        timer.mark("_end")

    def units_per_step(self):
        return self.Q

    def e2e_setup(self):
        torch = self.torch
        self.hsets = [(d.cpu().pin_memory(), R.cpu().pin_memory(), n.cpu().pin_memory()) for d, R, n in self.sets]
        host_out = {"loss": torch.empty(1).pin_memory()}
        self.copy_stream = torch.cuda.Stream()
        self.copied = [None] * self.n_sets  # event: that set's host-to-device copy is done
        d, R, n = self.sets[0]
        return host_out, (d.numel() + R.numel() + n.numel()) * 4, 4

    def _copy_set(self, i, stream):
        d, Rt, nt = self.sets[i]
        hd, hR, hn = self.hsets[i]
        with self.torch.cuda.stream(stream):
            d.copy_(hd, non_blocking=True)
            Rt.copy_(hR, non_blocking=True)
            nt.copy_(hn, non_blocking=True)
            ev = self.torch.cuda.Event()
            ev.record(stream)
        self.copied[i] = ev

    def e2e_step(self, host_out):
        """One training step from page-locked host memory, as a data loader would run it: this
        step's directions and targets arrived over the host link while the previous step computed
        (a second stream; the first step copies its own), the fused forward + loss + adjoint and
        Adam run while the next step's inputs copy, and the loss comes back."""
        torch = self.torch
        main = torch.cuda.current_stream()
        i, j = self.k % self.n_sets, (self.k + 1) % self.n_sets
        if self.copied[i] is None:
            self._copy_set(i, main)
        main.wait_event(self.copied[i])
        self.copied[i] = None
        # set j was last read three steps ago; the copy stream starts after this step's start
        self.copy_stream.wait_stream(main)
        self._copy_set(j, self.copy_stream)
        d, Rt, nt = self.sets[i]
        self.loss.zero_()
        self.k += 1
        self.S.fit_backward(self.lut, d, Rt, nt, self.dl, 1.0, 1.0, loss=self.loss, seg=self.seg)
        self.S.adam_step(self.lut.data, self.dl.data, self.m, self.v, lr=1e-2, step=self.k)
        host_out["loss"].copy_(self.loss, non_blocking=True)
        # the step ends when the next step's inputs have landed too: one copy per step is timed
        main.wait_stream(self.copy_stream)

    def roofline_terms(self, peaks, ktot, sms):
        T = 6 * (self.N + 2) ** 2
        tab = self.G * T * 16
        return {
            "fit_fwd_loss_bwd": {"bound": "hbm", "algorithmic": self.Q * (12 + 16 + 64) + 2 * tab, "unit": "GB/s",
                                 "peak": peaks["hbm_gbs"],
                                 "per_unit": "12 B direction + 16 B targets + 64 B table reads per query, plus the "
                                             "gradient table read-modify-written once (atomics hit L2)",
                                 "files": ["paper_2602_20063_gb300/csrc/shm_query_bwd.cu"]},
            "adam": {"bound": "hbm", "algorithmic": tab * 8, "unit": "GB/s", "peak": peaks["hbm_gbs"],
                     "per_unit": "param, grad, m, v read + param, m, v written + grad zeroed for the next step: "
                                 "32 B per scalar",
                     "files": ["paper_2602_20063_gb300/csrc/shm_query_bwd.cu"]},
        }

    def extras(self, S, torch, steps):
        """Plain forward on the same queries, fwd+bwd/fwd ratio, and the fitted error."""
        st = torch.cuda.current_stream()
        d, Rt, nt = self.sets[0]

        def timeit(fn, n=5):
            fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(n):
                fn()
            e1.record(st)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / n

        fwd = timeit(lambda: S.query(self.lut, d, seg=self.seg, out=self.out))
        fb = timeit(lambda: S.fit_backward(self.lut, d, Rt, nt, self.dl, 1.0, 1.0, loss=self.loss, seg=self.seg))
        S.query(self.lut, d, seg=self.seg, out=self.out)
        eR = float((self.out["R"] - Rt).abs().max())
        nerr = torch.rad2deg(torch.acos(torch.clamp((self.out["normal"] * nt).sum(1), -1, 1)))
        return {"fwd_ms": round(fwd, 4), "fused_fwd_loss_bwd_ms": round(fb, 4),
                "fwd_bwd_over_fwd": round(fb / fwd, 3), "steps_taken": self.k,
                "max_abs_err_R_after_steps": eR, "mean_normal_err_deg": float(nerr.mean()),
                "note": "error of the fitted tables against the L = 16 targets after the warm-up + timed steps"}

    def oracle_measure(self, budget_s, procs, pool=None):
        """Oracle rate: FP64 loss + adjoint of 4,096 queries on one N = 64 glyph per process, plus Adam
        over that glyph's table, projected to one step (1,024 glyphs, 2^24 queries)."""
        nq = 4096  # queries per process
        with _PoolScope(pool, procs) as pool:
            res = pool.map(_oracle_fit_task, [(k, self.coeffs[k], self.seed, nq) for k in range(procs)])
        tq = np.mean([r[0] for r in res]) / nq
        ta = np.mean([r[1] for r in res])
        t_step = (self.Q * tq + self.G * ta) / procs
        return self.Q / t_step, (f"{procs} processes each: FP64 loss + adjoint of {nq:,} queries and Adam over one "
                                 "N = 64 glyph table, projected to 2^24 queries + 1,024 tables")

    def oracle_task_args(self, n, start=0):
        return []


def _oracle_fit_task(args):
    k, c, seed, nq = args
    import oracle as O
    import oracle.fit as OF
    import shm_inputs as I
    N, L = 64, 16
    lut = np.zeros((6, N + 2, N + 2, 4))
    lut[..., 0] = c[0] * 0.28209479177387814
    pool, off, Ns = O.make_pool([lut])
    d = I.directions_range(k * nq, nq, seed + 100)
    Rt, _, nt = O.sh_eval(L, c.astype(np.float64), d, nthreads=1)
    t0 = time.perf_counter()
    loss, g = OF.loss_and_grad(pool, off, Ns, d, Rt, nt)
    t1 = time.perf_counter()
    OF.adam(pool, g, np.zeros_like(pool), np.zeros_like(pool), 1, 1e-2)
    t2 = time.perf_counter()
    return (t1 - t0, t2 - t1)


WORKLOADS = {"glyphs": GlyphField, "planet": Planet, "impostors": Impostors, "fit": Fit}


# ----------------------------------------------------------------------------------- arms
def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    work = WORKLOADS[args.workload](args, 0)
    procs = os.cpu_count() or 1
    # one spawned pool for the whole run; each step a sample of about steps_s seconds, so that the
    # warm-up and timed steps together take about two minutes
    steps_s = min(10.0, max(0.1, 120.0 / max(1, args.steps + args.warmup)))
    rates, times = [], []
    pool = _spawn_pool(procs)
    try:
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            v, sample = work.oracle_measure(steps_s, procs, pool=pool)
            dt = time.perf_counter() - t0
            if k >= args.warmup:
                rates.append(v)
                times.append(dt)
    finally:
        pool.close()
        pool.join()
    value = statistics.median(rates)
    sample = "each step: " + sample
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": work.unit, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * work.units_per_step() / value,
            "ms_per_step_basis": "projected: one whole step's units divided by the sampled rate; each timed step "
                                 "runs a bounded sample of the step, not the whole step",
            "sample_wall_ms_per_step": round(1e3 * statistics.median(times), 1),
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
        if hasattr(work, "oracle_truth") and not args.no_extras:
            # the same leg evaluates the float64 ground truth that extras.precision compares against
            work.truth = work.oracle_truth(os.cpu_count() or 1)

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
        ms = reduce_over_ranks(ms, dist, "cuda")
        dist.barrier()
    clk = clocks.stop()
    timer.active = False
    ktot = timer.totals()
    ms_step = ms / args.steps
    value = whole_job_rate(work.units_per_step(), world, ms_step)

    # ---- end to end through the public API from pinned host memory: E2E_WARMUP untimed steps, then
    # E2E_REPEATS windows of E2E_STEPS steps each (independent of --steps); the median window counts
    # (a window's begin / end hooks let a pipelined step overlap the next one inside the window:
    # the start event precedes every stream's first copy, the end event follows every last one)
    host_out, h2d, d2h = work.e2e_setup()
    begin, end = getattr(work, "e2e_begin", lambda: None), getattr(work, "e2e_end", lambda: None)
    begin()
    for _ in range(E2E_WARMUP):
        work.e2e_step(host_out)
    end()
    torch.cuda.synchronize()
    n_e2e = getattr(work, "e2e_steps", E2E_STEPS)
    windows = []
    for _ in range(E2E_REPEATS):
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        begin()
        for _ in range(n_e2e):
            work.e2e_step(host_out)
        end()
        a1.record(stream)
        torch.cuda.synchronize()
        windows.append(a0.elapsed_time(a1) / n_e2e)
    e2e_ms = statistics.median(windows)
    link = host_link_probe(torch)
    if world > 1:
        e2e_ms = reduce_over_ranks(e2e_ms, dist, "cuda")

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
                           (" hbm_gbs" if dk.get("unit") == "GB/s" else
                            " issue slots from unit counts x max clock" if dk.get("unit") == "T warp-inst/s" else
                            " FP32 SIMT from unit counts x max clock")}
    extras = {} if args.no_extras else work.extras(S, torch, args.steps)
    if extras:
        # the copy bandwidth behind every "frac_of_measured_hbm*" figure above, and where it came from
        extras["hbm_peak_used"] = {"GBps": peaks["hbm_gbs"], "source": peaks["_source"]}
    line = {"metric": METRIC, "value": value, "unit": work.unit, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": ["f32", "f16", "bf16"][args.dtype_id], "data": "synthetic",
            "config": dict(work.config, parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": world * work.units_per_step() / (e2e_ms * 1e-3), "unit": work.unit,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "host_link_GBps": round((h2d + d2h) / (e2e_ms * 1e-3) / 1e9, 1),
                    "mode": getattr(work, "e2e_mode", "copies"),
                    "pipeline": getattr(work, "e2e_note", None),
                    "timing": f"{E2E_WARMUP} warm-up steps, then the median of {E2E_REPEATS} windows of {n_e2e} steps "
                              f"(window ms per step: {', '.join(f'{w:.3f}' for w in windows)})",
                    "host_link_probe": link,
                    "frac_of_host_link_probe": round((h2d + d2h) / (e2e_ms * 1e-3) / 1e9 / link["both_GBps"], 3)},
            "gpu_launches": work.launches_per_step * args.steps, "clocks": clk, "kernels": kernels,
            "extras": extras}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def parse_args(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["shm", "reference"], default="shm")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="glyphs")
    ap.add_argument("--dtype", choices=["f32", "f16", "bf16"], default="f32")
    ap.add_argument("--layout", choices=["texel", "cell"], default="texel")
    ap.add_argument("--engine", choices=["tcgen05", "simt"], default="tcgen05", help="SH bake contraction engine")
    ap.add_argument("--glyphs", type=int, default=16384)
    ap.add_argument("--per-glyph", type=int, default=4096)
    ap.add_argument("--planet-queries", type=int, default=1 << 28)
    ap.add_argument("--planet-random", choices=["binned", "direct"], default="binned",
                    help="planet: random queries through shm_query_binned (default) or shm_query in query order")
    ap.add_argument("--planet-band-bytes", type=int, default=0,
                    help="planet: table bytes per partition band of the binned query (0 = library default)")
    ap.add_argument("--l2-fetch-granularity", default="auto",
                    help="planet: L2 fetch granularity in bytes for the process's context, or auto")
    ap.add_argument("--cpu-budget", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--e2e-chunks", type=int, default=16,
                    help="glyph field end to end: glyph chunks per step (copies and kernels of neighbouring chunks overlap)")
    ap.add_argument("--e2e-streams", type=int, default=1,
                    help="glyph field end to end: kernel streams the chunks rotate over (copies: one stream per direction)")
    ap.add_argument("--e2e-mode", choices=["zero_copy", "copy_pipeline"], default="copy_pipeline",
                    help="glyph field end to end: kernels on page-locked host buffers, or chunked copies")
    args = ap.parse_args(argv)
    args.dtype_id = {"f32": 0, "f16": 1, "bf16": 2}[args.dtype]
    args.layout_id = {"texel": 0, "cell": 1}[args.layout]
    return args


def main():
    args = parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
