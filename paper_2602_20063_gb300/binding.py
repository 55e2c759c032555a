"""Thin Python binding of libshm.so (include/shm.h): the same entry points, argument marshalling only.

Every computation runs in the CUDA library; PyTorch only provides device memory and the current
stream.  Importing this module does not load the library; the first call does, and raises
``RuntimeError`` if libshm.so has not been built (``python -c "import __graft_entry__ as g;
g.build()"``).  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Optional

import torch

from . import build as _build

SHM_F32, SHM_F16, SHM_BF16 = 0, 1, 2
SHM_LAYOUT_TEXEL, SHM_LAYOUT_CELL, SHM_LAYOUT_VALUE = 0, 1, 2
SHM_RECON_NEAREST, SHM_RECON_BILINEAR, SHM_RECON_BICUBIC, SHM_RECON_FAST_BICUBIC = 0, 1, 2, 3
SHM_SRC_SH, SHM_SRC_SAMPLES, SHM_SRC_BUMPS, SHM_SRC_FBM = 0, 1, 2, 3
SHM_DEV_NONFINITE, SHM_DEV_BOUNDS, SHM_DEV_TIMEOUT = 1, 2, 4
SHM_BWD_DETERMINISTIC = 1
SHM_BWD_CUDA_CORES = 2
STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported", 3: "workspace", 4: "cuda error", 5: "timeout"}

DTYPES = {SHM_F32: torch.float32, SHM_F16: torch.float16, SHM_BF16: torch.bfloat16}
DTYPE_NAMES = {"f32": SHM_F32, "f16": SHM_F16, "bf16": SHM_BF16}
LAYOUT_NAMES = {"texel": SHM_LAYOUT_TEXEL, "cell": SHM_LAYOUT_CELL, "value": SHM_LAYOUT_VALUE}


class ShmError(RuntimeError):
    pass


class c_lut(C.Structure):
    _fields_ = [("n_glyphs", C.c_int32), ("dtype", C.c_int32), ("layout", C.c_int32), ("N_uniform", C.c_int32),
                ("N", C.c_void_p), ("offset", C.c_void_p), ("r0", C.c_void_p), ("data", C.c_void_p)]


class c_source(C.Structure):
    _fields_ = [("kind", C.c_int32), ("L", C.c_int32), ("coeffs", C.c_void_p), ("basis", C.c_void_p),
                ("samples", C.c_void_p), ("sample_offset", C.c_void_p), ("bump_offset", C.c_void_p),
                ("mu", C.c_void_p), ("amp", C.c_void_p), ("width", C.c_void_p), ("octaves", C.c_int32),
                ("keys", C.c_void_p), ("base_freq", C.c_float), ("lacunarity", C.c_float), ("gain", C.c_float),
                ("amplitude", C.c_float), ("dev_status", C.c_void_p)]


class c_camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("fwd", C.c_float * 3), ("right", C.c_float * 3), ("up", C.c_float * 3),
                ("tan_half_fov_y", C.c_float), ("W", C.c_int32), ("H", C.c_int32)]


class c_raycast_params(C.Structure):
    _fields_ = [("march", C.c_int32), ("bisect", C.c_int32), ("newton", C.c_int32), ("ambient", C.c_float),
                ("kd", C.c_float), ("ks", C.c_float), ("shininess", C.c_float), ("light", C.c_float * 3),
                ("lod", C.c_int32), ("bisect_min", C.c_int32), ("newton_min", C.c_int32), ("recon", C.c_int32)]


class c_object(C.Structure):
    _fields_ = [("centre", C.c_float * 3), ("scale", C.c_float), ("rmax", C.c_float), ("glyph", C.c_int32)]


_lib = None

_VP, _I32, _I64, _SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
_SIGS = {
    "shm_records_per_glyph": (C.c_int64, [_I32, _I32]),
    "shm_record_bytes": (C.c_int64, [_I32, _I32]),
    "shm_lut_layout": (C.c_int, [_I32, _VP, _I32, _I32, _VP, _VP]),
    "shm_query": (C.c_int, [_VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "shm_query_recon": (C.c_int, [_VP, _I32, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "shm_tune_query": (C.c_int, [_VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _I32, _VP, _VP, _VP]),
    "shm_tune_reset": (C.c_int, []),
    "shm_query_binned_workspace_bytes": (C.c_int64, [_VP, _I64, _I64]),
    "shm_query_binned_bins": (C.c_int32, [_VP, _I64, C.POINTER(C.c_int32)]),
    "shm_query_binned": (C.c_int, [_VP, _I64, _VP, _VP, _VP, _VP, _VP, _I64, _VP, _SZ, _VP, _VP]),
    "shm_sh_basis_bytes": (C.c_int64, [_I32, _I32]),
    "shm_sh_basis": (C.c_int, [_I32, _I32, _VP, _VP]),
    "shm_build_lut": (C.c_int, [_VP, _VP, _VP, _SZ, _VP]),
    "shm_build_workspace_bytes": (C.c_int64, [_VP, _VP]),
    "shm_pack_lut": (C.c_int, [_VP, _VP, _VP]),
    "shm_lut_bounds": (C.c_int, [_VP, _VP, _VP]),
    "shm_build_mip": (C.c_int, [_VP, _VP, _VP, _VP]),
    "shm_query_backward": (C.c_int, [_VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, C.c_uint32, _VP, _VP]),
    "shm_build_lut_backward": (C.c_int, [_VP, _I32, _VP, _VP, C.c_uint32, _VP]),
    "shm_fit_backward": (C.c_int, [_VP, _I64, _VP, _VP, _VP, _VP, _VP, C.c_float, C.c_float, _VP, _VP, _VP, _VP]),
    "shm_adam_step": (C.c_int, [_VP, _VP, _VP, _VP, _I64, C.c_float, C.c_float, C.c_float, C.c_float, _I32, _I32, _VP]),
    "shm_sh_eval": (C.c_int, [_I32, _I32, _VP, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "shm_raycast_workspace_bytes": (C.c_int64, [_I32, _I32, _I32]),
    "shm_raycast": (C.c_int, [_VP, _VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _SZ, _VP, _VP]),
    "shm_raycast_noalloc": (C.c_int, [_VP, _VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "shm_l2_fetch_granularity": (C.c_int, [_I32, C.POINTER(C.c_int32)]),
    "shm_status_string": (C.c_char_p, [C.c_int]),
    "shm_version": (C.c_int32, []),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libshm.so (raises RuntimeError if it has not been built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libshm.so not found at {path}: build it with paper_2602_20063_gb300.build.build() "
                               "(nvcc, sm_103a); there is no CPU fallback")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(st: int, what: str):
    if st != 0:
        raise ShmError(f"{what}: {lib().shm_status_string(st).decode()} (status {st})")


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    return C.c_void_p(t.data_ptr())


def _io_ptr(t: Optional[torch.Tensor]):
    """Pointer of a per-query buffer: device memory, or host memory handed to the library, which
    accepts page-locked host buffers and refuses pageable ones (SHM_ERR_INVALID_ARG)."""
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _io_empty(shape, dtype, like: torch.Tensor) -> torch.Tensor:
    """An output buffer next to `like`: on its device, or page-locked host memory when `like` is
    page-locked host memory (the kernels write it directly)."""
    if like.device.type == "cpu":
        return torch.empty(shape, dtype=dtype, pin_memory=True)
    return torch.empty(shape, dtype=dtype, device=like.device)


def _need(t: Optional[torch.Tensor], dtype, shape=None, name="tensor"):
    if t is None:
        return
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")


# ------------------------------------------------------------------------------------------- tables
def records_per_glyph(N: int, layout: int) -> int:
    return int(lib().shm_records_per_glyph(int(N), int(layout)))


def record_bytes(dtype: int, layout: int) -> int:
    return int(lib().shm_record_bytes(int(dtype), int(layout)))


def records_per_glyph_host(N: int, layout: int) -> int:
    P = N + 1 if layout == SHM_LAYOUT_CELL else (N + 4 if layout == SHM_LAYOUT_VALUE else N + 2)
    return 6 * P * P


@dataclass
class Lut:
    """A pool of per-glyph tables on the device (see shm_lut in include/shm.h)."""
    data: torch.Tensor
    n_glyphs: int
    dtype: int = SHM_F32
    layout: int = SHM_LAYOUT_TEXEL
    N_uniform: int = 0
    N: Optional[torch.Tensor] = None       # int32 [G]
    offset: Optional[torch.Tensor] = None  # int64 [G]
    r0: Optional[torch.Tensor] = None      # float32 [G]
    _c: c_lut = field(default=None, repr=False)

    def c(self) -> c_lut:
        s = c_lut()
        s.n_glyphs, s.dtype, s.layout, s.N_uniform = self.n_glyphs, self.dtype, self.layout, self.N_uniform
        s.N = self.N.data_ptr() if self.N is not None else None
        s.offset = self.offset.data_ptr() if self.offset is not None else None
        s.r0 = self.r0.data_ptr() if self.r0 is not None else None
        s.data = self.data.data_ptr()
        self._c = s
        return s

    def glyph_N(self, g: int) -> int:
        return self.N_uniform if self.N_uniform > 0 else int(self.N[g])


def alloc_lut(n_glyphs: int, N, dtype: int = SHM_F32, layout: int = SHM_LAYOUT_TEXEL, r0=None, device="cuda",
              zero: bool = False) -> Lut:
    """Allocate a table pool: N is an int (uniform) or a sequence of per-glyph resolutions."""
    rb = 16 if dtype == SHM_F32 else 8
    if layout == SHM_LAYOUT_CELL:
        rb *= 4
    elif layout == SHM_LAYOUT_VALUE:
        rb //= 4
    elem = 4 if dtype == SHM_F32 else 2
    if isinstance(N, int):
        Ns = None
        total = n_glyphs * records_per_glyph_host(N, layout)
        N_uniform, Nt, Ot = N, None, None
    else:
        Ns = [int(n) for n in N]
        assert len(Ns) == n_glyphs
        offs, total = [], 0
        for n in Ns:
            offs.append(total)
            total += records_per_glyph_host(n, layout)
        N_uniform = 0
        Nt = torch.tensor(Ns, dtype=torch.int32, device=device)
        Ot = torch.tensor(offs, dtype=torch.int64, device=device)
    n_elem = total * rb // elem
    alloc = torch.zeros if zero else torch.empty
    data = alloc(n_elem, dtype=DTYPES[dtype], device=device)
    r0t = None
    if r0 is not None:
        r0t = torch.as_tensor(r0, dtype=torch.float32, device=device).reshape(-1).contiguous()
        if r0t.numel() == 1 and n_glyphs > 1:
            r0t = r0t.expand(n_glyphs).contiguous()
    return Lut(data=data, n_glyphs=n_glyphs, dtype=dtype, layout=layout, N_uniform=N_uniform, N=Nt, offset=Ot, r0=r0t)


def like_lut(L: Lut, dtype: int = None, layout: int = None, r0="same", zero=False) -> Lut:
    """A table with L's glyphs and resolutions in another dtype/layout."""
    dtype = L.dtype if dtype is None else dtype
    layout = L.layout if layout is None else layout
    if L.N_uniform > 0:
        N = L.N_uniform
    else:
        N = [int(n) for n in L.N.tolist()]
    rr = (L.r0 if isinstance(r0, str) else r0)
    out = alloc_lut(L.n_glyphs, N, dtype, layout, r0=None, device=L.data.device, zero=zero)
    if rr is not None:
        out.r0 = torch.as_tensor(rr, dtype=torch.float32, device=L.data.device).reshape(-1).contiguous()
    return out


# ------------------------------------------------------------------------------------------- query
def query(lut: Lut, dirs: torch.Tensor, glyph: torch.Tensor = None, seg: torch.Tensor = None,
          want=("R", "grad", "normal"), out: dict = None, dev_status: torch.Tensor = None, stream=None) -> dict:
    """shm_query: returns a dict of the requested outputs among R, grad, normal, chart, fij."""
    _need(dirs, torch.float32, name="dirs")
    Q = dirs.shape[0]
    _need(glyph, torch.int32, (Q,), "glyph")
    _need(seg, torch.int64, (lut.n_glyphs + 1,), "seg")
    out = {} if out is None else out
    shapes = {"R": (Q,), "grad": (Q, 3), "normal": (Q, 3), "chart": (Q, 2), "fij": (Q, 3)}
    for k in want:
        if k not in out:
            out[k] = _io_empty(shapes[k], torch.int32 if k == "fij" else torch.float32, dirs)
    st = lib().shm_query(C.byref(lut.c()), Q, _io_ptr(dirs), _io_ptr(glyph), _io_ptr(seg), _io_ptr(out.get("R")),
                         _io_ptr(out.get("grad")), _io_ptr(out.get("normal")), _io_ptr(out.get("chart")),
                         _io_ptr(out.get("fij")), _io_ptr(dev_status), _stream(stream))
    _check(st, "shm_query")
    return out


def query_binned_workspace_bytes(lut: Lut, Q: int, band_bytes: int = 0) -> int:
    """shm_query_binned_workspace_bytes (raises ShmError for an unsupported table)."""
    n = int(lib().shm_query_binned_workspace_bytes(C.byref(lut.c()), int(Q), int(band_bytes)))
    if n < 0:
        raise ShmError("shm_query_binned_workspace_bytes: unsupported table (uniform resolution needed)")
    return n


def query_binned_workspace(lut: Lut, Q: int, band_bytes: int = 0, device="cuda") -> torch.Tensor:
    """Device workspace for shm_query_binned on Q queries (uint8, 256-byte aligned by the allocator)."""
    return torch.empty(max(query_binned_workspace_bytes(lut, Q, band_bytes), 1), dtype=torch.uint8, device=device)


def query_binned_bins(lut: Lut, band_bytes: int = 0) -> dict:
    """shm_query_binned_bins: bins (6 faces x bands) and cell rows per band for this table."""
    rows = C.c_int32(0)
    B = int(lib().shm_query_binned_bins(C.byref(lut.c()), int(band_bytes), C.byref(rows)))
    if B < 0:
        raise ShmError("shm_query_binned_bins: unsupported table")
    return {"bins": B, "band_rows": rows.value}


def query_binned(lut: Lut, dirs: torch.Tensor, ws: torch.Tensor, band_bytes: int = 0,
                 want=("R", "grad", "normal"), out: dict = None, dev_status: torch.Tensor = None,
                 stream=None) -> dict:
    """shm_query_binned: every query on glyph 0 of a uniform-resolution table, partitioned by table
    region on the device so that the regions in flight stay in L2; outputs (R, grad, normal, chart)
    in query order, equal to shm_query's.  ws from query_binned_workspace(lut, Q, band_bytes)."""
    _need(dirs, torch.float32, name="dirs")
    Q = dirs.shape[0]
    out = {} if out is None else out
    shapes = {"R": (Q,), "grad": (Q, 3), "normal": (Q, 3), "chart": (Q, 2)}
    for k in want:
        if k not in out:
            out[k] = _io_empty(shapes[k], torch.float32, dirs)
    st = lib().shm_query_binned(C.byref(lut.c()), Q, _io_ptr(dirs), _io_ptr(out.get("R")), _io_ptr(out.get("grad")),
                                _io_ptr(out.get("normal")), _io_ptr(out.get("chart")), int(band_bytes), _ptr(ws),
                                ws.numel() * ws.element_size(), _io_ptr(dev_status), _stream(stream))
    _check(st, "shm_query_binned")
    return out


# ------------------------------------------------------------------------------------------- bake
def tune_query(lut: Lut, dirs: torch.Tensor, glyph: torch.Tensor = None, seg: torch.Tensor = None, reps: int = 3,
               stream=None) -> dict:
    """shm_tune_query: time the launch shapes of shm_query on this batch and keep the fastest for
    later calls.  Returns {"chosen": index, "times_ms": [per shape, -1 = not tried]}."""
    _need(dirs, torch.float32, name="dirs")
    Q = dirs.shape[0]
    _need(glyph, torch.int32, (Q,), "glyph")
    _need(seg, torch.int64, (lut.n_glyphs + 1,), "seg")
    out = {k: _io_empty(s, torch.float32, dirs) for k, s in (("R", (Q,)), ("grad", (Q, 3)), ("normal", (Q, 3)))}
    chosen = C.c_int32(-1)
    times = (C.c_float * 4)()
    _check(lib().shm_tune_query(C.byref(lut.c()), Q, _io_ptr(dirs), _io_ptr(glyph), _io_ptr(seg), _io_ptr(out["R"]),
                                _io_ptr(out["grad"]), _io_ptr(out["normal"]), int(reps), C.byref(chosen), times,
                                _stream(stream)), "shm_tune_query")
    return {"chosen": chosen.value, "times_ms": [round(float(t), 5) for t in times]}


def tune_reset():
    _check(lib().shm_tune_reset(), "shm_tune_reset")


def query_recon(lut: Lut, method: int, dirs: torch.Tensor, glyph: torch.Tensor = None, seg: torch.Tensor = None,
                want=("R", "grad", "normal"), out: dict = None, dev_status: torch.Tensor = None, stream=None) -> dict:
    """shm_query_recon: value-only reconstruction baseline `method` on a SHM_LAYOUT_VALUE table."""
    _need(dirs, torch.float32, name="dirs")
    Q = dirs.shape[0]
    _need(glyph, torch.int32, (Q,), "glyph")
    _need(seg, torch.int64, (lut.n_glyphs + 1,), "seg")
    out = {} if out is None else out
    shapes = {"R": (Q,), "grad": (Q, 3), "normal": (Q, 3), "chart": (Q, 2), "fij": (Q, 3)}
    for k in want:
        if k not in out:
            out[k] = _io_empty(shapes[k], torch.int32 if k == "fij" else torch.float32, dirs)
    st = lib().shm_query_recon(C.byref(lut.c()), int(method), Q, _io_ptr(dirs), _io_ptr(glyph), _io_ptr(seg),
                               _io_ptr(out.get("R")), _io_ptr(out.get("grad")), _io_ptr(out.get("normal")),
                               _io_ptr(out.get("chart")), _io_ptr(out.get("fij")), _io_ptr(dev_status),
                               _stream(stream))
    _check(st, "shm_query_recon")
    return out


def sh_basis(N: int, L: int, device="cuda", stream=None) -> torch.Tensor:
    nbytes = int(lib().shm_sh_basis_bytes(N, L))
    if nbytes < 0:
        raise ShmError("shm_sh_basis_bytes: invalid N/L")
    B = torch.empty(nbytes // 4, dtype=torch.float32, device=device)
    _check(lib().shm_sh_basis(N, L, _ptr(B), _stream(stream)), "shm_sh_basis")
    return B


@dataclass
class Source:
    kind: int
    L: int = 0
    coeffs: torch.Tensor = None
    basis: torch.Tensor = None
    samples: torch.Tensor = None
    sample_offset: torch.Tensor = None
    bump_offset: torch.Tensor = None
    mu: torch.Tensor = None
    amp: torch.Tensor = None
    width: torch.Tensor = None
    octaves: int = 0
    keys: torch.Tensor = None
    base_freq: float = 2.0
    lacunarity: float = 2.0
    gain: float = 0.5
    amplitude: float = 0.02
    dev_status: torch.Tensor = None

    def c(self) -> c_source:
        s = c_source()
        s.kind, s.L, s.octaves = self.kind, self.L, self.octaves
        for name in ("coeffs", "basis", "samples", "sample_offset", "bump_offset", "mu", "amp", "width", "keys",
                     "dev_status"):
            t = getattr(self, name)
            setattr(s, name, t.data_ptr() if t is not None else None)
        s.base_freq, s.lacunarity, s.gain, s.amplitude = self.base_freq, self.lacunarity, self.gain, self.amplitude
        return s


def build_workspace_bytes(lut: Lut, src: Source) -> int:
    return int(lib().shm_build_workspace_bytes(C.byref(lut.c()), C.byref(src.c())))


def build_lut(lut: Lut, src: Source, ws: torch.Tensor = None, stream=None):
    """shm_build_lut.  For SH sources a workspace of build_workspace_bytes selects the tensor-core
    engine; ws=None runs the float32 CUDA-core engine."""
    wp, wn = (None, 0) if ws is None else (_ptr(ws), ws.numel() * ws.element_size())
    _check(lib().shm_build_lut(C.byref(lut.c()), C.byref(src.c()), wp, wn, _stream(stream)), "shm_build_lut")


def build_workspace(lut: Lut, src: Source) -> torch.Tensor:
    n = build_workspace_bytes(lut, src)
    return torch.empty(max(n, 16), dtype=torch.uint8, device=lut.data.device)


def pack_lut(src: Lut, dst: Lut, stream=None):
    _check(lib().shm_pack_lut(C.byref(src.c()), C.byref(dst.c()), _stream(stream)), "shm_pack_lut")


def lut_bounds(lut: Lut, stream=None) -> torch.Tensor:
    r = torch.empty(lut.n_glyphs, dtype=torch.float32, device=lut.data.device)
    _check(lib().shm_lut_bounds(C.byref(lut.c()), _ptr(r), _stream(stream)), "shm_lut_bounds")
    return r


def mip_like(fine: Lut, dtype: int = None, layout: int = None, r0="same", zero=False) -> Lut:
    """A table for the next mip level of `fine`: every glyph at half the resolution."""
    if fine.N_uniform > 0:
        N = fine.N_uniform // 2
    else:
        N = [int(n) // 2 for n in fine.N.tolist()]
    dtype = fine.dtype if dtype is None else dtype
    layout = fine.layout if layout is None else layout
    out = alloc_lut(fine.n_glyphs, N, dtype, layout, device=fine.data.device, zero=zero)
    rr = fine.r0 if isinstance(r0, str) else r0
    if rr is not None:
        out.r0 = torch.as_tensor(rr, dtype=torch.float32, device=fine.data.device).reshape(-1).contiguous()
    return out


def build_mip(fine: Lut, coarse: Lut, dev_status: torch.Tensor = None, stream=None) -> Lut:
    """shm_build_mip: derivative-consistent coarse level (coarse N = fine N / 2) written into coarse."""
    _need(dev_status, torch.int32, name="dev_status")
    _check(lib().shm_build_mip(C.byref(fine.c()), C.byref(coarse.c()), _ptr(dev_status), _stream(stream)),
           "shm_build_mip")
    return coarse


def mip_chain(fine: Lut, levels: int, dtype: int = None, layout: int = None, stream=None) -> list:
    """[fine, level 1, ..., level `levels`], each built from the previous one on the device."""
    chain = [fine]
    for _ in range(levels):
        chain.append(build_mip(chain[-1], mip_like(chain[-1], dtype, layout), stream=stream))
    return chain


# ------------------------------------------------------------------------------------------- adjoint
def query_backward(lut: Lut, dirs: torch.Tensor, dlut: Lut, gR=None, ggrad=None, gnormal=None, glyph=None, seg=None,
                   want_ddirs=True, dev_status=None, stream=None, deterministic=False):
    """shm_query_backward: accumulates into dlut (float32 texel layout); returns ddirs or None.
    deterministic=True (SHM_BWD_DETERMINISTIC, segments only): dlut bit-identical run to run."""
    _need(dirs, torch.float32, name="dirs")
    Q = dirs.shape[0]
    for t, nm in ((gR, "gR"), (ggrad, "ggrad"), (gnormal, "gnormal")):
        _need(t, torch.float32, name=nm)
    ddirs = _io_empty((Q, 3), torch.float32, dirs) if want_ddirs else None
    st = lib().shm_query_backward(C.byref(lut.c()), Q, _io_ptr(dirs), _io_ptr(glyph), _io_ptr(seg), _io_ptr(gR),
                                  _io_ptr(ggrad), _io_ptr(gnormal), C.byref(dlut.c()), _io_ptr(ddirs),
                                  C.c_uint32(SHM_BWD_DETERMINISTIC if deterministic else 0), _io_ptr(dev_status),
                                  _stream(stream))
    _check(st, "shm_query_backward")
    return ddirs


def build_lut_backward(dlut: Lut, L: int, basis: torch.Tensor, stream=None, deterministic=False,
                       cuda_cores=False, out: torch.Tensor = None) -> torch.Tensor:
    """shm_build_lut_backward: dcoeffs [G][(L+1)^2] from dL/dtable (tensor cores unless cuda_cores)."""
    K = (L + 1) ** 2
    dc = torch.empty((dlut.n_glyphs, K), dtype=torch.float32, device=dlut.data.device) if out is None else out
    flags = (SHM_BWD_DETERMINISTIC if deterministic else 0) | (SHM_BWD_CUDA_CORES if cuda_cores else 0)
    _check(lib().shm_build_lut_backward(C.byref(dlut.c()), L, _ptr(basis), _ptr(dc), C.c_uint32(flags),
                                        _stream(stream)), "shm_build_lut_backward")
    return dc


def fit_backward(lut: Lut, dirs: torch.Tensor, R_target: torch.Tensor, n_target: torch.Tensor, dlut: Lut,
                 w_value: float = 1.0, w_normal: float = 1.0, loss: torch.Tensor = None, glyph=None, seg=None,
                 dev_status=None, stream=None):
    """shm_fit_backward: accumulates dL/dtable into dlut and sum_q L_q into loss (device float [1])."""
    _need(dirs, torch.float32, name="dirs")
    Q = dirs.shape[0]
    _need(R_target, torch.float32, (Q,), "R_target")
    _need(n_target, torch.float32, (Q, 3), "n_target")
    st = lib().shm_fit_backward(C.byref(lut.c()), Q, _io_ptr(dirs), _io_ptr(glyph), _io_ptr(seg), _io_ptr(R_target),
                                _io_ptr(n_target), float(w_value), float(w_normal), C.byref(dlut.c()),
                                _io_ptr(loss), _io_ptr(dev_status), _stream(stream))
    _check(st, "shm_fit_backward")


def adam_step(param: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, lr: float, step: int,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, zero_grad: bool = True, stream=None):
    for t, nm in ((param, "param"), (grad, "grad"), (m, "m"), (v, "v")):
        _need(t, torch.float32, (param.numel(),) if t.dim() == 1 else None, nm)
    st = lib().shm_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), float(lr), float(beta1),
                             float(beta2), float(eps), int(step), int(bool(zero_grad)), _stream(stream))
    _check(st, "shm_adam_step")


# ------------------------------------------------------------------------------------------- direct SH
def sh_eval(L: int, coeffs: torch.Tensor, dirs: torch.Tensor, glyph=None, seg=None, dev_status=None, stream=None):
    _need(coeffs, torch.float32, name="coeffs")
    _need(dirs, torch.float32, name="dirs")
    Q = dirs.shape[0]
    G = coeffs.shape[0]
    R = torch.empty(Q, dtype=torch.float32, device=dirs.device)
    grad = torch.empty((Q, 3), dtype=torch.float32, device=dirs.device)
    normal = torch.empty((Q, 3), dtype=torch.float32, device=dirs.device)
    st = lib().shm_sh_eval(L, G, _ptr(coeffs), Q, _ptr(dirs), _ptr(glyph), _ptr(seg), _ptr(R), _ptr(grad),
                           _ptr(normal), _ptr(dev_status), _stream(stream))
    _check(st, "shm_sh_eval")
    return R, grad, normal


# ------------------------------------------------------------------------------------------- raycast
def make_camera(eye, fwd, right, up, fov_y_deg: float, W: int, H: int) -> c_camera:
    import math
    cam = c_camera()
    for q in range(3):
        cam.eye[q], cam.fwd[q], cam.right[q], cam.up[q] = eye[q], fwd[q], right[q], up[q]
    cam.tan_half_fov_y = math.tan(math.radians(fov_y_deg) / 2.0)
    cam.W, cam.H = int(W), int(H)
    return cam


def make_raycast_params(march=32, bisect=12, newton=3, ambient=0.1, kd=0.7, ks=0.3, shininess=64.0,
                        light=(1.0, 1.0, 1.0), lod=0, bisect_min=8, newton_min=2, recon=0) -> c_raycast_params:
    """recon: the SHM_RECON_* baseline used when the table is SHM_LAYOUT_VALUE (ignored otherwise)."""
    p = c_raycast_params()
    p.recon = recon
    p.march, p.bisect, p.newton = march, bisect, newton
    p.lod, p.bisect_min, p.newton_min = lod, bisect_min, newton_min
    p.ambient, p.kd, p.ks, p.shininess = ambient, kd, ks, shininess
    for q in range(3):
        p.light[q] = light[q]
    return p


def objects_tensor(centre, scale, rmax, glyph, device="cuda") -> torch.Tensor:
    """Pack object records (shm_object, 24 B each) into a device byte tensor."""
    import numpy as np
    n = len(scale)
    rec = np.zeros(n, dtype=[("c", "<f4", 3), ("s", "<f4"), ("r", "<f4"), ("g", "<i4")])
    rec["c"] = np.asarray(centre, dtype=np.float32).reshape(n, 3)
    rec["s"] = np.asarray(scale, dtype=np.float32)
    rec["r"] = np.asarray(rmax, dtype=np.float32)
    rec["g"] = np.asarray(glyph, dtype=np.int32)
    return torch.from_numpy(rec.view(np.uint8).copy()).to(device)


def raycast_workspace_bytes(n_obj: int, W: int, H: int) -> int:
    return int(lib().shm_raycast_workspace_bytes(n_obj, W, H))


def raycast(lut: Lut, objs: torch.Tensor, n_obj: int, cam: c_camera, prm: c_raycast_params, ws: torch.Tensor = None,
            want=("rgba", "depth", "normal", "obj_id"), out: dict = None, dev_status=None, stream=None) -> dict:
    W, H = cam.W, cam.H
    dev = lut.data.device
    nb = raycast_workspace_bytes(n_obj, W, H)
    if ws is None:
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    out = {} if out is None else out
    shapes = {"rgba": (H, W, 4), "depth": (H, W), "normal": (H, W, 3), "obj_id": (H, W)}
    for k in want:
        if k not in out:
            out[k] = torch.empty(shapes[k], dtype=torch.int32 if k == "obj_id" else torch.float32, device=dev)
    st = lib().shm_raycast(C.byref(lut.c()), _ptr(objs), n_obj, C.byref(cam), C.byref(prm), _ptr(out.get("rgba")),
                           _ptr(out.get("depth")), _ptr(out.get("normal")), _ptr(out.get("obj_id")), _ptr(ws),
                           ws.numel(), _ptr(dev_status), _stream(stream))
    _check(st, "shm_raycast")
    out["_ws"] = ws
    return out


def raycast_noalloc(lut: Lut, objs: torch.Tensor, n_obj: int, cam: c_camera, prm: c_raycast_params,
                    want=("rgba", "depth", "normal", "obj_id"), out: dict = None, dev_status=None, stream=None) -> dict:
    """shm_raycast_noalloc: ray casting with the library's static device workspace, for callers that
    cannot allocate device memory while they render.  The outputs requested in `want` that are not
    in `out` are allocated here by torch; pass every buffer in `out` to allocate nothing at all.
    The static workspace is not exposed, so the surface-query counter that raycast_query_count reads
    from a caller's shm_raycast workspace cannot be read for this entry point."""
    W, H = cam.W, cam.H
    dev = lut.data.device
    out = {} if out is None else out
    shapes = {"rgba": (H, W, 4), "depth": (H, W), "normal": (H, W, 3), "obj_id": (H, W)}
    for k in want:
        if k not in out:
            out[k] = torch.empty(shapes[k], dtype=torch.int32 if k == "obj_id" else torch.float32, device=dev)
    st = lib().shm_raycast_noalloc(C.byref(lut.c()), _ptr(objs), n_obj, C.byref(cam), C.byref(prm),
                                   _ptr(out.get("rgba")), _ptr(out.get("depth")), _ptr(out.get("normal")),
                                   _ptr(out.get("obj_id")), _ptr(dev_status), _stream(stream))
    _check(st, "shm_raycast_noalloc")
    return out


def raycast_query_count(ws: torch.Tensor) -> int:
    """Surface queries the last shm_raycast on this workspace evaluated (workspace header)."""
    return int(ws[8:16].view(torch.int64).item())


# ------------------------------------------------------------------------------------------- L2 hint
def l2_fetch_granularity(nbytes: int = -1) -> int:
    """shm_l2_fetch_granularity: set the context's L2 fetch granularity hint (0..128 B; -1 only
    reads it).  Returns the value before the call."""
    prev = C.c_int32(-1)
    _check(lib().shm_l2_fetch_granularity(int(nbytes), C.byref(prev)), "shm_l2_fetch_granularity")
    return prev.value
