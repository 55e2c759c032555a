"""FP64 CPU oracle for Spherical Hermite Maps (arXiv 2602.20063) -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may import this
package.  It shares no code with the CUDA library (``paper_2602_20063_gb300``) and neither
imports the other; the two meet only in the seeded input generators of ``shm_inputs``.

The arithmetic lives in plain C (oracle/*.c, float64, one file per paper section); this
module only marshals numpy arrays.  Table layout: one glyph is [6][N+2][N+2][4] float64
(channels r, r_u h, r_v h, r_uv h^2, Eq. hermite_storage); pools concatenate glyph tables and
``off[g]`` is the first texel of glyph g.  Stored 16-bit or float32 tables are converted to
float64 exactly before they are passed in.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_d = C.POINTER(C.c_double)
_f = C.POINTER(C.c_float)
_i32 = C.POINTER(C.c_int32)
_i64 = C.POINTER(C.c_int64)
_u32 = C.POINTER(C.c_uint32)


class Camera(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("fwd", C.c_double * 3), ("right", C.c_double * 3),
                ("up", C.c_double * 3), ("tan_half_fov_y", C.c_double), ("W", C.c_int), ("H", C.c_int)]


class RaycastParams(C.Structure):
    _fields_ = [("march", C.c_int), ("bisect", C.c_int), ("newton", C.c_int),
                ("ambient", C.c_double), ("kd", C.c_double), ("ks", C.c_double),
                ("shininess", C.c_double), ("light", C.c_double * 3),
                ("lod", C.c_int), ("bisect_min", C.c_int), ("newton_min", C.c_int), ("recon", C.c_int)]


class QueryOut(C.Structure):
    _fields_ = [("face", C.c_int), ("i", C.c_int), ("j", C.c_int),
                ("u", C.c_double), ("v", C.c_double), ("s", C.c_double), ("t", C.c_double),
                ("R", C.c_double), ("Ru", C.c_double), ("Rv", C.c_double),
                ("grad", C.c_double * 3), ("normal", C.c_double * 3)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
    return _lib


def nthreads_default() -> int:
    return int(os.environ.get("SHM_ORACLE_THREADS", os.cpu_count() or 1))


def _p(a, ct):
    return a.ctypes.data_as(ct) if a is not None else None


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------------- single-point helpers (tests)
def face_uv(w):
    u, v = C.c_double(), C.c_double()
    f = lib().shmo_face_uv(_p(_c64(w), _d), C.byref(u), C.byref(v))
    return f, u.value, v.value


def face_frame(f):
    a, b, c = (np.zeros(3) for _ in range(3))
    lib().shmo_face_frame(C.c_int(f), _p(a, _d), _p(b, _d), _p(c, _d))
    return a, b, c


def dir_tilde(f, u, v):
    wt = np.zeros(3)
    lib().shmo_dir_tilde(C.c_int(f), C.c_double(u), C.c_double(v), _p(wt, _d))
    return wt


def texel_centre(i, N):
    fn = lib().shmo_texel_centre
    fn.restype = C.c_double
    return fn(C.c_int(i), C.c_int(N))


def tangents(f, u, v):
    e1, e2 = np.zeros(3), np.zeros(3)
    lib().shmo_tangents(C.c_int(f), C.c_double(u), C.c_double(v), _p(e1, _d), _p(e2, _d))
    return e1, e2


def metric(f, u, v):
    G = np.zeros(3)
    lib().shmo_metric(C.c_int(f), C.c_double(u), C.c_double(v), _p(G, _d))
    return G


def s2_gradient(f, u, v, Ru, Rv):
    g = np.zeros(3)
    lib().shmo_s2_gradient(C.c_int(f), C.c_double(u), C.c_double(v), C.c_double(Ru), C.c_double(Rv), _p(g, _d))
    return g


def normal(w, R, grad):
    n = np.zeros(3)
    lib().shmo_normal(_p(_c64(w), _d), C.c_double(R), _p(_c64(grad), _d), _p(n, _d))
    return n


def hermite_basis(s):
    H, dH, ddH = np.zeros(4), np.zeros(4), np.zeros(4)
    lib().shmo_hermite_basis(C.c_double(s), _p(H, _d), _p(dH, _d), _p(ddH, _d))
    return H, dH, ddH


def cell(N, u):
    i, s = C.c_int(), C.c_double()
    lib().shmo_cell(C.c_int(N), C.c_double(u), C.byref(i), C.byref(s))
    return i.value, s.value


def hermite_eval(face, N, i, j, s, t):
    """face: [P][P][4] float64.  Returns (r, r_s, r_t, r_ss, r_st, r_tt)."""
    out = np.zeros(6)
    lib().shmo_hermite_eval(_p(_c64(face), _d), C.c_int(N), C.c_int(i), C.c_int(j),
                            C.c_double(s), C.c_double(t), _p(out, _d))
    return out


def hermite_weights(s, t):
    w = np.zeros((3, 4, 4))
    lib().shmo_hermite_weights(C.c_double(s), C.c_double(t), _p(w, _d))
    return w


def sh_count(L):
    return (L + 1) * (L + 1)


def sh_basis(L, w):
    Y = np.zeros(sh_count(L))
    lib().shmo_sh_basis(C.c_int(L), _p(_c64(w), _d), _p(Y, _d))
    return Y


def sh_chart_basis(L, f, u, v):
    out = np.zeros((sh_count(L), 4))
    lib().shmo_sh_chart_basis(C.c_int(L), C.c_int(f), C.c_double(u), C.c_double(v), _p(out, _d))
    return out


def sh_chart(L, coeffs, f, u, v):
    out = np.zeros(4)
    lib().shmo_sh_chart(C.c_int(L), _p(_c64(coeffs), _d), C.c_int(f), C.c_double(u), C.c_double(v), _p(out, _d))
    return out


def sh_value_grad(L, coeffs, w):
    r = C.c_double()
    g = np.zeros(3)
    lib().shmo_sh_value_grad(C.c_int(L), _p(_c64(coeffs), _d), _p(_c64(w), _d), C.byref(r), _p(g, _d))
    return r.value, g


def sh_eval(L, coeffs, dirs, glyph=None, nthreads=None):
    """Direct SH evaluation: returns R [Q], grad [Q][3], normal [Q][3] (float64)."""
    dirs = np.ascontiguousarray(dirs, dtype=np.float32)
    Q = dirs.shape[0]
    coeffs = _c64(coeffs)
    gl = None if glyph is None else np.ascontiguousarray(glyph, dtype=np.int32)
    R, G, Nn = np.zeros(Q), np.zeros((Q, 3)), np.zeros((Q, 3))
    lib().shmo_sh_eval_batch(C.c_int(L), _p(coeffs, _d), C.c_int64(Q), _p(dirs, _f), _p(gl, _i32),
                             _p(R, _d), _p(G, _d), _p(Nn, _d), C.c_int(nthreads or nthreads_default()))
    return R, G, Nn


# ----------------------------------------------------------------- bake (Algorithm 1)
def bake_sh(N, L, coeffs):
    P = N + 2
    lut = np.zeros((6, P, P, 4))
    lib().shmo_bake_sh(C.c_int(N), C.c_int(L), _p(_c64(coeffs), _d), _p(lut, _d))
    return lut


def sh_basis_records(N, L):
    P = N + 2
    B = np.zeros((sh_count(L), 6, P, P, 4))
    lib().shmo_sh_basis_records(C.c_int(N), C.c_int(L), _p(B, _d))
    return B


def bake_fd(N, samples, r0=0.0):
    P = N + 2
    samples = _c64(samples)
    assert samples.shape == (6, N + 4, N + 4)
    lut = np.zeros((6, P, P, 4))
    lib().shmo_bake_fd(C.c_int(N), _p(samples, _d), C.c_double(r0), _p(lut, _d))
    return lut


def sample_grid_bumps(N, mu, amp, width):
    S = N + 4
    out = np.zeros((6, S, S))
    mu, amp, width = _c64(mu), _c64(amp), _c64(width)
    lib().shmo_sample_grid_bumps(C.c_int(N), C.c_int(len(amp)), _p(mu, _d), _p(amp, _d), _p(width, _d), _p(out, _d))
    return out


def sample_grid_fbm(N, keys, base_freq=2.0, lacunarity=2.0, gain=0.5, amplitude=0.02):
    S = N + 4
    out = np.zeros((6, S, S))
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    lib().shmo_sample_grid_fbm(C.c_int(N), C.c_int(keys.shape[0]), _p(keys, _u32), C.c_double(base_freq),
                               C.c_double(lacunarity), C.c_double(gain), C.c_double(amplitude), _p(out, _d))
    return out


def lut_bound(glut, N, r0=0.0):
    fn = lib().shmo_lut_bound
    fn.restype = C.c_double
    return fn(_p(_c64(glut), _d), C.c_int(N), C.c_double(r0))


# ----------------------------------------------------------------- procedural
def bumps(w, mu, amp, width):
    fn = lib().shmo_bumps
    fn.restype = C.c_double
    return fn(_p(_c64(w), _d), C.c_int(len(amp)), _p(_c64(mu), _d), _p(_c64(amp), _d), _p(_c64(width), _d))


def value_noise(p, key):
    fn = lib().shmo_value_noise
    fn.restype = C.c_double
    return fn(_p(_c64(p), _d), _p(np.ascontiguousarray(key, dtype=np.uint32), _u32))


def fbm(w, keys, base_freq=2.0, lacunarity=2.0, gain=0.5):
    fn = lib().shmo_fbm
    fn.restype = C.c_double
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    return fn(_p(_c64(w), _d), C.c_int(keys.shape[0]), _p(keys, _u32), C.c_double(base_freq),
              C.c_double(lacunarity), C.c_double(gain))


def pcg3d(v):
    a = np.array(v, dtype=np.uint32)
    lib().shmo_pcg3d(_p(a, _u32))
    return a


# ----------------------------------------------------------------- pools and queries
def make_pool(luts):
    """Concatenate glyph tables [6][P][P][4] -> (pool [T_total][4] f64, off [G] i64, Ns [G] i32)."""
    Ns = np.array([l.shape[1] - 2 for l in luts], dtype=np.int32)
    sizes = np.array([6 * (n + 2) ** 2 for n in Ns], dtype=np.int64)
    off = np.zeros(len(luts), dtype=np.int64)
    off[1:] = np.cumsum(sizes)[:-1]
    pool = np.concatenate([_c64(l).reshape(-1, 4) for l in luts], axis=0)
    return pool, off, Ns


def query_one(glut, N, d, r0=0.0):
    o = QueryOut()
    lib().shmo_query_one(_p(_c64(glut), _d), C.c_int(N), C.c_double(r0), _p(_c64(d), _d), C.byref(o))
    return o


def query(pool, off, Ns, dirs, glyph=None, r0=None, nthreads=None):
    """Batched query.  Returns dict R [Q], grad [Q][3], normal [Q][3], chart [Q][2] (R_u, R_v),
    fij [Q][3] (face, i, j)."""
    pool = _c64(pool)
    off = np.ascontiguousarray(off, dtype=np.int64)
    Ns = np.ascontiguousarray(Ns, dtype=np.int32)
    dirs = np.ascontiguousarray(dirs, dtype=np.float32)
    Q = dirs.shape[0]
    gl = None if glyph is None else np.ascontiguousarray(glyph, dtype=np.int32)
    r0a = None if r0 is None else _c64(r0)
    out = dict(R=np.zeros(Q), grad=np.zeros((Q, 3)), normal=np.zeros((Q, 3)), chart=np.zeros((Q, 2)),
               fij=np.zeros((Q, 3), dtype=np.int32))
    lib().shmo_query_batch(_p(pool, _d), _p(off, _i64), _p(Ns, _i32), _p(r0a, _d), C.c_int64(Q), _p(dirs, _f),
                           _p(gl, _i32), _p(out["R"], _d), _p(out["grad"], _d), _p(out["normal"], _d),
                           _p(out["chart"], _d), _p(out["fij"], _i32), C.c_int(nthreads or nthreads_default()))
    return out


def query_vjp(pool, off, Ns, dirs, gR=None, gG=None, gn=None, glyph=None, r0=None, want_dlut=True,
              want_ddirs=True):
    pool = _c64(pool)
    off = np.ascontiguousarray(off, dtype=np.int64)
    Ns = np.ascontiguousarray(Ns, dtype=np.int32)
    dirs = np.ascontiguousarray(dirs, dtype=np.float32)
    Q = dirs.shape[0]
    gl = None if glyph is None else np.ascontiguousarray(glyph, dtype=np.int32)
    r0a = None if r0 is None else _c64(r0)
    gR = None if gR is None else _c64(gR)
    gG = None if gG is None else _c64(gG)
    gn = None if gn is None else _c64(gn)
    dpool = np.zeros_like(pool) if want_dlut else None
    ddirs = np.zeros((Q, 3)) if want_ddirs else None
    lib().shmo_query_vjp_batch(_p(pool, _d), _p(off, _i64), _p(Ns, _i32), _p(r0a, _d), C.c_int64(Q),
                               _p(dirs, _f), _p(gl, _i32), _p(gR, _d), _p(gG, _d), _p(gn, _d),
                               _p(dpool, _d), _p(ddirs, _d))
    return dpool, ddirs


def query_vjp_one(glut, N, d, gR, gG, gn, r0=0.0):
    dglut = np.zeros_like(_c64(glut))
    dd = np.zeros(3)
    lib().shmo_query_vjp_one(_p(_c64(glut), _d), C.c_int(N), C.c_double(r0), _p(_c64(d), _d), C.c_double(gR),
                             _p(_c64(gG), _d), _p(_c64(gn), _d), _p(dglut, _d), _p(dd, _d))
    return dglut, dd


def bake_sh_vjp(N, L, dlut):
    dc = np.zeros(sh_count(L))
    lib().shmo_bake_sh_vjp(C.c_int(N), C.c_int(L), _p(_c64(dlut), _d), _p(dc, _d))
    return dc


def lod_steps(cam, prm, centre, rmax):
    """(bisection steps, Newton steps, projected radius in pixels) of one object."""
    b, n, p = C.c_int(), C.c_int(), C.c_float()
    c = _c64(centre)
    lib().shmo_lod_steps(C.byref(cam), C.byref(prm), _p(c, _d), C.c_double(rmax), C.byref(b), C.byref(n), C.byref(p))
    return b.value, n.value, p.value


# ----------------------------------------------------------------- value-only baselines (§4.2, §4.5)
RECON_NEAREST, RECON_BILINEAR, RECON_BICUBIC, RECON_FAST_BICUBIC = 0, 1, 2, 3


def value_grid_sh(N, L, coeffs):
    """Value table [6][N+4][N+4] of an SH function: r at every texel centre, two-texel gutter."""
    g = np.zeros((6, N + 4, N + 4))
    lib().shmo_value_grid_sh(C.c_int(N), C.c_int(L), _p(_c64(coeffs), _d), _p(g, _d))
    return g


def make_value_pool(grids):
    """Concatenate value tables; returns (pool, offset in scalars, Ns)."""
    Ns = np.array([g.shape[1] - 4 for g in grids], dtype=np.int32)
    off = np.zeros(len(grids), dtype=np.int64)
    for k in range(1, len(grids)):
        off[k] = off[k - 1] + grids[k - 1].size
    return np.concatenate([np.asarray(g, dtype=np.float64).reshape(-1) for g in grids]), off, Ns


def recon(method, pool, off, Ns, dirs, glyph=None, r0=None, nthreads=None):
    """Batched value-only reconstruction (same outputs as ``query``)."""
    pool = _c64(pool)
    off = np.ascontiguousarray(off, dtype=np.int64)
    Ns = np.ascontiguousarray(Ns, dtype=np.int32)
    dirs = np.ascontiguousarray(dirs, dtype=np.float32)
    Q = dirs.shape[0]
    gl = None if glyph is None else np.ascontiguousarray(glyph, dtype=np.int32)
    r0a = None if r0 is None else _c64(r0)
    out = dict(R=np.zeros(Q), grad=np.zeros((Q, 3)), normal=np.zeros((Q, 3)), chart=np.zeros((Q, 2)),
               fij=np.zeros((Q, 3), dtype=np.int32))
    lib().shmo_recon_batch(C.c_int(method), _p(pool, _d), _p(off, _i64), _p(Ns, _i32), _p(r0a, _d), C.c_int64(Q),
                           _p(dirs, _f), _p(gl, _i32), _p(out["R"], _d), _p(out["grad"], _d), _p(out["normal"], _d),
                           _p(out["chart"], _d), _p(out["fij"], _i32), C.c_int(nthreads or nthreads_default()))
    return out


def catmull_rom(s):
    w, dw = np.zeros(4), np.zeros(4)
    lib().shmo_catmull_rom(C.c_double(s), _p(w, _d), _p(dw, _d))
    return w, dw


def bspline3(s):
    w = np.zeros(4)
    lib().shmo_bspline3(C.c_double(s), _p(w, _d))
    return w


# ----------------------------------------------------------------- mip levels (§4.7)
def mip_samples(fine, r0=0.0):
    """Coarse margin samples [6][Nc+4][Nc+4] (absolute radius) of one fine glyph table."""
    fine = _c64(fine)
    Nf = fine.shape[1] - 2
    assert Nf % 2 == 0 and Nf >= 2
    S = Nf // 2 + 4
    samples = np.zeros((6, S, S))
    lib().shmo_mip_samples(_p(fine, _d), C.c_int(Nf), C.c_double(r0), _p(samples, _d))
    return samples


def mip_consistent(fine, r0=0.0, r0_coarse=None):
    """Derivative-consistent coarse level of one glyph table [6][Nf+2][Nf+2][4] (stored channel 0
    relative to r0; the coarse one relative to r0_coarse, default r0): box-filtered fine
    interpolant, then central-difference records."""
    fine = _c64(fine)
    Nc = (fine.shape[1] - 2) // 2
    return bake_fd(Nc, mip_samples(fine, r0), r0=r0 if r0_coarse is None else r0_coarse)


def mip_naive(fine):
    """Naive coarse level: every record channel box-filtered over the 2x2 children."""
    fine = _c64(fine)
    Nf = fine.shape[1] - 2
    Pc = Nf // 2 + 2
    out = np.zeros((6, Pc, Pc, 4))
    lib().shmo_mip_naive(_p(fine, _d), C.c_int(Nf), _p(out, _d))
    return out


# ----------------------------------------------------------------- raycast
def make_camera(eye, fwd, right, up, fov_y_deg, W, H):
    cam = Camera()
    for q in range(3):
        cam.eye[q], cam.fwd[q], cam.right[q], cam.up[q] = eye[q], fwd[q], right[q], up[q]
    cam.tan_half_fov_y = float(np.tan(np.radians(fov_y_deg) / 2.0))
    cam.W, cam.H = int(W), int(H)
    return cam


def make_raycast_params(march=32, bisect=12, newton=3, ambient=0.1, kd=0.7, ks=0.3, shininess=64.0,
                        light=(1.0, 1.0, 1.0), lod=0, bisect_min=8, newton_min=2, recon=-1):
    """recon = -1: Hermite tables; else a RECON_* baseline on value grids (raycast's pool is then a
    value pool from make_value_pool)."""
    p = RaycastParams()
    p.recon = recon
    p.march, p.bisect, p.newton = march, bisect, newton
    p.lod, p.bisect_min, p.newton_min = lod, bisect_min, newton_min
    p.ambient, p.kd, p.ks, p.shininess = ambient, kd, ks, shininess
    for q in range(3):
        p.light[q] = light[q]
    return p


def raycast(pool, off, Ns, centre, scale, rmax, glyph, cam, prm, px=None, py=None, r0=None, nthreads=None):
    """Raycast pixels (px, py) (default: the whole W x H image, row-major).  Returns dict rgba [n][4],
    depth [n], normal [n][3], obj_id [n], margin [n]."""
    if px is None:
        yy, xx = np.meshgrid(np.arange(cam.H, dtype=np.int32), np.arange(cam.W, dtype=np.int32), indexing="ij")
        px, py = xx.ravel(), yy.ravel()
    px = np.ascontiguousarray(px, dtype=np.int32)
    py = np.ascontiguousarray(py, dtype=np.int32)
    n = px.shape[0]
    pool = _c64(pool)
    off = np.ascontiguousarray(off, dtype=np.int64)
    Ns = np.ascontiguousarray(Ns, dtype=np.int32)
    r0a = None if r0 is None else _c64(r0)
    centre, scale, rmax = _c64(centre), _c64(scale), _c64(rmax)
    glyph = np.ascontiguousarray(glyph, dtype=np.int32)
    out = dict(rgba=np.zeros((n, 4)), depth=np.zeros(n), normal=np.zeros((n, 3)),
               obj_id=np.zeros(n, dtype=np.int32), margin=np.zeros(n))
    lib().shmo_raycast_image(_p(pool, _d), _p(off, _i64), _p(Ns, _i32), _p(r0a, _d), C.c_int(len(scale)),
                             _p(centre, _d), _p(scale, _d), _p(rmax, _d), _p(glyph, _i32), C.byref(cam),
                             C.byref(prm), C.c_int64(n), _p(px, _i32), _p(py, _i32), _p(out["rgba"], _d),
                             _p(out["depth"], _d), _p(out["normal"], _d), _p(out["obj_id"], _i32),
                             _p(out["margin"], _d), C.c_int(nthreads or nthreads_default()))
    return out


# ----------------------------------------------------------------- storage quantisation
def quantize_f16(x32):
    """float32 -> float16 -> float64, round to nearest even (IEEE conversion)."""
    return np.asarray(x32, dtype=np.float32).astype(np.float16).astype(np.float64)


def quantize_bf16(x32):
    """float32 -> bfloat16 (round to nearest even on the top 16 bits) -> float64."""
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    nan = np.isnan(np.asarray(x32, dtype=np.float32))
    out = (rounded.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def bf16_bits(x32):
    b = np.ascontiguousarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)
