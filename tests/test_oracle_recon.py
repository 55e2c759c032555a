"""Pins for the oracle's value-only reconstruction baselines (§4.2 Table psnr_value, §4.5
Table cost_extended).

Pins: bilinear and the cubic B-spline ("fast bicubic") equal scipy.ndimage.map_coordinates of
orders 1 and 3 (no prefilter) on the same face grid; the B-spline also equals the GPU Gems 2
four-bilinear-fetch form; Catmull-Rom interpolates the texel values and reproduces quadratics
exactly, value and analytic gradient; nearest returns the texel whose square holds (u, v); the
value grid of an SH function agrees with the Hermite bake's value channel; Table psnr_value's
method ordering and per-doubling gains.
"""
import math
import os

import numpy as np
import pytest

import shm_inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
ndimage = pytest.importorskip("scipy.ndimage")


def _dir(oracle, f, u, v):
    return oracle.dir_tilde(f, u, v).astype(np.float32)[None, :]


def _face_grid_from(p, N):
    """Grid [6][N+4][N+4] with p(x, y) in texel-index coordinates (texel i at x = i)."""
    idx = np.arange(-1, N + 3, dtype=np.float64)
    X, Y = np.meshgrid(idx, idx, indexing="xy")
    return np.broadcast_to(p(X, Y), (6, N + 4, N + 4)).copy()


def _points(rng, n, N, margin=0.0):
    """Chart points (u, v) well inside the face (away from face edges by `margin` texels)."""
    lo, hi = margin / N, 1.0 - margin / N
    return rng.uniform(lo, hi, size=(n, 2))


def test_bilinear_and_bspline_match_scipy(oracle):
    N = 9
    rng = np.random.default_rng(1)
    grid = rng.normal(size=(6, N + 4, N + 4))
    pool, off, Ns = oracle.make_value_pool([grid])
    for f in (0, 3, 5):
        for u, v in _points(rng, 40, N, margin=1e-3):
            d = _dir(oracle, f, u, v)
            fu, uu, vv = oracle.face_uv(d[0].astype(np.float64))
            assert fu == f
            x, y = uu * N + 0.5, vv * N + 0.5   # texel-index coordinates; array index = coordinate + 1
            coords = np.array([[y + 1.0], [x + 1.0]])
            bl = oracle.recon(oracle.RECON_BILINEAR, pool, off, Ns, d)["R"][0]
            bs = oracle.recon(oracle.RECON_FAST_BICUBIC, pool, off, Ns, d)["R"][0]
            assert abs(bl - ndimage.map_coordinates(grid[f], coords, order=1)[0]) < 1e-12
            assert abs(bs - ndimage.map_coordinates(grid[f], coords, order=3, prefilter=False)[0]) < 1e-12


def test_bspline_equals_four_bilinear_fetches(oracle):
    """GPU Gems 2 ch. 20: g0 = w0 + w1, g1 = w2 + w3, sample positions i - 1 + w1/g0 and i + 1 + w3/g1."""
    N = 7
    rng = np.random.default_rng(2)
    face = rng.normal(size=(N + 4, N + 4))

    def bil(x, y):  # bilinear at texel-index coordinates
        i, j = int(math.floor(x)), int(math.floor(y))
        s, t = x - i, y - j
        v = lambda a, b: face[b + 1, a + 1]
        return (1 - s) * (1 - t) * v(i, j) + s * (1 - t) * v(i + 1, j) + (1 - s) * t * v(i, j + 1) + s * t * v(i + 1, j + 1)

    for _ in range(50):
        x, y = rng.uniform(0.5, N + 0.5, size=2)
        i, j = min(int(math.floor(x)), N), min(int(math.floor(y)), N)
        s, t = x - i, y - j
        wu, wv = oracle.bspline3(s), oracle.bspline3(t)
        ref = sum(wu[a] * wv[b] * face[j - 1 + b + 1, i - 1 + a + 1] for a in range(4) for b in range(4))
        gu = (wu[0] + wu[1], wu[2] + wu[3])
        gv = (wv[0] + wv[1], wv[2] + wv[3])
        xs = (i - 1 + wu[1] / gu[0], i + 1 + wu[3] / gu[1])
        ys = (j - 1 + wv[1] / gv[0], j + 1 + wv[3] / gv[1])
        fast = sum(gu[a] * gv[b] * bil(xs[a], ys[b]) for a in range(2) for b in range(2))
        assert abs(fast - ref) < 1e-12


def test_catmull_rom_interpolates_and_reproduces_quadratics(oracle):
    N = 8
    a, b, c, d, e, g = 0.7, 0.05, -0.03, 0.004, -0.002, 0.003
    p = lambda X, Y: a + b * X + c * Y + d * X * X + e * X * Y + g * Y * Y
    grid = _face_grid_from(p, N)
    pool, off, Ns = oracle.make_value_pool([grid])
    rng = np.random.default_rng(3)
    for f in (1, 4):
        for u, v in _points(rng, 30, N, margin=1e-3):
            dd = _dir(oracle, f, u, v)
            fu, uu, vv = oracle.face_uv(dd[0].astype(np.float64))
            out = oracle.recon(oracle.RECON_BICUBIC, pool, off, Ns, dd)
            X, Y = uu * N + 0.5, vv * N + 0.5
            assert abs(out["R"][0] - p(X, Y)) < 1e-12
            # analytic chart gradient: R_u = N dp/dx
            assert abs(out["chart"][0, 0] - N * (b + 2 * d * X + e * Y)) < 1e-10
            assert abs(out["chart"][0, 1] - N * (c + e * X + 2 * g * Y)) < 1e-10
    # interpolation at texel centres, and the weights' partition of unity / derivative
    for s in (0.0, 0.25, 0.5, 0.9):
        w, dw = oracle.catmull_rom(s)
        assert abs(w.sum() - 1.0) < 1e-15 and abs(dw.sum()) < 1e-14
        wp, _ = oracle.catmull_rom(s + 1e-6)
        wm, _ = oracle.catmull_rom(s - 1e-6)
        assert np.abs((wp - wm) / 2e-6 - dw).max() < 1e-8
    assert np.allclose(oracle.catmull_rom(0.0)[0], [0, 1, 0, 0])


def test_bilinear_fd_gradient_exact_on_linear_field(oracle):
    N = 6
    p = lambda X, Y: 0.4 + 0.02 * X - 0.05 * Y
    pool, off, Ns = oracle.make_value_pool([_face_grid_from(p, N)])
    rng = np.random.default_rng(4)
    for u, v in _points(rng, 30, N, margin=1e-3):
        out = oracle.recon(oracle.RECON_BILINEAR, pool, off, Ns, _dir(oracle, 2, u, v))
        assert abs(out["chart"][0, 0] - 0.02 * N) < 1e-10 and abs(out["chart"][0, 1] + 0.05 * N) < 1e-10


def test_nearest_returns_the_containing_texel(oracle):
    N = 5
    rng = np.random.default_rng(5)
    grid = rng.normal(size=(6, N + 4, N + 4))
    pool, off, Ns = oracle.make_value_pool([grid])
    for u, v in _points(rng, 60, N, margin=1e-3):
        dd = _dir(oracle, 0, u, v)
        f, uu, vv = oracle.face_uv(dd[0].astype(np.float64))
        i, j = int(uu * N) + 1, int(vv * N) + 1
        out = oracle.recon(oracle.RECON_NEAREST, pool, off, Ns, dd)
        assert out["R"][0] == grid[f, j + 1, i + 1]
        assert np.abs(out["chart"]).max() == 0.0


def test_value_grid_matches_hermite_value_channel(oracle):
    N, L = 10, 6
    c = I.sh_coeffs(1, L, 6)[0]
    g = oracle.value_grid_sh(N, L, c)
    lut = oracle.bake_sh(N, L, c)
    # Hermite table texel (i, j), i in 0..N+1 = grid entry (i + 1, j + 1)
    assert np.abs(g[:, 1:N + 3, 1:N + 3] - lut[..., 0]).max() < 1e-12


def _golden_psnr():
    rows = []
    for line in open(os.path.join(HERE, "golden", "psnr_value.txt")):
        if line.startswith("#") or not line.strip():
            continue
        N, bl, bc, he = line.split()
        rows.append((int(N), float(bl), float(bc), float(he)))
    return rows


def test_psnr_value_table_trend(oracle):
    rows = _golden_psnr()
    L = 8
    c = I.sh_coeffs(1, L, 20063 + 1)[0]
    dirs = I.directions(100000, 26)
    Rt, _, _ = oracle.sh_eval(L, c, dirs)
    peak = np.abs(Rt).max()
    psnr = lambda R: 20 * math.log10(peak / math.sqrt(((R - Rt) ** 2).mean()))
    got = []
    for N, *_ in rows:
        pool, off, Ns = oracle.make_value_pool([oracle.value_grid_sh(N, L, c)])
        bl = psnr(oracle.recon(oracle.RECON_BILINEAR, pool, off, Ns, dirs)["R"])
        bc = psnr(oracle.recon(oracle.RECON_BICUBIC, pool, off, Ns, dirs)["R"])
        hp, ho, hn = oracle.make_pool([oracle.bake_sh(N, L, c)])
        he = psnr(oracle.query(hp, ho, hn, dirs)["R"])
        print(f"N={N}: bilinear {bl:.1f}  bicubic {bc:.1f}  hermite {he:.1f} dB")
        got.append((bl, bc, he))
        assert he > bc > bl
    for k in range(len(got) - 1):
        gain_bl = got[k + 1][0] - got[k][0]
        gain_bc = got[k + 1][1] - got[k][1]
        paper_bl = rows[k + 1][1] - rows[k][1]
        paper_bc = rows[k + 1][2] - rows[k][2]
        assert abs(gain_bl - paper_bl) < 2.0, (gain_bl, paper_bl)      # O(h^2): ~12 dB per doubling
        assert 17.0 < gain_bc < 26.0 and 17.0 < paper_bc < 26.0         # O(h^3..h^4)
    margins = [g[2] - g[1] for g in got]
    assert margins[0] < margins[1] < margins[2]   # Hermite's lead over bicubic grows with N, as in the table
