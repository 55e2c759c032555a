"""Pins for the oracle's full query (§3.2-§3.4) and its convergence (§4.2).

Pins: a constant table is a sphere (R const, grad 0, n = w); the returned S^2 gradient equals
directional differences of the interpolated R on the sphere; the normal equals the normalised
gradient of the implicit F(x) = |x| - R(x/|x|) (§3.1) by 3-D central differences; against direct
SH the value error falls as h^4 and the gradient error as h^3; seams between faces close as N
grows; the Table psnr_value trend (golden fixture).
"""
import math
import os

import numpy as np
import pytest

import shm_inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sh_pool(oracle, N, L, seed):
    c = I.sh_coeffs(1, L, seed)[0]
    lut = oracle.bake_sh(N, L, c)
    return c, lut, oracle.make_pool([lut])


def test_constant_table_is_a_sphere(oracle):
    N = 10
    lut = np.zeros((6, N + 2, N + 2, 4))
    lut[..., 0] = 0.25
    pool, off, Ns = oracle.make_pool([lut])
    d = I.directions(500, 20)
    out = oracle.query(pool, off, Ns, d, r0=np.array([1.0]))
    w = d.astype(np.float64) / np.linalg.norm(d.astype(np.float64), axis=1, keepdims=True)
    assert np.allclose(out["R"], 1.25, atol=1e-15)
    assert np.abs(out["grad"]).max() < 1e-15
    assert np.allclose(out["normal"], w, atol=1e-15)


def _away_from_edges(oracle, N, w, margin):
    f, u, v = oracle.face_uv(w)
    su = (u * N + 0.5) % 1.0
    sv = (v * N + 0.5) % 1.0
    return min(su, 1 - su, sv, 1 - sv) > margin and min(u, 1 - u, v, 1 - v) > margin / N


def test_gradient_is_sphere_derivative_of_interpolant(oracle):
    N, L = 12, 6
    _, lut, _ = _sh_pool(oracle, N, L, 21)
    rng = np.random.default_rng(21)
    e = 1e-7
    n_checked = 0
    for d in I.directions(400, 22).astype(np.float64):
        w = d / np.linalg.norm(d)
        if not _away_from_edges(oracle, N, w, 0.01):
            continue
        o = oracle.query_one(lut, N, w)
        t = rng.normal(size=3)
        t -= (t @ w) * w
        t /= np.linalg.norm(t)
        Rp = oracle.query_one(lut, N, w + e * t).R
        Rm = oracle.query_one(lut, N, w - e * t).R
        g = np.array(o.grad[:])
        assert abs(g @ t - (Rp - Rm) / (2 * e)) < 1e-6
        assert abs(g @ w) < 1e-13
        n_checked += 1
    assert n_checked > 200


def test_normal_is_implicit_function_gradient(oracle):
    N, L = 12, 6
    _, lut, _ = _sh_pool(oracle, N, L, 23)
    e = 1e-6

    def F(x):
        return np.linalg.norm(x) - oracle.query_one(lut, N, x).R

    n_checked = 0
    for d in I.directions(300, 24).astype(np.float64):
        w = d / np.linalg.norm(d)
        if not _away_from_edges(oracle, N, w, 0.01):
            continue
        o = oracle.query_one(lut, N, w)
        if o.R < 0.1:
            continue  # x = R w lies on the surface only where R > 0 (signed glyphs dip below 0)
        x = o.R * w  # a point on the surface
        gF = np.array([(F(x + e * ax) - F(x - e * ax)) / (2 * e) for ax in np.eye(3)])
        gF /= np.linalg.norm(gF)
        assert np.allclose(np.array(o.normal[:]), gF, atol=2e-6)
        n_checked += 1
    assert n_checked > 100


def test_convergence_rates_against_direct_sh(oracle):
    L = 8
    c = I.sh_coeffs(1, L, 20063 + 1)[0]
    dirs = I.directions(20000, 25)
    Rt, Gt, _ = oracle.sh_eval(L, c, dirs)
    ev, eg = [], []
    for N in (16, 32):
        pool, off, Ns = oracle.make_pool([oracle.bake_sh(N, L, c)])
        out = oracle.query(pool, off, Ns, dirs)
        ev.append(np.sqrt(((out["R"] - Rt) ** 2).mean()))
        eg.append(np.sqrt((np.linalg.norm(out["grad"] - Gt, axis=1) ** 2).mean()))
    assert 12.0 < ev[0] / ev[1] < 20.0, ev   # h^4
    assert 6.0 < eg[0] / eg[1] < 10.0, eg    # h^3


def _golden_psnr():
    rows = []
    for line in open(os.path.join(GOLDEN, "psnr_value.txt")):
        if line.startswith("#") or not line.strip():
            continue
        N, bl, bc, he = line.split()
        rows.append((int(N), float(bl), float(bc), float(he)))
    return rows


def test_psnr_trend_matches_table(oracle):
    rows = _golden_psnr()
    gains = [rows[k + 1][3] - rows[k][3] for k in range(len(rows) - 1)]
    assert min(gains) > 30.0  # the paper: +30.5 and +30.4 dB per doubling of N
    L = 8
    c = I.sh_coeffs(1, L, 20063 + 1)[0]
    dirs = I.directions(100000, 26)
    Rt, _, _ = oracle.sh_eval(L, c, dirs)
    peak = np.abs(Rt).max()
    ps = []
    for N, *_ in rows:
        pool, off, Ns = oracle.make_pool([oracle.bake_sh(N, L, c)])
        err = oracle.query(pool, off, Ns, dirs)["R"] - Rt
        ps.append(20 * math.log10(peak / math.sqrt((err ** 2).mean())))
    mine = [ps[k + 1] - ps[k] for k in range(len(ps) - 1)]
    # The asymptotic O(h^4) rate is 24.1 dB per doubling; the paper's rougher glyph sits above it.
    assert all(20.0 < g < 40.0 for g in mine), mine


def test_seams_close_with_resolution(oracle):
    L = 8
    c = I.sh_coeffs(1, L, 27)[0]
    rng = np.random.default_rng(27)
    jumps = []
    for N in (8, 16, 32):
        lut = oracle.bake_sh(N, L, c)
        worst = 0.0
        for _ in range(200):
            # a point on the edge between face +x (k=0) and face +y (k=1): |x| = |y|
            z = rng.uniform(-0.5, 0.5)  # |z| < |x| = |y| keeps the point on that edge
            a = math.sqrt((1 - z * z) / 2)
            e = 1e-12
            wa = np.array([a + e, a, z])   # face 0 side
            wb = np.array([a, a + e, z])   # face 2 side
            oa, ob = oracle.query_one(lut, N, wa), oracle.query_one(lut, N, wb)
            assert oa.face == 0 and ob.face == 2
            worst = max(worst, abs(oa.R - ob.R))
        jumps.append(worst)
    assert jumps[0] > jumps[1] > jumps[2]
    assert jumps[1] / jumps[2] > 8.0
