"""Pins for the oracle's real spherical harmonics and their exact chart derivatives (§3.3).

Pins: Y_00 = 1/(2 sqrt(pi)); the addition theorem sum_m Y_lm^2 = (2l+1)/(4 pi) (independent of
phase convention); orthonormality by a quadrature exact to degree 2L; the l = 1 span; scipy's
complex spherical harmonics (with the Condon-Shortley phase removed); hyper-dual chart
derivatives against central differences; and the paper's chain rule r_u = grad_{S^2} r . e1
against directional differences on the sphere.
"""
import math

import numpy as np
import pytest
import scipy.special as sp

import shm_inputs as I


def _dirs(n, seed):
    d = I.directions(n, seed).astype(np.float64)
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_y00(oracle):
    assert abs(oracle.sh_basis(0, [0.3, 0.4, 0.5])[0] - 1.0 / (2.0 * math.sqrt(math.pi))) < 1e-15


@pytest.mark.parametrize("L", [4, 8, 16])
def test_addition_theorem(oracle, L):
    for w in _dirs(50, L):
        Y = oracle.sh_basis(L, w)
        for l in range(L + 1):
            s = (Y[l * l:(l + 1) * (l + 1)] ** 2).sum()
            assert abs(s - (2 * l + 1) / (4 * math.pi)) < 1e-11 * (2 * l + 1)


@pytest.mark.parametrize("L", [4, 8])
def test_orthonormality_quadrature(oracle, L):
    nz, nphi = L + 1, 2 * L + 2
    z, wz = np.polynomial.legendre.leggauss(nz)
    phi = 2 * np.pi * np.arange(nphi) / nphi
    K = (L + 1) ** 2
    Gm = np.zeros((K, K))
    for zi, wzi in zip(z, wz):
        for ph in phi:
            r = math.sqrt(1 - zi * zi)
            Y = oracle.sh_basis(L, [r * math.cos(ph), r * math.sin(ph), zi])
            Gm += wzi * (2 * np.pi / nphi) * np.outer(Y, Y)
    assert np.abs(Gm - np.eye(K)).max() < 1e-12


def test_l1_span(oracle):
    c = math.sqrt(3.0 / (4.0 * math.pi))
    for w in _dirs(20, 3):
        Y = oracle.sh_basis(1, w)
        assert np.allclose(Y[1:4], c * np.array([w[1], w[2], w[0]]), atol=1e-15)


@pytest.mark.parametrize("L", [8, 16])
def test_against_scipy(oracle, L):
    for w in _dirs(30, 100 + L):
        theta = math.acos(max(-1.0, min(1.0, w[2])))
        phi = math.atan2(w[1], w[0]) % (2 * math.pi)
        Y = oracle.sh_basis(L, w)
        for l in range(L + 1):
            ref0 = sp.sph_harm_y(l, 0, theta, phi).real
            assert abs(Y[l * l + l] - ref0) < 1e-11
            for m in range(1, l + 1):
                z = sp.sph_harm_y(l, m, theta, phi) * (-1) ** m  # remove Condon-Shortley phase
                assert abs(Y[l * l + l + m] - math.sqrt(2) * z.real) < 1e-10
                assert abs(Y[l * l + l - m] - math.sqrt(2) * z.imag) < 1e-10


def test_chart_derivatives_vs_finite_differences(oracle):
    L = 8
    c = I.sh_coeffs(1, L, 42)[0]
    rng = np.random.default_rng(8)
    e = 1e-5
    for _ in range(100):
        f = int(rng.integers(0, 6))
        u, v = rng.uniform(-0.05, 1.05, size=2)
        r, ru, rv, ruv = oracle.sh_chart(L, c, f, u, v)
        val = lambda uu, vv: oracle.sh_chart(L, c, f, uu, vv)[0]
        assert abs(ru - (val(u + e, v) - val(u - e, v)) / (2 * e)) < 1e-7
        assert abs(rv - (val(u, v + e) - val(u, v - e)) / (2 * e)) < 1e-7
        fd_uv = (val(u + e, v + e) - val(u + e, v - e) - val(u - e, v + e) + val(u - e, v - e)) / (4 * e * e)
        assert abs(ruv - fd_uv) < 2e-4 * max(1.0, abs(ruv))


def test_chain_rule_gradient_vs_sphere_differences(oracle):
    L = 8
    c = I.sh_coeffs(1, L, 43)[0]
    e = 1e-6
    rng = np.random.default_rng(9)
    for w in _dirs(100, 44):
        r, g = oracle.sh_value_grad(L, c, w)
        assert abs(g @ w) < 1e-12
        t = rng.normal(size=3)
        t -= (t @ w) * w
        t /= np.linalg.norm(t)
        wp = (w + e * t) / np.linalg.norm(w + e * t)
        wm = (w - e * t) / np.linalg.norm(w - e * t)
        fd = (oracle.sh_value_grad(L, c, wp)[0] - oracle.sh_value_grad(L, c, wm)[0]) / (2 * e)
        assert abs(g @ t - fd) < 1e-7
        # the paper's chain rule r_u = grad . e1, r_v = grad . e2
        f, u, v = oracle.face_uv(w)
        _, ru, rv, _ = oracle.sh_chart(L, c, f, u, v)
        e1, e2 = oracle.tangents(f, u, v)
        assert abs(g @ e1 - ru) < 1e-11 and abs(g @ e2 - rv) < 1e-11
