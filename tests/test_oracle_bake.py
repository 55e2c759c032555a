"""Pins for the oracle's bake (Algorithm 1), procedural functions and bound.

Pins: constant functions bake to (r, 0, 0, 0); every stored texel, gutter included, equals
direct evaluation at its own centre direction (§3.2: gutters evaluated, not copied); the
stored derivative channels are the h-scaled chart derivatives (central differences of the
plain value path); the finite-difference stencil is exact on polynomials of degree <= 2 per
chart axis and agrees with the analytic bake to O(h^2) (§3.3); the bake is the linear map
lut = sum_k c_k B_k; closed forms of the bump and value-noise definitions.
"""
import math

import numpy as np
import pytest

import shm_inputs as I


def _centre_dir(oracle, f, i, j, N):
    wt = oracle.dir_tilde(f, oracle.texel_centre(i, N), oracle.texel_centre(j, N))
    return wt / np.linalg.norm(wt)


def test_constant_function_bakes_to_constant(oracle):
    N, L = 10, 4
    c = np.zeros(25)
    c[0] = 3.0
    lut = oracle.bake_sh(N, L, c)
    assert np.allclose(lut[..., 0], 3.0 / (2 * math.sqrt(math.pi)), atol=1e-14)
    assert np.abs(lut[..., 1:]).max() < 1e-14


def test_every_texel_is_evaluated_at_its_centre(oracle):
    N, L = 10, 4
    c = I.sh_coeffs(1, L, 20063)[0]
    lut = oracle.bake_sh(N, L, c)
    P = N + 2
    for f in range(6):
        for j in range(P):
            for i in range(P):
                w = _centre_dir(oracle, f, i, j, N)
                assert abs(lut[f, j, i, 0] - oracle.sh_basis(L, w) @ c) < 1e-13


def test_derivative_channels_are_h_scaled_chart_derivatives(oracle):
    N, L = 12, 6
    c = I.sh_coeffs(1, L, 5)[0]
    lut = oracle.bake_sh(N, L, c)
    e = 1e-5

    def val(f, u, v):
        wt = oracle.dir_tilde(f, u, v)
        return oracle.sh_basis(L, wt / np.linalg.norm(wt)) @ c

    rng = np.random.default_rng(10)
    for _ in range(60):
        f = int(rng.integers(0, 6))
        i, j = (int(x) for x in rng.integers(0, N + 2, size=2))
        u, v = oracle.texel_centre(i, N), oracle.texel_centre(j, N)
        ru = (val(f, u + e, v) - val(f, u - e, v)) / (2 * e)
        rv = (val(f, u, v + e) - val(f, u, v - e)) / (2 * e)
        ruv = (val(f, u + e, v + e) - val(f, u + e, v - e) - val(f, u - e, v + e) + val(f, u - e, v - e)) / (4 * e * e)
        assert abs(lut[f, j, i, 1] - ru / N) < 1e-8
        assert abs(lut[f, j, i, 2] - rv / N) < 1e-8
        assert abs(lut[f, j, i, 3] - ruv / N ** 2) < 1e-5 / N ** 2 * max(1, abs(ruv))


def test_fd_stencil_exact_on_quadratics(oracle):
    N = 9
    S = N + 4
    rng = np.random.default_rng(11)
    A = rng.normal(size=(3, 3))
    h = 1.0 / N
    cen = [(ii - 1.5) / N for ii in range(S)]
    samples = np.zeros((6, S, S))
    for f in range(6):
        for jj in range(S):
            for ii in range(S):
                u, v = cen[ii], cen[jj]
                samples[f, jj, ii] = sum(A[a, b] * u ** a * v ** b for a in range(3) for b in range(3))
    lut = oracle.bake_fd(N, samples, r0=0.25)
    for f in range(6):
        for j in range(N + 2):
            for i in range(N + 2):
                u, v = oracle.texel_centre(i, N), oracle.texel_centre(j, N)
                p = sum(A[a, b] * u ** a * v ** b for a in range(3) for b in range(3))
                pu = sum(A[a, b] * a * u ** (a - 1) * v ** b for a in range(1, 3) for b in range(3))
                pv = sum(A[a, b] * b * u ** a * v ** (b - 1) for a in range(3) for b in range(1, 3))
                puv = sum(A[a, b] * a * b * u ** (a - 1) * v ** (b - 1) for a in range(1, 3) for b in range(1, 3))
                assert abs(lut[f, j, i, 0] - (p - 0.25)) < 1e-13
                assert abs(lut[f, j, i, 1] - pu * h) < 1e-13
                assert abs(lut[f, j, i, 2] - pv * h) < 1e-13
                assert abs(lut[f, j, i, 3] - puv * h * h) < 1e-13


def _sh_samples(oracle, N, L, c):
    S = N + 4
    out = np.zeros((6, S, S))
    for f in range(6):
        for jj in range(S):
            for ii in range(S):
                w = _centre_dir(oracle, f, ii - 1, jj - 1, N)
                out[f, jj, ii] = oracle.sh_basis(L, w) @ c
    return out


def test_fd_bake_converges_to_analytic_at_h2(oracle):
    L = 6
    c = I.sh_coeffs(1, L, 12)[0]
    errs = []
    for N in (16, 32):
        a = oracle.bake_sh(N, L, c)
        fd = oracle.bake_fd(N, _sh_samples(oracle, N, L, c))
        assert np.abs(fd[..., 0] - a[..., 0]).max() < 1e-13
        errs.append(np.abs(fd[..., 1] - a[..., 1]).max() * N)  # error in r_u itself
    ratio = errs[0] / errs[1]
    assert 3.0 < ratio < 5.0, ratio  # O(h^2): halving h divides the error by ~4


def test_bake_is_linear_in_coefficients(oracle):
    N, L = 6, 3
    c = I.sh_coeffs(1, L, 13)[0]
    B = oracle.sh_basis_records(N, L)
    assert np.allclose(np.tensordot(c, B, axes=1), oracle.bake_sh(N, L, c), atol=1e-14)


def test_bound_is_an_upper_bound(oracle):
    N, L = 8, 8
    c = I.sh_coeffs(1, L, 14)[0]
    lut = oracle.bake_sh(N, L, c)
    b = oracle.lut_bound(lut, N)
    pool, off, Ns = oracle.make_pool([lut])
    out = oracle.query(pool, off, Ns, I.directions(20000, 15))
    assert np.abs(out["R"]).max() <= b
    const = np.zeros((6, N + 2, N + 2, 4))
    const[..., 0] = 0.5
    assert oracle.lut_bound(const, N, r0=1.0) == 1.5


def test_bump_closed_form(oracle):
    mu = np.array([[0.0, 0.0, 1.0]])
    amp = np.array([0.15])
    width = np.array([0.3])
    assert abs(oracle.bumps(mu[0], mu, amp, width) - 1.15) < 1e-15
    for th in (0.05, 0.2, 0.6, 1.5):
        w = np.array([math.sin(th), 0.0, math.cos(th)])
        ref = 1.0 + 0.15 * math.exp(-(1.0 - math.cos(th)) / 0.09)
        assert abs(oracle.bumps(w, mu, amp, width) - ref) < 1e-14


def test_value_noise_lattice_and_fade(oracle):
    key = np.array([17, 4242, 99], dtype=np.uint32)
    rng = np.random.default_rng(16)
    for _ in range(50):
        p = rng.integers(-50, 50, size=3).astype(np.float64)
        n0 = oracle.value_noise(p, key)
        assert -1.0 <= n0 < 1.0
        # the quintic fade has zero slope at lattice points: the noise is flat there
        e = 1e-4
        for ax in range(3):
            dp = np.zeros(3)
            dp[ax] = e
            assert abs(oracle.value_noise(p + dp, key) - oracle.value_noise(p - dp, key)) < 1e-9
    # continuity across a lattice plane
    for _ in range(50):
        p = rng.uniform(-20, 20, size=3)
        p[0] = math.floor(p[0])
        a = oracle.value_noise(p - [1e-12, 0, 0], key)
        b = oracle.value_noise(p + [1e-12, 0, 0], key)
        assert abs(a - b) < 1e-9


def test_hash_statistics(oracle):
    # The PCG3D bit pattern has no published test vector (parity of the exact bits is pinned only
    # between the oracle and the CUDA path); its mixing quality is pinned here.
    rng = np.random.default_rng(17)
    flips = []
    vals = []
    for _ in range(3000):
        v = rng.integers(0, 2 ** 32, size=3, dtype=np.uint64).astype(np.uint32)
        h = oracle.pcg3d(v)
        vals.append(h[0])
        bit = int(rng.integers(0, 96))
        v2 = v.copy()
        v2[bit // 32] ^= np.uint32(1 << (bit % 32))
        h2 = oracle.pcg3d(v2)
        flips.append(bin(int(h[0]) ^ int(h2[0])).count("1"))
    # measured ~14 of 32 bits; without the xorshift round a flip only reaches higher bits (~8)
    assert 12.5 < np.mean(flips) < 19.0
    u = np.array(vals, dtype=np.float64) / 2 ** 32
    assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1 / 12) < 0.01


def test_fbm_octave_sum(oracle):
    keys = I.fbm_keys(18)
    w = np.array([0.3, -0.5, 0.81])
    w /= np.linalg.norm(w)
    assert oracle.fbm(w, keys[:1], base_freq=2.0) == oracle.value_noise(2.0 * w, keys[0])
    two = oracle.fbm(w, keys[:2], base_freq=2.0, lacunarity=2.0, gain=0.5)
    assert abs(two - (oracle.value_noise(2.0 * w, keys[0]) + 0.5 * oracle.value_noise(4.0 * w, keys[1]))) < 1e-15


def test_fbm_sample_grid_directions(oracle):
    N = 6
    keys = I.fbm_keys(19)
    g = oracle.sample_grid_fbm(N, keys, amplitude=0.02)
    for (f, jj, ii) in [(0, 0, 0), (3, 4, 7), (5, N + 3, N + 3)]:
        w = _centre_dir(oracle, f, ii - 1, jj - 1, N)
        assert abs(g[f, jj, ii] - 0.02 * oracle.fbm(w, keys)) < 1e-16
