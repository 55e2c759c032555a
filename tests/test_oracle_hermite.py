"""Pins for the oracle's Hermite reconstruction and derivative extraction (§3.3).

Pins: the textbook cubic-Hermite end conditions of the 1-D basis; reproduction of the stored
value and scaled derivatives at texel centres; exact reproduction of any per-face bicubic
polynomial whose exact derivatives are stored (this fixes the tensor structure, the h scaling,
the r_uv channel and the cell-centred texel convention at once); C^1 continuity across cell
edges inside a face.
"""
import numpy as np
import pytest


def test_basis_end_conditions(oracle):
    H0, dH0, _ = oracle.hermite_basis(0.0)
    H1, dH1, _ = oracle.hermite_basis(1.0)
    # values: H0 interpolates the left value, H1 the right one, H^d vanish at both ends
    assert np.array_equal(H0, [1, 0, 0, 0]) and np.array_equal(H1, [0, 1, 0, 0])
    # slopes: only H0d has unit slope at 0, only H1d at 1
    assert np.array_equal(dH0, [0, 0, 1, 0]) and np.array_equal(dH1, [0, 0, 0, 1])


def test_basis_partition_and_second_derivatives(oracle):
    for s in np.linspace(0, 1, 41):
        H, dH, ddH = oracle.hermite_basis(s)
        assert abs(H[0] + H[1] - 1.0) < 1e-15
        eps = 1e-6
        Hp, _, _ = oracle.hermite_basis(s + eps)
        Hm, _, _ = oracle.hermite_basis(s - eps)
        assert np.allclose((Hp - Hm) / (2 * eps), dH, atol=1e-8)
        _, dHp, _ = oracle.hermite_basis(s + eps)
        _, dHm, _ = oracle.hermite_basis(s - eps)
        assert np.allclose((dHp - dHm) / (2 * eps), ddH, atol=1e-7)


def test_cell_location(oracle):
    N = 10
    # centres at (i - 1/2)/N: u = 0 lies halfway between gutter texel 0 and interior texel 1
    assert oracle.cell(N, 0.0) == (0, 0.5)
    assert oracle.cell(N, 1.0) == (N, 0.5)
    i, s = oracle.cell(N, 0.05)
    assert i == 1 and abs(s) < 1e-15
    i, s = oracle.cell(N, 0.37)
    assert i == 4 and abs(s - 0.2) < 1e-12


def test_reconstruction_at_texel_centres(oracle):
    N, P = 6, 8
    rng = np.random.default_rng(5)
    face = rng.normal(size=(P, P, 4))
    for j in range(N + 1):
        for i in range(N + 1):
            out = oracle.hermite_eval(face, N, i, j, 0.0, 0.0)
            assert abs(out[0] - face[j, i, 0]) < 1e-14
            assert abs(out[1] - face[j, i, 1]) < 1e-14   # dr/ds = r_u h
            assert abs(out[2] - face[j, i, 2]) < 1e-14   # dr/dt = r_v h
            assert abs(out[4] - face[j, i, 3]) < 1e-14   # d2r/dsdt = r_uv h^2
            out1 = oracle.hermite_eval(face, N, i, j, 1.0, 1.0)
            assert abs(out1[0] - face[j + 1, i + 1, 0]) < 1e-14


@pytest.mark.parametrize("N", [5, 10, 16])
def test_bicubic_polynomial_reproduction(oracle, N):
    P = N + 2
    rng = np.random.default_rng(N)
    A = rng.normal(size=(4, 4))  # p(u,v) = sum A[a,b] u^a v^b

    def p(u, v, du=0, dv=0):
        tot = 0.0
        for a in range(4):
            for b in range(4):
                if a < du or b < dv:
                    continue
                ca = np.prod(range(a - du + 1, a + 1)) if du else 1.0
                cb = np.prod(range(b - dv + 1, b + 1)) if dv else 1.0
                tot += A[a, b] * ca * cb * u ** (a - du) * v ** (b - dv)
        return tot

    h = 1.0 / N
    lut = np.zeros((6, P, P, 4))
    f = 2
    for j in range(P):
        for i in range(P):
            u, v = oracle.texel_centre(i, N), oracle.texel_centre(j, N)
            lut[f, j, i] = [p(u, v), p(u, v, 1, 0) * h, p(u, v, 0, 1) * h, p(u, v, 1, 1) * h * h]
    for _ in range(200):
        u, v = rng.uniform(0, 1, size=2)
        i, s = oracle.cell(N, u)
        j, t = oracle.cell(N, v)
        out = oracle.hermite_eval(lut[f], N, i, j, s, t)
        assert abs(out[0] - p(u, v)) < 1e-11
        assert abs(N * out[1] - p(u, v, 1, 0)) < 1e-9
        assert abs(N * out[2] - p(u, v, 0, 1)) < 1e-9
        assert abs(N * N * out[4] - p(u, v, 1, 1)) < 1e-7


def test_c1_across_cell_edges(oracle):
    N, P = 8, 10
    rng = np.random.default_rng(6)
    face = rng.normal(size=(P, P, 4))
    eps = 1e-9
    for _ in range(100):
        i = int(rng.integers(0, N))
        j = int(rng.integers(0, N + 1))
        t = rng.uniform()
        left = oracle.hermite_eval(face, N, i, j, 1.0 - eps, t)
        right = oracle.hermite_eval(face, N, i + 1, j, eps, t)
        assert abs(left[0] - right[0]) < 1e-7          # value continuous
        assert abs(left[1] - right[1]) < 1e-7          # d/ds continuous (C^1)
        assert abs(left[2] - right[2]) < 1e-7          # d/dt continuous


def test_weights_match_eval(oracle):
    N, P = 7, 9
    rng = np.random.default_rng(7)
    face = rng.normal(size=(P, P, 4))
    for _ in range(50):
        i, j = rng.integers(0, N + 1, size=2)
        s, t = rng.uniform(size=2)
        W = oracle.hermite_weights(s, t)
        recs = np.stack([face[j, i], face[j, i + 1], face[j + 1, i], face[j + 1, i + 1]])
        out = oracle.hermite_eval(face, N, int(i), int(j), s, t)
        for k in range(3):
            assert abs((W[k] * recs).sum() - out[k]) < 1e-13
