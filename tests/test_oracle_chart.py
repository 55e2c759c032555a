"""Pins for the oracle's cubemap chart, tangents, metric and S^2 gradient (§3.2, §3.4).

Each check compares against something the oracle does not compute itself: the round trip
through the chart definition, central differences of the normalised direction, the closed
form det G = 16 / rho^6 (derived below), and the defining equations grad.e1 = R_u,
grad.e2 = R_v, grad . w = 0 of §3.4.
"""
import numpy as np
import pytest

import shm_inputs as I


def _rand_dirs(n, seed):
    d = I.directions(n, seed).astype(np.float64)
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_round_trip(oracle):
    for w in _rand_dirs(2000, 11):
        f, u, v = oracle.face_uv(w)
        assert 0.0 <= u <= 1.0 and 0.0 <= v <= 1.0
        wt = oracle.dir_tilde(f, u, v)
        assert np.allclose(wt / np.linalg.norm(wt), w, atol=1e-15, rtol=0)


def test_face_is_dominant_axis_and_sign(oracle):
    for w in _rand_dirs(2000, 12):
        f, _, _ = oracle.face_uv(w)
        k = int(np.argmax(np.abs(w)))
        assert f == 2 * k + (1 if w[k] < 0 else 0)


@pytest.mark.parametrize("w,face", [((1.0, 1.0, 0.5), 0), ((-1.0, 1.0, 0.0), 1), ((0.0, 1.0, 1.0), 2),
                                    ((0.2, -1.0, -1.0), 3), ((-1.0, -1.0, -1.0), 1), ((0.3, 0.1, -2.0), 5)])
def test_face_ties_lowest_axis(oracle, w, face):
    assert oracle.face_uv(np.array(w))[0] == face


def test_tangents_match_finite_differences(oracle):
    rng = np.random.default_rng(1)
    eps = 1e-6
    for _ in range(200):
        f = int(rng.integers(0, 6))
        u, v = rng.uniform(-0.05, 1.05, size=2)

        def w_of(uu, vv):
            wt = oracle.dir_tilde(f, uu, vv)
            return wt / np.linalg.norm(wt)

        e1_fd = (w_of(u + eps, v) - w_of(u - eps, v)) / (2 * eps)
        e2_fd = (w_of(u, v + eps) - w_of(u, v - eps)) / (2 * eps)
        e1, e2 = oracle.tangents(f, u, v)
        assert np.allclose(e1, e1_fd, atol=1e-8)
        assert np.allclose(e2, e2_fd, atol=1e-8)


def test_det_metric_closed_form(oracle):
    # e_xi = (2/rho)(I - w w^T) b or c with x = 2u-1, y = 2v-1, rho^2 = 1+x^2+y^2 gives
    # g11 = 4(1 - x^2/rho^2)/rho^2, g22 = 4(1 - y^2/rho^2)/rho^2, g12 = -4xy/rho^4,
    # so det G = 16/rho^4 (1 - (x^2+y^2)/rho^2) = 16/rho^6.
    rng = np.random.default_rng(2)
    for _ in range(500):
        f = int(rng.integers(0, 6))
        u, v = rng.uniform(0, 1, size=2)
        g11, g12, g22 = oracle.metric(f, u, v)
        x, y = 2 * u - 1, 2 * v - 1
        rho2 = 1 + x * x + y * y
        det = g11 * g22 - g12 * g12
        assert abs(det - 16.0 / rho2 ** 3) < 1e-12
        # det G lies in [16/27, 16] on every face, so the clamp of §3.4 never binds there
        assert 16.0 / 27.0 - 1e-12 <= det <= 16.0 + 1e-12


def test_gradient_solves_defining_equations(oracle):
    rng = np.random.default_rng(3)
    for _ in range(500):
        f = int(rng.integers(0, 6))
        u, v = rng.uniform(0, 1, size=2)
        Ru, Rv = rng.normal(size=2)
        g = oracle.s2_gradient(f, u, v, Ru, Rv)
        e1, e2 = oracle.tangents(f, u, v)
        wt = oracle.dir_tilde(f, u, v)
        w = wt / np.linalg.norm(wt)
        assert abs(g @ e1 - Ru) < 1e-12
        assert abs(g @ e2 - Rv) < 1e-12
        assert abs(g @ w) < 1e-12


def test_gradient_closed_form(oracle):
    # grad = (rho/2) [R_u b + R_v c - (x R_u + y R_v) a] is tangent and satisfies grad.e1 = R_u,
    # grad.e2 = R_v, hence equals the unique Cramer solution.
    rng = np.random.default_rng(4)
    for _ in range(500):
        f = int(rng.integers(0, 6))
        u, v = rng.uniform(0, 1, size=2)
        Ru, Rv = rng.normal(size=2)
        a, b, c = oracle.face_frame(f)
        x, y = 2 * u - 1, 2 * v - 1
        rho = np.sqrt(1 + x * x + y * y)
        closed = 0.5 * rho * (Ru * b + Rv * c - (x * Ru + y * Rv) * a)
        assert np.allclose(oracle.s2_gradient(f, u, v, Ru, Rv), closed, atol=1e-12)


def test_face_frames_are_right_or_left_handed_orthonormal(oracle):
    for f in range(6):
        a, b, c = oracle.face_frame(f)
        M = np.stack([a, b, c])
        assert np.allclose(M @ M.T, np.eye(3))


def test_texel_centres_cell_centred(oracle):
    N = 10
    assert oracle.texel_centre(0, N) == -0.05
    assert oracle.texel_centre(1, N) == 0.05
    assert abs(oracle.texel_centre(N + 1, N) - 1.05) < 1e-15


def test_normal_of_constant_radius_is_direction(oracle):
    for w in _rand_dirs(50, 13):
        assert np.allclose(oracle.normal(w, 2.0, np.zeros(3)), w, atol=1e-15)
