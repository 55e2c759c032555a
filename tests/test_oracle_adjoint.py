"""Pins for the oracle's adjoint of the query and of the SH bake.

Pins: central finite differences of the forward query (query.c) with respect to table
entries and query directions; the dot-product test <J x, y> = <x, J^T y> for the part that is
linear in the table; the bake adjoint is the exact transpose of the linear bake.
"""
import numpy as np

import shm_inputs as I


def _setup(oracle, N=10, L=6, seed=30):
    c = I.sh_coeffs(1, L, seed)[0]
    c[0] += 2.0  # keep R well away from 0 for the normal's normalisation
    lut = oracle.bake_sh(N, L, c)
    return lut


def _loss(oracle, lut, N, d, gR, gG, gn, r0=0.3):
    o = oracle.query_one(lut, N, d, r0=r0)
    return gR * o.R + np.dot(gG, o.grad[:]) + np.dot(gn, o.normal[:])


def _interior(oracle, N, d, margin=0.02):
    w = d / np.linalg.norm(d)
    f, u, v = oracle.face_uv(w)
    su, sv = (u * N + 0.5) % 1.0, (v * N + 0.5) % 1.0
    a = np.sort(np.abs(w))
    return min(su, 1 - su, sv, 1 - sv) > margin and a[2] - a[1] > 1e-3


def test_vjp_table_entries_vs_finite_differences(oracle):
    N = 10
    lut = _setup(oracle, N)
    rng = np.random.default_rng(31)
    e = 1e-6
    for d in I.directions(40, 32).astype(np.float64):
        if not _interior(oracle, N, d):
            continue
        gR, gG, gn = rng.normal(), rng.normal(size=3), rng.normal(size=3)
        dl, _ = oracle.query_vjp_one(lut, N, d, gR, gG, gn, r0=0.3)
        nz = np.argwhere(dl != 0)
        assert len(nz) == 16  # exactly the 4 corner records x 4 channels
        for idx in nz[:: 3]:
            idx = tuple(idx)
            lp, lm = lut.copy(), lut.copy()
            lp[idx] += e
            lm[idx] -= e
            fd = (_loss(oracle, lp, N, d, gR, gG, gn) - _loss(oracle, lm, N, d, gR, gG, gn)) / (2 * e)
            assert abs(dl[idx] - fd) < 1e-6 * max(1.0, abs(fd))


def test_vjp_directions_vs_finite_differences(oracle):
    N = 10
    lut = _setup(oracle, N)
    rng = np.random.default_rng(33)
    e = 1e-7
    n_checked = 0
    for d in I.directions(200, 34).astype(np.float64):
        d = d * rng.uniform(0.5, 2.0)  # unnormalised inputs are allowed
        if not _interior(oracle, N, d, margin=0.05):
            continue
        gR, gG, gn = rng.normal(), rng.normal(size=3), rng.normal(size=3)
        _, dd = oracle.query_vjp_one(lut, N, d, gR, gG, gn, r0=0.3)
        fd = np.array([(_loss(oracle, lut, N, d + e * ax, gR, gG, gn) -
                        _loss(oracle, lut, N, d - e * ax, gR, gG, gn)) / (2 * e) for ax in np.eye(3)])
        assert np.allclose(dd, fd, atol=2e-6 * max(1.0, np.abs(fd).max()))
        n_checked += 1
    assert n_checked > 50


def test_dot_product_linear_part(oracle):
    N = 8
    rng = np.random.default_rng(35)
    X = rng.normal(size=(6, N + 2, N + 2, 4))
    pool, off, Ns = oracle.make_pool([X])
    dirs = I.directions(300, 36)
    y = rng.normal(size=300)
    JX = oracle.query(pool, off, Ns, dirs)["R"]
    JTy, _ = oracle.query_vjp(pool, off, Ns, dirs, gR=y, want_ddirs=False)
    lhs, rhs = JX @ y, (pool * JTy).sum()
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_bake_vjp_is_transpose(oracle):
    N, L = 6, 4
    rng = np.random.default_rng(37)
    c = rng.normal(size=(L + 1) ** 2)
    Y = rng.normal(size=(6, N + 2, N + 2, 4))
    lhs = (oracle.bake_sh(N, L, c) * Y).sum()
    rhs = c @ oracle.bake_sh_vjp(N, L, Y)
    assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


def test_fit_loss_gradient_vs_finite_differences(oracle):
    import oracle.fit as OF
    N = 8
    lut = _setup(oracle, N, seed=41)
    pool, off, Ns = oracle.make_pool([lut])
    dirs = I.directions(200, 42)
    rng = np.random.default_rng(43)
    Rt = rng.normal(size=200) * 0.1 + 0.7
    nt = rng.normal(size=(200, 3))
    nt /= np.linalg.norm(nt, axis=1, keepdims=True)
    loss, g = OF.loss_and_grad(pool, off, Ns, dirs, Rt, nt, 1.0, 0.5)
    e = 1e-6
    for idx in [tuple(x) for x in np.argwhere(g != 0)[::97][:12]]:
        p2 = pool.copy()
        p2[idx] += e
        lp, _ = OF.loss_and_grad(p2, off, Ns, dirs, Rt, nt, 1.0, 0.5)
        p2[idx] -= 2 * e
        lm, _ = OF.loss_and_grad(p2, off, Ns, dirs, Rt, nt, 1.0, 0.5)
        assert abs((lp - lm) / (2 * e) - g[idx]) <= 1e-5 * max(1.0, abs(g[idx]))


def test_adam_first_step_closed_form():
    import oracle.fit as OF
    rng = np.random.default_rng(44)
    g = rng.normal(size=1000)
    p, m, v = OF.adam(np.zeros(1000), g, np.zeros(1000), np.zeros(1000), 1, 0.01, eps=1e-8)
    # bias-corrected first moments are g and g^2: the step is -lr g / (|g| + eps)
    assert np.allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
