"""Pins for the oracle's mip levels (§4.7, Table lod).

Pins: a constant table stays constant at every coarse texel, gutter and margin included, for both
constructions; on a table holding an exactly representable chart polynomial
f = a x + b y + g x^2 the interior coarse records equal the closed form of "mean of the four child
values, then central differences at the coarse spacing" (the +g delta^2 term fixes the filter
footprint, a != b fixes u against v, the 1/Nc scale fixes the derivative rescaling); the naive
construction keeps the fine-scale derivative channels (half the correct slope record); and the
normal-error trend of Table lod on a synthetic L = 8 glyph.
"""
import os

import numpy as np

import shm_inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def _chart_poly_table(oracle, N, a, b, g):
    """Records of f(x, y) = a x + b y + g x^2 in each face's own chart (x = 2u - 1), every texel."""
    P = N + 2
    u = np.array([oracle.texel_centre(i, N) for i in range(P)])
    x = 2 * u - 1
    X, Y = np.meshgrid(x, x, indexing="xy")  # [j][i]
    rec = np.stack([a * X + b * Y + g * X ** 2, (2 * a + 4 * g * X) / N, np.full_like(X, 2 * b / N),
                    np.zeros_like(X)], axis=-1)
    return np.broadcast_to(rec, (6, P, P, 4)).copy()


def test_constant_table_stays_constant(oracle):
    N = 12
    lut = np.zeros((6, N + 2, N + 2, 4))
    lut[..., 0] = 0.75
    for coarse in (oracle.mip_consistent(lut), oracle.mip_naive(lut)):
        assert coarse.shape == (6, N // 2 + 2, N // 2 + 2, 4)
        assert np.abs(coarse[..., 0] - 0.75).max() < 1e-14
        assert np.abs(coarse[..., 1:]).max() < 1e-14


def test_consistent_level_on_a_chart_polynomial(oracle):
    Nf, a, b, g = 16, 0.3, -0.2, 0.15
    Nc = Nf // 2
    fine = _chart_poly_table(oracle, Nf, a, b, g)
    coarse = oracle.mip_consistent(fine)
    delta = 0.5 / Nc  # children sit at x_c +- 1/(2 Nc)
    for i in range(2, Nc):
        for j in range(2, Nc):
            xc = 2 * oracle.texel_centre(i, Nc) - 1
            yc = 2 * oracle.texel_centre(j, Nc) - 1
            want = [a * xc + b * yc + g * (xc ** 2 + delta ** 2), (2 * a + 4 * g * xc) / Nc, 2 * b / Nc, 0.0]
            for f in range(6):
                assert np.allclose(coarse[f, j, i], want, atol=1e-12), (f, i, j)


def test_naive_level_keeps_fine_scale_derivatives(oracle):
    Nf, a, b = 16, 0.3, -0.2
    Nc = Nf // 2
    fine = _chart_poly_table(oracle, Nf, a, b, 0.0)
    naive = oracle.mip_naive(fine)
    good = oracle.mip_consistent(fine)
    inner = naive[:, 2:Nc, 2:Nc]
    assert np.allclose(inner[..., 1], 2 * a / Nf, atol=1e-14)
    assert np.allclose(inner[..., 2], 2 * b / Nf, atol=1e-14)
    assert np.allclose(good[:, 2:Nc, 2:Nc, 1], 2 * inner[..., 1], atol=1e-12)
    # the value channel of a linear field is the same for both constructions
    assert np.allclose(inner[..., 0], good[:, 2:Nc, 2:Nc, 0], atol=1e-12)


def _normal_errors(oracle, lut, N, dirs, n_true):
    pool, off, Ns = oracle.make_pool([lut])
    out = oracle.query(pool, off, Ns, dirs)
    cosang = np.clip((out["normal"] * n_true).sum(1), -1.0, 1.0)
    ang = np.degrees(np.arccos(cosang))
    return ang.mean(), np.percentile(ang, 95)


def test_lod_table_trend(oracle):
    rows = np.loadtxt(os.path.join(HERE, "golden", "lod_table.txt"))
    L = 8
    c = I.sh_coeffs(1, L, 20063 + 1)[0]
    dirs = I.directions(20000, 5)
    _, _, n_true = oracle.sh_eval(L, c, dirs)
    good = naive = oracle.bake_sh(32, L, c)
    N = 32
    ratios, means = [], []
    for lvl in (1, 2, 3):
        good, naive, N = oracle.mip_consistent(good), oracle.mip_naive(naive), N // 2
        gm, gp = _normal_errors(oracle, good, N, dirs, n_true)
        nm, npct = _normal_errors(oracle, naive, N, dirs, n_true)
        print(f"level {lvl} {N}^2: correct {gm:.2f} / {gp:.2f} deg, naive {nm:.2f} / {npct:.2f} deg, ratio {nm / gm:.2f}"
              f"  (paper: {rows[lvl, 2]} / {rows[lvl, 3]}, {rows[lvl, 4]} / {rows[lvl, 5]}, {rows[lvl, 6]})")
        ratios.append(nm / gm)
        means.append(gm)
        assert npct > gp
    assert ratios[0] > 3.0 and ratios[1] > 1.5
    assert ratios[0] > ratios[1] > ratios[2] > 1.0
    assert ratios[2] < 2.0
    assert means[0] < means[1] < means[2]


def test_children_on_cube_edges_take_the_exact_tie(oracle):
    """Table = face index on each face (derivatives 0): every coarse sample is the mean face index of
    its four children.  Children near cube corners lie exactly on a cube edge (|X| = |Y| > 1); the
    expected face comes from exact rational arithmetic with ties -> lowest axis (§3.2 reading)."""
    from fractions import Fraction
    Nf = 6
    P = Nf + 2
    lut = np.zeros((6, P, P, 4))
    for f in range(6):
        lut[f, ..., 0] = f
    samples = oracle.mip_samples(lut)
    Sg = Nf // 2 + 4
    ties = 0
    for f in range(6):
        k, sg = f // 2, (-1 if f % 2 else 1)
        for jj in range(Sg):
            for ii in range(Sg):
                faces = []
                for b in range(2):
                    for a in range(2):
                        X = Fraction(2 * (2 * ii - 3 + a) - 1 - Nf, Nf)
                        Y = Fraction(2 * (2 * jj - 3 + b) - 1 - Nf, Nf)
                        d = [Fraction(0)] * 3
                        d[k], d[(k + 1) % 3], d[(k + 2) % 3] = Fraction(sg), X, Y
                        m = max(abs(x) for x in d)
                        kk = min(q for q in range(3) if abs(d[q]) == m)
                        ties += sum(abs(x) == m for x in d) > 1
                        faces.append(2 * kk + (d[kk] < 0))
                assert abs(samples[f, jj, ii] - sum(faces) / 4.0) < 1e-12, (f, jj, ii, faces)
    assert ties > 0
