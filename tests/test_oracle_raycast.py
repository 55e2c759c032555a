"""Pins for the oracle's ray caster (§3.1).

Pins: a constant-radius table is a sphere, so hit depth and normal have closed forms; on a
small scene of bump objects the bisection + Newton refinement lands on the root of F that a
60-step float64 bisection of the same bracket finds, and a dense 2000-sample march finds the
same nearest object on almost every pixel (the 32-sample march of this reading can step over a
thin sliver of surface near a silhouette).
"""
import math

import numpy as np

import shm_inputs as I


def _camera(oracle, W, H, eye=(0.0, 0.0, 6.0), fov=40.0):
    eye = np.array(eye)
    fwd = -eye / np.linalg.norm(eye)
    right = np.cross(fwd, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    return oracle.make_camera(eye, fwd, right, up, fov, W, H), (eye, fwd, right, up, math.tan(math.radians(fov) / 2))


def _ray(frame, W, H, px, py):
    eye, fwd, right, up, th = frame
    xn = (2 * (px + 0.5) / W - 1) * th * (W / H)
    yn = (1 - 2 * (py + 0.5) / H) * th
    d = fwd + xn * right + yn * up
    return eye, d / np.linalg.norm(d)


def test_sphere_closed_form(oracle):
    N = 8
    lut = np.zeros((6, N + 2, N + 2, 4))
    lut[..., 0] = 0.75
    pool, off, Ns = oracle.make_pool([lut])
    centre = np.array([[0.3, -0.2, 0.0]])
    W, H = 32, 24
    cam, frame = _camera(oracle, W, H)
    prm = oracle.make_raycast_params()
    out = oracle.raycast(pool, off, Ns, centre, [1.2], [1.5], [0], cam, prm, r0=np.array([0.25]))
    R = 1.2
    hits = 0
    for q in range(W * H):
        px, py = q % W, q // W
        o, d = _ray(frame, W, H, px, py)
        oc = o - centre[0]
        b = oc @ d
        disc = b * b - (oc @ oc - R * R)
        if disc <= 1e-6:
            assert out["obj_id"][q] == -1 or disc > -1e-6
            continue
        t = -b - math.sqrt(disc)
        assert out["obj_id"][q] == 0
        assert abs(out["depth"][q] - t) < 1e-9
        p = o + t * d
        assert np.allclose(out["normal"][q], (p - centre[0]) / R, atol=1e-7)
        hits += 1
    assert hits > 50


def test_value_only_sphere_closed_form(oracle):
    """The value-only baselines (§4.5) reproduce a constant exactly (bilinear and Catmull-Rom weights
    sum to one, their derivative weights to zero), so on a constant-radius value grid the ray caster's
    recon mode must hit the analytic sphere with the radial normal, like the Hermite path."""
    N = 8
    grid = np.full((6, N + 4, N + 4), 0.75)
    pool, off, Ns = oracle.make_value_pool([grid])
    centre = np.array([[0.3, -0.2, 0.0]])
    W, H = 32, 24
    cam, frame = _camera(oracle, W, H)
    R = 1.2
    for method in (oracle.RECON_BILINEAR, oracle.RECON_BICUBIC):
        prm = oracle.make_raycast_params(recon=method)
        out = oracle.raycast(pool, off, Ns, centre, [1.2], [1.5], [0], cam, prm, r0=np.array([0.25]))
        hits = 0
        for q in range(W * H):
            px, py = q % W, q // W
            o, d = _ray(frame, W, H, px, py)
            oc = o - centre[0]
            b = oc @ d
            disc = b * b - (oc @ oc - R * R)
            if disc <= 1e-6:
                assert out["obj_id"][q] == -1 or disc > -1e-6
                continue
            t = -b - math.sqrt(disc)
            assert out["obj_id"][q] == 0
            assert abs(out["depth"][q] - t) < 1e-9
            p = o + t * d
            assert np.allclose(out["normal"][q], (p - centre[0]) / R, atol=1e-7)
            hits += 1
        assert hits > 50


def _bump_scene(oracle, N=16):
    counts, offs, mu, amp, width = I.bump_params(2, 40)
    luts = []
    for o in range(2):
        s = slice(offs[o], offs[o + 1])
        samples = oracle.sample_grid_bumps(N, mu[s], amp[s], width[s])
        luts.append(oracle.bake_fd(N, samples, r0=1.0))
    pool, off, Ns = oracle.make_pool(luts)
    r0 = np.array([1.0, 1.0])
    rmax = np.array([oracle.lut_bound(l, N, 1.0) for l in luts])
    centre = np.array([[-1.1, 0.0, 0.0], [1.1, 0.2, -0.5]])
    return pool, off, Ns, r0, rmax, centre, luts


def _F(oracle, lut, N, r0, c, o, d, t):
    x = o + t * d - c
    return np.linalg.norm(x) - abs(oracle.query_one(lut, N, x, r0=r0).R)


def test_refinement_converges_to_bracketed_root(oracle):
    N = 16
    pool, off, Ns, r0, rmax, centre, luts = _bump_scene(oracle, N)
    W, H = 20, 14
    cam, frame = _camera(oracle, W, H)
    prm = oracle.make_raycast_params()
    out = oracle.raycast(pool, off, Ns, centre, [1.0, 1.0], rmax, [0, 1], cam, prm, r0=r0)
    n_hit = 0
    for q in range(W * H):
        ob = out["obj_id"][q]
        if ob < 0 or out["margin"][q] < 1e-3:
            continue
        o, d = _ray(frame, W, H, q % W, q // W)
        c = centre[ob]
        oc = o - c
        b = oc @ d
        sq = math.sqrt(b * b - (oc @ oc - rmax[ob] ** 2))
        t0, t1 = -b - sq, -b + sq
        F = lambda t: _F(oracle, luts[ob], N, 1.0, c, o, d, t)
        lo = hi = None
        for k in range(1, 33):
            if F(t0 + (t1 - t0) * k / 32) < 0:
                lo, hi = t0 + (t1 - t0) * (k - 1) / 32, t0 + (t1 - t0) * k / 32
                break
        assert lo is not None
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if F(mid) < 0:
                hi = mid
            else:
                lo = mid
        assert abs(out["depth"][q] - lo) < 1e-9
        n_hit += 1
    assert n_hit > 40


def test_dense_march_agrees(oracle):
    N = 16
    pool, off, Ns, r0, rmax, centre, luts = _bump_scene(oracle, N)
    W, H = 16, 10
    cam, frame = _camera(oracle, W, H)
    prm = oracle.make_raycast_params()
    out = oracle.raycast(pool, off, Ns, centre, [1.0, 1.0], rmax, [0, 1], cam, prm, r0=r0)
    agree = 0
    for q in range(W * H):
        o, d = _ray(frame, W, H, q % W, q // W)
        best, best_t = -1, math.inf
        for ob in range(2):
            c = centre[ob]
            oc = o - c
            b = oc @ d
            disc = b * b - (oc @ oc - rmax[ob] ** 2)
            if disc < 0:
                continue
            sq = math.sqrt(disc)
            t0, t1 = -b - sq, -b + sq
            ts = np.linspace(t0, t1, 2000)
            for t in ts:
                if _F(oracle, luts[ob], N, 1.0, c, o, d, t) < 0:
                    if t < best_t:
                        best, best_t = ob, t
                    break
        agree += int(best == out["obj_id"][q])
    assert agree >= int(0.97 * W * H)


def test_lod_refinement_allocation(oracle):
    """§3.1 refinement by projected size (reading: fewest bisections with M 2^b >= 128 p, Newton
    steps full from 64 px).  Checked against the closed-form projected radius and an independent
    float32 evaluation; more iterations for larger projected objects; off -> fixed counts."""
    W, H, fov = 1920, 1080, 45.0
    cam = oracle.make_camera([0.0, 0.0, 30.0], [0.0, 0.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], fov, W, H)
    off = oracle.make_raycast_params(march=32, bisect=14, newton=4, lod=0)
    assert oracle.lod_steps(cam, off, np.zeros(3), 1.0)[:2] == (14, 4)
    prm = oracle.make_raycast_params(march=32, bisect=16, newton=4, lod=1, bisect_min=8, newton_min=2)
    th = np.float32(math.tan(math.radians(fov / 2)))
    last = (0, 0)
    for D in (200.0, 100.0, 40.0, 20.0, 10.0, 5.0, 2.5, 1.2):
        rmax = 1.1
        b, n, p = oracle.lod_steps(cam, prm, np.array([0.0, 0.0, 30.0 - D]), rmax)
        assert abs(p - rmax * H / 2 / (D * math.tan(math.radians(fov / 2)))) <= 1e-5 * p
        f32 = np.float32
        dz = f32(30.0 - D) - f32(30.0)
        D32 = np.sqrt((f32(0.0) + f32(0.0)) + dz * dz, dtype=np.float32)
        p32 = (f32(rmax) * f32(0.5 * H)) / (D32 * th)
        assert p == p32
        want = next((k for k in range(8, 17) if 32 * 2.0 ** k >= 128 * float(p32)), 16)
        assert b == want and 8 <= b <= 16
        assert n == (4 if p >= 64 else 2)
        assert (b, n) >= last
        last = (b, n)
    assert last[0] >= 12 and last[1] == 4   # a close object gets the most refinement
