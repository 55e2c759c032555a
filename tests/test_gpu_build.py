"""GPU parity of the bake (Algorithm 1) against the FP64 oracle.

Record tolerances are derived from float32 arithmetic (each channel is compared against the
oracle's float64 record of the same function):
  SH bake      basis values carry ~K ulp; channel c error <= 4e-6 * max|channel c| (ch 3: 4e-5).
  FD bake      from identical float32 samples: differences of float32 numbers, error <= 2 ulp of the
               sample magnitude; from bumps / fBm evaluated on the device: the float32 evaluation
               error eps_S of one sample (measured below against the float64 samples) bounds every
               channel by 2 eps_S, since each channel is a difference of at most four samples / 4.
End to end, a device-built table queried on the device meets the query bar against the oracle's
table queried by the oracle.
"""
import numpy as np
import pytest
import torch

import oracle as O
import shm_inputs as I
from gpu_common import check_query, shm, upload_pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return shm()


def _rel_err(got, ref):
    return [np.abs(got[..., c] - ref[..., c]).max() / max(np.abs(ref[..., c]).max(), 1e-30) for c in range(4)]


def _split_basis(buf, N, L):
    K, M = (L + 1) ** 2, 4 * 6 * (N + 2) ** 2
    Kp = (K + 31) // 32 * 32
    full = buf[:K * M].reshape(K, M)
    hi = buf[K * M:K * M + M * Kp].reshape(M, Kp)
    lo = buf[K * M + M * Kp:K * M + 2 * M * Kp].reshape(M, Kp)
    return full, hi, lo, K, Kp


def _split_basis_t(buf, N, L):
    """The adjoint's operands after the forward ones, slabs [M16/16][Kp][16] with each row's four
    16-byte chunks permuted (chunk j of row k stored at j XOR (k/2)%4), unpacked to hiT, loT [Kp][M16]."""
    K, M = (L + 1) ** 2, 4 * 6 * (N + 2) ** 2
    Kp = (K + 31) // 32 * 32
    M16 = (M + 15) // 16 * 16
    o = K * M + 2 * M * Kp
    out = []
    for part in range(2):
        slabs = buf[o + part * M16 * Kp:o + (part + 1) * M16 * Kp].reshape(M16 // 16, Kp, 4, 4)
        k = np.arange(Kp)[:, None]
        src = np.arange(4)[None, :] ^ ((k >> 1) & 3)                 # stored chunk of logical chunk j
        logical = np.take_along_axis(slabs, src[None, :, :, None].repeat(slabs.shape[0], 0), axis=2)
        out.append(logical.reshape(M16 // 16, Kp, 16).transpose(1, 0, 2).reshape(Kp, M16))
    return out[0], out[1]


@pytest.mark.parametrize("N,L", [(10, 4), (32, 8), (7, 16)])
def test_sh_basis(S, N, L):
    buf = S.sh_basis(N, L).cpu().numpy()
    full, hi, lo, K, Kp = _split_basis(buf, N, L)
    B = full.astype(np.float64).reshape(K, 6, N + 2, N + 2, 4)
    ref = O.sh_basis_records(N, L)
    for c in range(4):
        scale = np.abs(ref[..., c]).max()
        err = np.abs(B[..., c] - ref[..., c]).max()
        assert err <= (4e-6 if c < 3 else 4e-5) * scale, (c, err / scale)
    # tensor-core operands: tf32 (low 13 mantissa bits clear) hi + lo reproduces the float32 basis
    assert np.all(hi.view(np.uint32) & 0x1FFF == 0) and np.all(lo.view(np.uint32) & 0x1FFF == 0)
    assert np.all(hi[:, K:] == 0) and np.all(lo[:, K:] == 0)
    fT = full.T.astype(np.float64)
    assert np.all(np.abs(hi[:, :K] + lo[:, :K].astype(np.float64) - fT) <= 2.0 ** -21 * np.abs(fT))
    # the adjoint's untransposed split: the same values row by row, zero rows k >= K
    hiT, loT = _split_basis_t(buf, N, L)
    M = full.shape[1]
    assert buf.size == K * M + 2 * M * Kp + 2 * ((M + 15) // 16 * 16) * Kp
    assert np.array_equal(hiT[:K, :M], hi[:, :K].T) and np.array_equal(loT[:K, :M], lo[:, :K].T)
    assert np.all(hiT[K:] == 0) and np.all(loT[K:] == 0) and np.all(hiT[:, M:] == 0) and np.all(loT[:, M:] == 0)


@pytest.mark.parametrize("engine", ["simt", "tcgen05"])
@pytest.mark.parametrize("N,L,G", [(10, 4, 1), (32, 8, 70), (12, 16, 3), (9, 8, 300)])
def test_sh_build(S, N, L, G, engine):
    """Against the oracle bake, element by element, within the float32 summation bound of the
    contraction, |err| <= (2^-20 + K 2^-24) sum_k |c_k| |B_k|, plus the float32 basis error that
    test_sh_basis bounds (4e-6 of each basis function's channel range, r_uv 4e-5) times |c_k|; the tf32
    split of the tensor-core engine contributes < 2^-21 sum_k |c_k B_k|."""
    c = I.sh_coeffs(G, L, 20063 + N)
    basis = S.sh_basis(N, L)
    r0 = np.linspace(0.0, 0.3, G).astype(np.float32)
    lut = S.alloc_lut(G, N, r0=r0)
    src = S.Source(kind=S.SHM_SRC_SH, L=L, coeffs=torch.from_numpy(c.astype(np.float32)).cuda(), basis=basis,
                   dev_status=torch.zeros(1, dtype=torch.int32, device="cuda"))
    S.build_lut(lut, src, ws=S.build_workspace(lut, src) if engine == "tcgen05" else None)
    assert src.dev_status.item() == 0
    got = lut.data.cpu().numpy().astype(np.float64).reshape(G, 6, N + 2, N + 2, 4)
    K = (L + 1) ** 2
    Babs = np.abs(O.sh_basis_records(N, L))
    Bmax = Babs.max(axis=(1, 2, 3))  # [K][4]: per basis function and channel
    worst = 0.0
    for g in range(min(G, 8)):
        cg = c[g].astype(np.float32).astype(np.float64)
        ref = O.bake_sh(N, L, cg)
        ref[..., 0] -= r0[g]
        # contraction rounding + the float32 basis error (<= 4e-6 of each basis channel's range, 4e-5 for r_uv)
        bound = (2.0 ** -20 + K * 2.0 ** -24) * np.tensordot(np.abs(cg), Babs, axes=1) + \
            np.abs(cg) @ Bmax * np.array([4e-6, 4e-6, 4e-6, 4e-5])
        err = np.abs(got[g] - ref)
        worst = max(worst, float((err / bound).max()))
        assert np.all(err <= bound), (g, float((err / bound).max()))
    print(f"{engine} N={N} L={L}: worst error / bound = {worst:.3f}")


@pytest.mark.parametrize("engine", ["simt", "tcgen05"])
@pytest.mark.parametrize("dtype,layout", [(0, 1), (1, 0), (2, 1)])
def test_sh_build_other_encodings(S, dtype, layout, engine):
    """Building straight into 16-bit / cell layout equals building f32 texel then packing."""
    N, L, G = 16, 8, 5
    c = torch.from_numpy(I.sh_coeffs(G, L, 3).astype(np.float32)).cuda()
    basis = S.sh_basis(N, L)
    a = S.alloc_lut(G, N, r0=[0.5] * G)
    src = S.Source(kind=S.SHM_SRC_SH, L=L, coeffs=c, basis=basis)
    ws = S.build_workspace(a, src) if engine == "tcgen05" else None
    S.build_lut(a, src, ws=ws)
    b = S.alloc_lut(G, N, dtype=dtype, layout=layout, r0=[0.5] * G)
    S.build_lut(b, src, ws=ws)
    p = S.like_lut(a, dtype=dtype, layout=layout)
    S.pack_lut(a, p)
    assert torch.equal(b.data, p.data)


def test_tensor_core_bake_matches_cuda_core_bake(S):
    """The full glyph-field shape (G = 16384, L = 8, N = 32): both engines within float32 rounding."""
    N, L, G = 32, 8, 16384
    c = torch.from_numpy(I.sh_coeffs(G, L, 20063 + 1).astype(np.float32)).cuda()
    basis = S.sh_basis(N, L)
    src = S.Source(kind=S.SHM_SRC_SH, L=L, coeffs=c, basis=basis)
    a = S.alloc_lut(G, N)
    S.build_lut(a, src)
    b = S.alloc_lut(G, N)
    S.build_lut(b, src, ws=S.build_workspace(b, src))
    A, B = a.data.view(G, -1, 4), b.data.view(G, -1, 4)
    for ch in range(4):
        scale = float(A[..., ch].abs().max())
        err = float((A[..., ch] - B[..., ch]).abs().max())
        assert err <= (4e-6 if ch < 3 else 4e-5) * scale, (ch, err / scale)
    # sampled glyphs against the oracle
    for g in (0, 4097, G - 1):
        ref = O.bake_sh(N, L, c[g].double().cpu().numpy())
        got = B[g].double().cpu().numpy().reshape(ref.shape)
        e = _rel_err(got, ref)
        assert max(e[:3]) <= 4e-6 and e[3] <= 4e-5, e


def test_sh_end_to_end_query(S):
    N, L, G = 32, 8, 8
    c = I.sh_coeffs(G, L, 77)
    c32 = c.astype(np.float32)
    basis = S.sh_basis(N, L)
    lut = S.alloc_lut(G, N)
    src = S.Source(kind=S.SHM_SRC_SH, L=L, coeffs=torch.from_numpy(c32).cuda(), basis=basis)
    S.build_lut(lut, src, ws=S.build_workspace(lut, src))
    per = 4096
    dirs = I.directions(G * per, 78)
    seg = torch.from_numpy(I.query_glyphs_csr(G, per)).cuda()
    out = S.query(lut, torch.from_numpy(dirs).cuda(), seg=seg)
    luts = [O.bake_sh(N, L, c32[g].astype(np.float64)) for g in range(G)]
    pool, off, Ns = O.make_pool(luts)
    glyph = np.repeat(np.arange(G), per).astype(np.int32)
    ref = O.query(pool, off, Ns, dirs, glyph=glyph)
    check_query(out, ref)


def test_fd_build_from_samples(S):
    Ns = [5, 16, 33]
    rng = np.random.default_rng(4)
    samples = [(1.0 + 0.1 * rng.normal(size=(6, n + 4, n + 4))).astype(np.float32) for n in Ns]
    offs = np.concatenate([[0], np.cumsum([s.size for s in samples])[:-1]]).astype(np.int64)
    lut = S.alloc_lut(3, Ns, r0=[1.0, 1.0, 0.0])
    src = S.Source(kind=S.SHM_SRC_SAMPLES, samples=torch.from_numpy(np.concatenate([s.ravel() for s in samples])).cuda(),
                   sample_offset=torch.from_numpy(offs).cuda())
    S.build_lut(lut, src)
    got = lut.data.cpu().numpy().astype(np.float64)
    o = 0
    for g, n in enumerate(Ns):
        ref = O.bake_fd(n, samples[g].astype(np.float64), r0=[1.0, 1.0, 0.0][g])
        sz = ref.size
        err = np.abs(got[o:o + sz].reshape(ref.shape) - ref).max()
        assert err <= 2 * 2.0 ** -23 * 1.6, err
        o += sz


def _bump_scene(n_obj, seed, choices):
    counts, offs, mu, amp, width = I.bump_params(n_obj, seed)
    Ns = I.uneven_N(n_obj, seed + 1, choices=choices)
    return counts, offs, mu, amp, width, Ns


def test_fd_build_bumps(S):
    counts, offs, mu, amp, width, Ns = _bump_scene(6, 90, (16, 32, 64, 128))
    lut = S.alloc_lut(6, [int(n) for n in Ns], r0=[1.0] * 6)
    mu32, amp32, w32 = mu.astype(np.float32), amp.astype(np.float32), width.astype(np.float32)
    src = S.Source(kind=S.SHM_SRC_BUMPS, bump_offset=torch.from_numpy(offs).cuda(),
                   mu=torch.from_numpy(mu32).cuda(), amp=torch.from_numpy(amp32).cuda(),
                   width=torch.from_numpy(w32).cuda())
    S.build_lut(lut, src)
    got = lut.data.cpu().numpy().astype(np.float64)
    o = 0
    worst = 0.0
    for g in range(6):
        s = slice(offs[g], offs[g + 1])
        n = int(Ns[g])
        samples = O.sample_grid_bumps(n, mu32[s].astype(np.float64), amp32[s].astype(np.float64),
                                      w32[s].astype(np.float64))
        ref = O.bake_fd(n, samples, r0=1.0)
        eps_S = 8 * 2.0 ** -24 * np.abs(amp32[s]).sum()  # float32 evaluation of the bump sum
        sz = ref.size
        err = np.abs(got[o:o + sz].reshape(ref.shape) - ref).max(axis=(0, 1, 2))
        worst = max(worst, (err / eps_S).max())
        assert np.all(err <= 2 * eps_S), (g, n, err, eps_S)
        o += sz
    print("bumps: worst record error / eps_S =", worst)


@pytest.mark.parametrize("N", [96, 104, 144])
def test_fd_build_bumps_uniform(S, N):
    """Uniform pools whole-face (N = 96) and split into 2 x 2 regions (N = 104: 53-texel regions,
    N = 144: 73) give the oracle's records within the float32 bound of the bump sum."""
    counts, offs, mu, amp, width = I.bump_params(3, 91 + N)
    lut = S.alloc_lut(3, N, r0=[1.0] * 3)
    mu32, amp32, w32 = mu.astype(np.float32), amp.astype(np.float32), width.astype(np.float32)
    src = S.Source(kind=S.SHM_SRC_BUMPS, bump_offset=torch.from_numpy(offs).cuda(),
                   mu=torch.from_numpy(mu32).cuda(), amp=torch.from_numpy(amp32).cuda(),
                   width=torch.from_numpy(w32).cuda())
    S.build_lut(lut, src)
    got = lut.data.cpu().numpy().astype(np.float64).reshape(3, 6, N + 2, N + 2, 4)
    for g in range(3):
        s = slice(offs[g], offs[g + 1])
        samples = O.sample_grid_bumps(N, mu32[s].astype(np.float64), amp32[s].astype(np.float64),
                                      w32[s].astype(np.float64))
        ref = O.bake_fd(N, samples, r0=1.0)
        eps_S = 8 * 2.0 ** -24 * np.abs(amp32[s]).sum()
        err = np.abs(got[g] - ref).max(axis=(0, 1, 2))
        assert np.all(err <= 2 * eps_S), (g, err, eps_S)


def test_fd_build_fbm_split(S):
    """fBm at N = 128 (faces split into 2 x 2 regions of 65 texels, directions divided per sample)."""
    N = 128
    keys = I.fbm_keys(12)
    lut = S.alloc_lut(1, N, r0=[1.0])
    src = S.Source(kind=S.SHM_SRC_FBM, octaves=8, keys=torch.from_numpy(keys.view(np.int32)).cuda(),
                   base_freq=2.0, lacunarity=2.0, gain=0.5, amplitude=0.02)
    S.build_lut(lut, src)
    got = lut.data.cpu().numpy().astype(np.float64).reshape(6, N + 2, N + 2, 4)
    ref = O.bake_fd(N, O.sample_grid_fbm(N, keys, 2.0, 2.0, 0.5, 0.02), r0=0.0)
    err = np.abs(got - ref).max(axis=(0, 1, 2))
    assert np.all(err <= 2 * 4e-8), err


def test_fd_build_fbm(S):
    N = 64
    keys = I.fbm_keys(11)
    lut = S.alloc_lut(1, N, r0=[1.0])
    src = S.Source(kind=S.SHM_SRC_FBM, octaves=8, keys=torch.from_numpy(keys.view(np.int32)).cuda(),
                   base_freq=2.0, lacunarity=2.0, gain=0.5, amplitude=0.02)
    S.build_lut(lut, src)
    got = lut.data.cpu().numpy().astype(np.float64).reshape(6, N + 2, N + 2, 4)
    ref = O.bake_fd(N, O.sample_grid_fbm(N, keys, 2.0, 2.0, 0.5, 0.02), r0=0.0)
    err = np.abs(got - ref).max(axis=(0, 1, 2))
    print("fbm N=64 record errors:", err, "channel max:", np.abs(ref).max(axis=(0, 1, 2)))
    eps_S = 4e-8  # float32 direction and lattice coordinate rounding, amplitude 0.02
    assert np.all(err <= 2 * eps_S), err


def test_fbm_planet_sampled_texels(S):
    """Full planet resolution N = 2048: sampled texels against the oracle's one-by-one bake."""
    N = 2048
    keys = I.fbm_keys(20063 + 3)
    lut = S.alloc_lut(1, N, r0=[1.0])
    src = S.Source(kind=S.SHM_SRC_FBM, octaves=8, keys=torch.from_numpy(keys.view(np.int32)).cuda(),
                   base_freq=2.0, lacunarity=2.0, gain=0.5, amplitude=0.02)
    S.build_lut(lut, src)
    P = N + 2
    rng = np.random.default_rng(12)
    got = lut.data.view(-1, 4)
    errs = []
    for _ in range(40):
        f, j, i = int(rng.integers(0, 6)), int(rng.integers(0, P)), int(rng.integers(0, P))
        # the oracle bakes a 1-texel-interior patch around (i, j) by evaluating its 3x3 sample stencil
        w = []
        stencil = np.zeros((3, 3))
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                wt = O.dir_tilde(f, O.texel_centre(i + di, N), O.texel_centre(j + dj, N))
                stencil[dj + 1, di + 1] = 0.02 * O.fbm(wt / np.linalg.norm(wt), keys)
        ref = np.array([stencil[1, 1], (stencil[1, 2] - stencil[1, 0]) / 2, (stencil[2, 1] - stencil[0, 1]) / 2,
                        (stencil[2, 2] - stencil[0, 2] - stencil[2, 0] + stencil[0, 0]) / 4])
        rec = got[(f * P + j) * P + i].double().cpu().numpy()
        errs.append(np.abs(rec - ref))
    errs = np.array(errs)
    print("planet sampled record errors (max per channel):", errs.max(0))
    assert np.all(errs <= 8e-8)


def test_bounds(S):
    luts = [O.bake_sh(n, 6, I.sh_coeffs(1, 6, 50 + n)[0]) for n in (4, 9, 20)]
    r0 = np.array([0.0, 0.5, -0.25], dtype=np.float32)
    L, stored = upload_pool(S, luts, r0=r0)
    got = S.lut_bounds(L).cpu().numpy()
    pool = stored.reshape(-1, 4)
    off, Ns = O.make_pool(luts)[1:]
    for g in range(3):
        n = Ns[g]
        glut = pool[off[g]:off[g] + 6 * (n + 2) ** 2].reshape(6, n + 2, n + 2, 4)
        ref = O.lut_bound(glut, n, float(r0[g]))
        assert abs(got[g] - ref) <= 4e-7 * ref


def test_pack_round_trip(S):
    luts = [O.bake_sh(n, 4, I.sh_coeffs(1, 4, n)[0]) for n in (3, 8)]
    L, stored = upload_pool(S, luts, r0=np.array([0.25, 0.0], np.float32))
    C = S.like_lut(L, layout=1)
    S.pack_lut(L, C)
    T = S.like_lut(C, layout=0)
    S.pack_lut(C, T)
    assert torch.equal(T.data, L.data)


def test_sh_eval_direct(S):
    G, L = 5, 16
    c = I.sh_coeffs(G, L, 61).astype(np.float32)
    dirs = I.directions(20000, 62)
    glyph = I.random_glyph_ids(20000, G, 63)
    R, grad, normal = S.sh_eval(L, torch.from_numpy(c).cuda(), torch.from_numpy(dirs).cuda(),
                                glyph=torch.from_numpy(glyph).cuda())
    Rr, Gr, Nr = O.sh_eval(L, c.astype(np.float64), dirs, glyph=glyph)
    out = {"R": R, "grad": grad, "normal": normal}
    check_query(out, {"R": Rr, "grad": Gr, "normal": Nr})
