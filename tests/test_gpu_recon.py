"""GPU parity of the value-only reconstruction baselines (shm_query_recon) and of value-table
builds (SHM_LAYOUT_VALUE) against the FP64 oracle (oracle/recon.c) on identical stored values.

Bar: value <= 1e-5 max|R|; chart gradient (analytic for Catmull-Rom, central differences of the
float32 reconstruction otherwise) <= 1e-4 max|grad R| + N * 2^-23 max|R| (a difference of two
float32 lookups divided by 2h); normals within the bound those propagate to; cell / texel
indices bit-exact away from edges and ties."""
import numpy as np
import pytest
import torch

import oracle as O
import shm_inputs as I
from gpu_common import near_edge, shm

pytestmark = pytest.mark.gpu

METHODS = [0, 1, 2, 3]


@pytest.fixture(scope="module")
def S():
    return shm()


def upload_value_pool(S, grids, dtype=0, r0=None):
    Ns = [g.shape[1] - 4 for g in grids]
    uniform = len(set(Ns)) == 1
    lut = S.alloc_lut(len(grids), Ns[0] if uniform else Ns, dtype, S.SHM_LAYOUT_VALUE, r0=r0)
    host = np.concatenate([np.asarray(g, dtype=np.float32).reshape(-1) for g in grids])
    lut.data.copy_(torch.from_numpy(host).to(lut.data.dtype))
    stored = lut.data.double().cpu().numpy()  # round to nearest even on the 16-bit conversion
    return lut, stored


def _check(out, ref, N, mask=None):
    R = out["R"].double().cpu().numpy()
    G = out["grad"].double().cpu().numpy()
    if mask is None:
        mask = np.ones(len(R), bool)
    maxR = np.abs(ref["R"]).max()
    maxG = max(np.linalg.norm(ref["grad"], axis=1).max(), 1e-30)
    tR = 1e-5 * maxR
    tG = 1e-4 * maxG + N * 2.0 ** -23 * maxR
    assert np.abs(R - ref["R"])[mask].max() <= tR
    assert np.abs(G - ref["grad"])[mask].max() <= tG
    Nn = out["normal"].double().cpu().numpy()
    mlen = np.sqrt(ref["R"] ** 2 + (ref["grad"] ** 2).sum(1))
    bound = 2.0 * (tR + tG) / mlen + 1e-6
    assert np.all((np.abs(Nn - ref["normal"]).max(1) <= bound)[mask])


@pytest.mark.parametrize("method", METHODS)
@pytest.mark.parametrize("dtype", [0, 1])
def test_single_glyph_parity(S, method, dtype):
    N, L = 12, 6
    c = I.sh_coeffs(1, L, 400)[0]
    g = O.value_grid_sh(N, L, c)
    lut, stored = upload_value_pool(S, [g], dtype=dtype)
    dirs = I.directions(50000, 401)
    out = S.query_recon(lut, method, torch.from_numpy(dirs).cuda(), want=("R", "grad", "normal", "chart", "fij"))
    pool, off, Ns = O.make_value_pool([stored.reshape(g.shape)])
    ref = O.recon(method, pool, off, Ns, dirs)
    ok = ~near_edge(ref["fij"], dirs, [N], None)
    if method == 0:
        # nearest: texel boundaries sit half a cell from the cell edges
        d = dirs.astype(np.float64)
        k = np.argmax(np.abs(d), 1)
        m = np.abs(d[np.arange(len(d)), k])
        for ax in (1, 2):
            fr = ((d[np.arange(len(d)), (k + ax) % 3] / m + 1) / 2 * N) % 1.0
            ok &= (fr > 1e-5) & (fr < 1 - 1e-5)
    assert np.array_equal(out["fij"].cpu().numpy()[ok], ref["fij"][ok])
    _check(out, ref, N, mask=ok if method == 0 else None)


@pytest.mark.parametrize("mode", ["glyph", "seg"])
def test_uneven_pool(S, mode):
    Ns = [4, 9, 16, 33, 5]
    grids = [O.value_grid_sh(n, 5, I.sh_coeffs(1, 5, 410 + k)[0]) for k, n in enumerate(Ns)]
    r0 = np.array([0.0, 0.5, -0.25, 1.0, 0.125], np.float32)
    lut, stored = upload_value_pool(S, grids, r0=r0)
    counts = np.array([100, 0, 3001, 517, 64])
    Q = int(counts.sum())
    dirs = I.directions(Q, 411)
    glyph = np.repeat(np.arange(5, dtype=np.int32), counts)
    pool, off, Nn = O.make_value_pool([stored[o:o + g.size].reshape(g.shape) for o, g in
                                       zip(np.cumsum([0] + [g.size for g in grids[:-1]]), grids)])
    for method in (1, 2, 3):
        if mode == "glyph":
            out = S.query_recon(lut, method, torch.from_numpy(dirs).cuda(), glyph=torch.from_numpy(glyph).cuda())
        else:
            seg = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
            out = S.query_recon(lut, method, torch.from_numpy(dirs).cuda(), seg=torch.from_numpy(seg).cuda())
        ref = O.recon(method, pool, off, Nn, dirs, glyph=glyph, r0=r0.astype(np.float64))
        _check(out, ref, max(Ns))


def test_sh_value_table_build(S):
    N, L, G = 16, 8, 40
    coeffs = I.sh_coeffs(G, L, 420).astype(np.float32)
    r0 = np.linspace(-0.5, 0.5, G).astype(np.float32)
    lut = S.alloc_lut(G, N, 0, S.SHM_LAYOUT_VALUE, r0=r0)
    S.build_lut(lut, S.Source(kind=S.SHM_SRC_SH, L=L, coeffs=torch.from_numpy(coeffs).cuda()))
    got = lut.data.double().cpu().numpy().reshape(G, 6, N + 4, N + 4)
    for g in (0, 17, G - 1):
        r = O.value_grid_sh(N, L, coeffs[g].astype(np.float64))
        # the bar of the direct SH evaluation (float32 Legendre recurrence): 1e-5 max|r|
        assert np.abs(got[g] - (r - r0[g])).max() <= 1e-5 * np.abs(r).max()


def test_fd_source_value_tables(S):
    """Sampled sources: the value table is the margin sample grid itself."""
    N = 20
    counts, offs, mu, amp, width = I.bump_params(3, 430)
    mu32, amp32, w32 = mu.astype(np.float32), amp.astype(np.float32), width.astype(np.float32)
    lut = S.alloc_lut(3, N, 0, S.SHM_LAYOUT_VALUE, r0=[1.0] * 3)
    S.build_lut(lut, S.Source(kind=S.SHM_SRC_BUMPS, bump_offset=torch.from_numpy(offs).cuda(),
                              mu=torch.from_numpy(mu32).cuda(), amp=torch.from_numpy(amp32).cuda(),
                              width=torch.from_numpy(w32).cuda()))
    got = lut.data.double().cpu().numpy().reshape(3, 6, N + 4, N + 4)
    for g in range(3):
        sl = slice(offs[g], offs[g + 1])
        ref = O.sample_grid_bumps(N, mu32[sl].astype(np.float64), amp32[sl].astype(np.float64),
                                  w32[sl].astype(np.float64)) - 1.0
        eps_S = 8 * 2.0 ** -24 * np.abs(amp32[sl]).sum()  # float32 evaluation of the bump sum
        assert np.abs(got[g] - ref).max() <= 2 * eps_S
    keys = I.fbm_keys(431)
    lut = S.alloc_lut(1, 64, 0, S.SHM_LAYOUT_VALUE, r0=[1.0])
    S.build_lut(lut, S.Source(kind=S.SHM_SRC_FBM, octaves=8, keys=torch.from_numpy(keys.view(np.int32)).cuda(),
                              base_freq=2.0, lacunarity=2.0, gain=0.5, amplitude=0.02))
    got = lut.data.double().cpu().numpy().reshape(6, 68, 68)
    ref = O.sample_grid_fbm(64, keys, 2.0, 2.0, 0.5, 0.02)
    assert np.abs(got - ref).max() <= 2 * 4e-8  # float32 direction and lattice rounding, amplitude 0.02


def test_invalid_combinations(S):
    g = O.value_grid_sh(8, 4, I.sh_coeffs(1, 4, 440)[0])
    vlut, _ = upload_value_pool(S, [g])
    d = torch.from_numpy(I.directions(10, 441)).cuda()
    with pytest.raises(S.ShmError):
        S.query(vlut, d)                       # the Hermite query needs derivative channels
    with pytest.raises(S.ShmError):
        S.query_recon(vlut, 7, d)              # unknown method
    herm = S.alloc_lut(1, 8)
    with pytest.raises(S.ShmError):
        S.query_recon(herm, 1, d)              # not a value table
    out = S.query_recon(vlut, 2, torch.empty((0, 3), device="cuda"))
    assert out["R"].numel() == 0
