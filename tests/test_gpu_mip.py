"""GPU parity of shm_build_mip (derivative-consistent mip level, §4.7) against the FP64 oracle on
identical stored fine-table bytes.

Tolerance: every channel within 2e-6 * max|stored fine value| (+ |r0 shift|): the kernel sums four
float32 Hermite values (relative error ~1e-7 of the table's scale) and differences neighbouring
sums, which adds no amplification (the derivative records are h-scaled differences, not divided
by h)."""
import numpy as np
import pytest
import torch

import oracle as O
import shm_inputs as I
from gpu_common import shm, upload_pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return shm()


def _glyph_tables(Ns, L, seed):
    return [O.bake_sh(int(n), L, I.sh_coeffs(1, L, seed + g)[0]) for g, n in enumerate(Ns)]


def _coarse_host(S, lut):
    return lut.data.double().cpu().numpy() if lut.dtype == 0 and lut.layout == 0 else None


def _compare(got, ref, scale):
    for ch in range(4):
        e = np.abs(got[..., ch] - ref[..., ch]).max()
        assert e <= 2e-6 * scale, (ch, e, scale)


def test_uniform_pool_with_r0_shift(S):
    Nf, L = 32, 8
    luts = _glyph_tables([Nf] * 3, L, 300)
    r0f = np.array([0.3, -0.2, 0.0], np.float32)
    r0c = np.array([0.1, 0.1, -0.4], np.float32)
    fine, stored = upload_pool(S, luts, r0=r0f)
    coarse = S.mip_like(fine, r0=r0c)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.build_mip(fine, coarse, dev_status=st)
    assert st.item() == 0
    got = coarse.data.double().cpu().numpy().reshape(3, 6, Nf // 2 + 2, Nf // 2 + 2, 4)
    T = 6 * (Nf + 2) ** 2 * 4
    for g in range(3):
        f64 = stored[g * T:(g + 1) * T].reshape(6, Nf + 2, Nf + 2, 4)
        ref = O.mip_consistent(f64, r0=float(r0f[g]), r0_coarse=float(r0c[g]))
        _compare(got[g], ref, np.abs(f64[..., 0] + r0f[g]).max())


@pytest.mark.parametrize("dtype,layout", [(1, 0), (2, 1), (0, 1)])
def test_any_input_encoding(S, dtype, layout):
    Nf, L = 20, 6
    luts = _glyph_tables([Nf] * 2, L, 310)
    fine, stored = upload_pool(S, luts, dtype=dtype, layout=layout)
    coarse = S.mip_like(fine, dtype=0, layout=0)
    S.build_mip(fine, coarse)
    got = coarse.data.double().cpu().numpy().reshape(2, 6, Nf // 2 + 2, Nf // 2 + 2, 4)
    # the oracle works on the texel layout of the same stored values
    f32_texel, stored_t = upload_pool(S, luts)
    if dtype == 1:
        stored_t = O.quantize_f16(stored_t.astype(np.float32))
    elif dtype == 2:
        stored_t = O.quantize_bf16(stored_t.astype(np.float32))
    T = 6 * (Nf + 2) ** 2 * 4
    for g in range(2):
        f64 = stored_t[g * T:(g + 1) * T].reshape(6, Nf + 2, Nf + 2, 4)
        _compare(got[g], O.mip_consistent(f64), np.abs(f64[..., 0]).max())


def test_output_encoding_matches_pack(S):
    """Storing the coarse level as f16 cells equals packing the f32 texel result: same rounding."""
    luts = _glyph_tables([16, 8, 34], 6, 320)
    fine, _ = upload_pool(S, luts)
    c32 = S.build_mip(fine, S.mip_like(fine))
    c16 = S.build_mip(fine, S.mip_like(fine, dtype=1, layout=1))
    packed = S.like_lut(c32, dtype=1, layout=1)
    S.pack_lut(c32, packed)
    assert torch.equal(c16.data.view(torch.int16), packed.data.view(torch.int16))


def test_uneven_chain_down_to_N1(S):
    Ns = [16, 4, 36, 8, 12]
    luts = _glyph_tables(Ns, 6, 330)
    fine, stored = upload_pool(S, luts)
    ref = [l.astype(np.float32).astype(np.float64) for l in luts]
    cur = fine
    for lvl in range(4):
        if any(n % 2 for n in (cur.N.tolist())):
            break
        nxt = S.build_mip(cur, S.mip_like(cur))
        host = nxt.data.double().cpu().numpy()
        offs = nxt.offset.tolist()
        ref = [O.mip_consistent(r) for r in ref]
        for g, r in enumerate(ref):
            n = r.shape[1] - 2
            got = host[offs[g] * 4:offs[g] * 4 + r.size].reshape(r.shape)
            _compare(got, r, np.abs(r[..., 0]).max())
        # the oracle continues from the device's float32 records, like the device chain
        ref = [host[offs[g] * 4:offs[g] * 4 + r.size].reshape(r.shape) for g, r in enumerate(ref)]
        cur = nxt
    assert lvl >= 1


def test_unpaired_resolutions(S):
    luts = _glyph_tables([8, 6], 4, 340)
    fine, _ = upload_pool(S, luts)
    bad = S.alloc_lut(2, [4, 4])          # glyph 1: 6 / 2 = 3, not 4
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.build_mip(fine, bad, dev_status=st)
    host = bad.data.view(2 * 6 * 36, 4).cpu().numpy()
    assert np.isfinite(host[:6 * 36]).all() and np.isnan(host[6 * 36:]).all()
    assert st.item() & S.SHM_DEV_BOUNDS
    with pytest.raises(S.ShmError):
        odd = S.alloc_lut(1, 7)
        S.build_mip(odd, S.alloc_lut(1, 3))
    with pytest.raises(S.ShmError):
        S.build_mip(fine, fine)


def test_many_uneven_glyphs_span_several_launch_chunks(S):
    """4,500 glyphs with per-glyph N: the exact per-glyph block grids are split over several launches
    (at most 2,000 glyphs each); mip, pack and bounds are checked on glyphs around every split."""
    G = 4500
    Ns = I.uneven_N(G, 350, choices=(2, 4, 6, 10))
    luts = [O.bake_sh(int(n), 2, I.sh_coeffs(1, 2, 351 + g)[0]) for g, n in enumerate(Ns)]
    fine, stored = upload_pool(S, luts)
    coarse = S.build_mip(fine, S.mip_like(fine))
    packed = S.like_lut(coarse, dtype=1, layout=1)
    S.pack_lut(coarse, packed)
    rmax = S.lut_bounds(fine).cpu().numpy()
    host = coarse.data.double().cpu().numpy()
    hp = packed.data.float().double().cpu().numpy()
    offs_f, offs_c, offs_p = fine.offset.tolist(), coarse.offset.tolist(), packed.offset.tolist()
    for g in (0, 1, 1998, 1999, 2000, 2001, 3999, 4000, 4001, G - 1):
        n = int(Ns[g])
        f64 = stored[offs_f[g] * 4:offs_f[g] * 4 + 6 * (n + 2) ** 2 * 4].reshape(6, n + 2, n + 2, 4)
        ref = O.mip_consistent(f64)
        got = host[offs_c[g] * 4:offs_c[g] * 4 + ref.size].reshape(ref.shape)
        _compare(got, ref, np.abs(f64[..., 0]).max())
        # f16 cell pool: corner 0 of cell (i, j) is texel (i, j)
        nc = n // 2
        cells = hp[offs_p[g] * 16:offs_p[g] * 16 + 6 * (nc + 1) ** 2 * 16].reshape(6, nc + 1, nc + 1, 4, 4)
        want = O.quantize_f16(got[:, :nc + 1, :nc + 1].astype(np.float32))
        assert np.array_equal(cells[:, :, :, 0, :], want), g
        assert abs(rmax[g] - O.lut_bound(f64, n)) <= 1e-6 * O.lut_bound(f64, n), g


def test_planet_full_resolution(S):
    """The N = 2048 fBm planet table (403 MB) to N = 1024, every record against the oracle."""
    N = 2048
    keys = I.fbm_keys(20063 + 3)
    fine = S.alloc_lut(1, N, r0=[1.0])
    S.build_lut(fine, S.Source(kind=S.SHM_SRC_FBM, octaves=8, keys=torch.from_numpy(keys.view(np.int32)).cuda(),
                               base_freq=2.0, lacunarity=2.0, gain=0.5, amplitude=0.02))
    coarse = S.build_mip(fine, S.mip_like(fine))
    f64 = fine.data.double().cpu().numpy().reshape(6, N + 2, N + 2, 4)
    ref = O.mip_consistent(f64, r0=1.0)
    got = coarse.data.double().cpu().numpy().reshape(ref.shape)
    _compare(got, ref, np.abs(f64[..., 0]).max())
