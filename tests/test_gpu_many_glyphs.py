"""More glyphs than one grid dimension holds (65,535): the launch helpers split the glyph range.
70,000 tiny glyphs, uniform and per-glyph resolutions, through the FD bake, pack, bounds, mip level
and query, spot-checked against the oracle on glyphs on both sides of every split."""
import numpy as np
import pytest
import torch

import oracle as O
import shm_inputs as I
from gpu_common import shm

pytestmark = pytest.mark.gpu

G = 70000
CHECK = [0, 1, 65534, 65535, 65536, G - 1]


@pytest.fixture(scope="module")
def S():
    return shm()


def _bump_tables(S, Ns):
    counts, offs, mu, amp, width = I.bump_params(G, 800, count_range=(1, 3))
    mu32, amp32, w32 = mu.astype(np.float32), amp.astype(np.float32), width.astype(np.float32)
    lut = S.alloc_lut(G, Ns, r0=[1.0] * G)
    S.build_lut(lut, S.Source(kind=S.SHM_SRC_BUMPS, bump_offset=torch.from_numpy(offs).cuda(),
                              mu=torch.from_numpy(mu32).cuda(), amp=torch.from_numpy(amp32).cuda(),
                              width=torch.from_numpy(w32).cuda()))
    return lut, offs, mu32, amp32, w32


@pytest.mark.parametrize("uniform", [True, False])
def test_many_glyphs(S, uniform):
    Ns = 4 if uniform else [int(n) for n in I.uneven_N(G, 801, choices=(2, 4, 6))]
    lut, offs, mu, amp, width = _bump_tables(S, Ns)
    host = lut.data.double().cpu().numpy()
    rb = 4  # floats per record
    offsets = (np.arange(G) * 6 * 36) if uniform else lut.offset.cpu().numpy()
    Nof = (lambda g: 4) if uniform else (lambda g: Ns[g])
    rmax = S.lut_bounds(lut).cpu().numpy()
    f16 = S.like_lut(lut, dtype=1)
    S.pack_lut(lut, f16)
    h16 = f16.data.float().double().cpu().numpy()
    coarse = S.build_mip(lut, S.mip_like(lut))
    hc = coarse.data.double().cpu().numpy()
    coffs = (np.arange(G) * 6 * 16) if uniform else coarse.offset.cpu().numpy()
    for g in CHECK:
        n = Nof(g)
        sl = slice(offs[g], offs[g + 1])
        ref = O.bake_fd(n, O.sample_grid_bumps(n, mu[sl].astype(np.float64), amp[sl].astype(np.float64),
                                               width[sl].astype(np.float64)), r0=1.0)
        got = host[offsets[g] * rb:offsets[g] * rb + ref.size].reshape(ref.shape)
        assert np.abs(got - ref).max() <= 1e-6, g
        assert np.array_equal(h16[offsets[g] * rb:offsets[g] * rb + ref.size],
                              O.quantize_f16(got.astype(np.float32)).ravel()), g
        assert abs(rmax[g] - O.lut_bound(got, n, 1.0)) <= 1e-6 * rmax[g], g
        cref = O.mip_consistent(got, r0=1.0)
        cgot = hc[coffs[g] * rb:coffs[g] * rb + cref.size].reshape(cref.shape)
        assert np.abs(cgot - cref).max() <= 2e-6, g
    # queries on the checked glyphs, by glyph id
    dirs = I.directions(len(CHECK) * 100, 802)
    glyph = np.repeat(np.array(CHECK, np.int32), 100)
    out = S.query(lut, torch.from_numpy(dirs).cuda(), glyph=torch.from_numpy(glyph).cuda())
    pool = host.reshape(-1, 4)
    Nn = np.array([Nof(g) for g in range(G)], np.int32) if not uniform else np.full(G, 4, np.int32)
    ref = O.query(pool, np.asarray(offsets, np.int64), Nn, dirs, glyph=glyph, r0=np.ones(G))
    assert np.abs(out["R"].double().cpu().numpy() - ref["R"]).max() <= 1e-5 * np.abs(ref["R"]).max()
