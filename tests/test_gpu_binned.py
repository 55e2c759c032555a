"""GPU parity of shm_query_binned (the region-partitioned query of one large table) against the FP64
oracle, and its equality with shm_query on the same inputs.

The partition only reorders work: every output must equal shm_query's bit for bit, in query order,
for any band size (one band per face up to one cell row per band), any batch length (empty, one
query, ragged tails of the 16,384-query tiles and of the 2,048-query rounds) and any record dtype
and layout.  Against the oracle the bar is the spec one: value <= 1e-5 max|R|, gradient
<= 1e-4 max|grad R|, normals within the bound those propagate to.  At the full planet size
(N = 2048, 2^28 uniform random directions, the benchmark's launch) the outputs equal shm_query's
and sampled queries match the oracle evaluated from the procedural source.
"""
import numpy as np
import pytest
import torch

import oracle as O
import shm_inputs as I
from gpu_common import check_query, shm, upload_pool

pytestmark = pytest.mark.gpu

WANT = ("R", "grad", "normal", "chart")


@pytest.fixture(scope="module")
def S():
    return shm()


def _glyph(seed=20063, N=10, L=4):
    c = I.sh_coeffs(1, L, seed)[0]
    return O.bake_sh(N, L, c)


def _binned(S, L, d, band_bytes=0, dev_status=None):
    ws = S.query_binned_workspace(L, d.shape[0], band_bytes)
    return S.query_binned(L, d, ws, band_bytes=band_bytes, want=WANT, dev_status=dev_status)


def _equal(a, b):
    """Bit-identical outputs (NaN payloads included)."""
    for k in WANT:
        assert torch.equal(a[k].view(torch.int32), b[k].view(torch.int32)), k


@pytest.mark.parametrize("band_bytes", [0, 1, 2000, 10 ** 9])
def test_binned_parity_single_glyph(S, band_bytes):
    lut = _glyph()
    L, stored = upload_pool(S, [lut])
    dirs = I.directions(65536 + 777, 20063 + 100)
    d = torch.from_numpy(dirs).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = _binned(S, L, d, band_bytes, st)
    ref_dev = S.query(L, d, want=WANT)
    torch.cuda.synchronize()
    assert st.item() == 0
    info = S.query_binned_bins(L, band_bytes)
    assert 6 <= info["bins"] <= 252 and info["bins"] % 6 == 0
    _equal(out, ref_dev)
    ref = O.query(stored.reshape(-1, 4), [0], [10], dirs)
    check_query(out, ref)


@pytest.mark.parametrize("Q", [0, 1, 31, 2047, 2049, 16384, 16385, 3 * 16384 + 4097])
def test_binned_ragged_lengths(S, Q):
    lut = _glyph(7, N=24, L=6)
    L, _ = upload_pool(S, [lut])
    d = torch.from_numpy(I.directions(Q, 20063 + 5)).cuda().reshape(Q, 3)
    out = _binned(S, L, d, band_bytes=4000)
    if Q == 0:
        return
    _equal(out, S.query(L, d, want=WANT))


@pytest.mark.parametrize("dtype,layout", [(0, 1), (1, 0), (2, 1)])
def test_binned_dtypes_layouts(S, dtype, layout):
    lut = _glyph(11, N=32, L=8)
    L, stored = upload_pool(S, [lut], dtype=dtype, layout=layout)
    dirs = I.directions(100000, 20063 + 6)
    d = torch.from_numpy(dirs).cuda()
    out = _binned(S, L, d, band_bytes=3000)
    _equal(out, S.query(L, d, want=WANT))
    ref = O.query(stored.reshape(-1, 4), [0], [32], dirs)
    check_query(out, ref)


def test_binned_edge_directions(S):
    """Axis directions, exact face ties, -0, zero and non-finite directions, unnormalised lengths."""
    lut = _glyph(13, N=16, L=4)
    L, _ = upload_pool(S, [lut])
    special = [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1], [1, 1, 0], [1, -1, 1],
               [-0.0, 0, 1], [0, -0.0, -1], [3, 3, 3], [1e-20, 0, 0], [0, 0, 0], [np.nan, 0, 1], [np.inf, 0, 0],
               [5e3, -2e3, 1e3]]
    rnd = I.directions(5000, 20063 + 8) * np.float32(2.5)
    dirs = np.concatenate([np.asarray(special, dtype=np.float32), rnd]).astype(np.float32)
    d = torch.from_numpy(dirs).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = _binned(S, L, d, band_bytes=500, dev_status=st)
    ref = S.query(L, d, want=WANT)
    torch.cuda.synchronize()
    assert st.item() & S.SHM_DEV_NONFINITE
    _equal(out, ref)
    bad = ~np.isfinite(dirs).all(1) | (np.abs(dirs).max(1) == 0)
    assert torch.isnan(out["R"][torch.from_numpy(bad).cuda()]).all()


def test_binned_rejects(S):
    lut = _glyph(17, N=8, L=2)
    L, _ = upload_pool(S, [lut])
    d = torch.from_numpy(I.directions(1000, 3)).cuda()
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(S.ShmError, match="workspace"):
        S.query_binned(L, d, small)
    ws = S.query_binned_workspace(L, 1000)
    with pytest.raises(S.ShmError, match="invalid"):
        S.query_binned(L, d, ws, band_bytes=-1)
    uneven = S.alloc_lut(2, [8, 4])
    with pytest.raises(S.ShmError):
        S.query_binned_workspace(uneven, 1000)


def test_binned_repeat_is_identical(S):
    """The workspace keeps nothing between calls: a second call (stale workspace) gives the same bytes."""
    lut = _glyph(19, N=40, L=6)
    L, _ = upload_pool(S, [lut])
    d = torch.from_numpy(I.directions(200000, 20063 + 9)).cuda()
    ws = S.query_binned_workspace(L, d.shape[0], 6000)
    a = S.query_binned(L, d, ws, band_bytes=6000, want=WANT)
    ws.fill_(0xA5)
    b = S.query_binned(L, d, ws, band_bytes=6000, want=WANT)
    _equal(a, b)


def test_binned_planet_full_size(S):
    """The benchmark's launch: N = 2048 fBm planet, 2^28 uniform random directions, default bands."""
    from test_gpu_planet import _oracle_query_from_source
    N, Q = 2048, 1 << 28
    keys = I.fbm_keys(20063 + 3)
    lut = S.alloc_lut(1, N, r0=[1.0])
    S.build_lut(lut, S.Source(kind=S.SHM_SRC_FBM, octaves=8, keys=torch.from_numpy(keys.view(np.int32)).cuda(),
                              base_freq=2.0, lacunarity=2.0, gain=0.5, amplitude=0.02))
    d = torch.empty((Q, 3), dtype=torch.float32, device="cuda")
    for s0, c in I.directions_chunked(Q, 20063 + 3 + 11):
        d[s0:s0 + len(c)].copy_(torch.from_numpy(c))
    ws = S.query_binned_workspace(lut, Q)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = S.query_binned(lut, d, ws, dev_status=st)
    del ws
    ref = S.query(lut, d)
    torch.cuda.synchronize()
    assert st.item() == 0
    for k in ("R", "grad", "normal"):
        assert torch.equal(out[k].view(torch.int32), ref[k].view(torch.int32)), k
    del ref
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(Q, 600, replace=False))
    dirs_s = d[torch.from_numpy(idx).cuda()].cpu().numpy()
    R = out["R"][torch.from_numpy(idx).cuda()].double().cpu().numpy()
    G = out["grad"][torch.from_numpy(idx).cuda()].double().cpu().numpy()
    refs = [_oracle_query_from_source(keys, dirs_s[k].astype(np.float64)) for k in range(len(idx))]
    Rr = np.array([r[0] for r in refs])
    Gr = np.array([r[1] for r in refs])
    maxG = np.linalg.norm(Gr, axis=1).max()
    assert np.abs(R - Rr).max() <= 1e-5 * np.abs(Rr).max()
    assert np.abs(G - Gr).max() <= 1e-4 * maxG + 3 * N * 2e-8
