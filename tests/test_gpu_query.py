"""GPU parity of shm_query against the FP64 oracle on identical stored table bytes.

Bar (spec tolerances): face and cell indices bit-exact away from ties within 1e-6 of an
edge; value max-abs error <= 1e-5 max|R|; gradient <= 1e-4 max|grad R|; normals within the bound
those two propagate to.  16-bit storage: the device quantisation must equal the oracle's
round-to-nearest-even bytes, and the query on those bytes meets the same bar.
"""
import numpy as np
import pytest
import torch

import oracle as O
import shm_inputs as I
from gpu_common import check_query, near_edge, shm, upload_pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return shm()


def _config1(seed=20063):
    """Single SH glyph: L=4, N=10, 65,536 uniform directions."""
    c = I.sh_coeffs(1, 4, seed)[0]
    lut = O.bake_sh(10, 4, c)
    dirs = I.directions(65536, seed + 100)
    return lut, dirs


@pytest.mark.parametrize("dtype,layout", [(0, 0), (0, 1), (1, 0), (2, 0), (1, 1), (2, 1)])
def test_single_glyph_parity(S, dtype, layout):
    lut, dirs = _config1()
    L, stored = upload_pool(S, [lut], dtype=dtype, layout=layout)
    d = torch.from_numpy(dirs).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = S.query(L, d, want=("R", "grad", "normal", "chart", "fij"), dev_status=st)
    torch.cuda.synchronize()
    ref = O.query(stored.reshape(-1, 4), [0], [10], dirs)
    assert st.item() == 0
    fij = out["fij"].cpu().numpy()
    ok = ~near_edge(ref["fij"], dirs, [10], None)
    assert ok.sum() > 0.999 * len(dirs)
    assert np.array_equal(fij[ok], ref["fij"][ok])
    check_query(out, ref)


def test_cell_layout_is_bit_identical_to_texel(S):
    lut, dirs = _config1(7)
    Lt, _ = upload_pool(S, [lut], dtype=0, layout=0)
    Lc, _ = upload_pool(S, [lut], dtype=0, layout=1)
    d = torch.from_numpy(dirs).cuda()
    a = S.query(Lt, d)
    b = S.query(Lc, d)
    for k in a:
        assert torch.equal(a[k], b[k]), k


@pytest.mark.parametrize("dtype", [1, 2])
def test_quantised_bytes_match_oracle(S, dtype):
    lut, _ = _config1(8)
    L, stored = upload_pool(S, [lut], dtype=dtype, layout=0)
    got = L.data.float().double().cpu().numpy()
    assert np.array_equal(got, stored)


def _uneven_pool(n, seed):
    Ns = I.uneven_N(n, seed, choices=(3, 5, 16, 33))
    luts = []
    for g in range(n):
        c = I.sh_coeffs(1, 6, seed + 1000 + g)[0]
        luts.append(O.bake_sh(int(Ns[g]), 6, c))
    return luts, Ns


@pytest.mark.parametrize("mode", ["glyph", "seg"])
def test_uneven_glyphs(S, mode):
    luts, Ns = _uneven_pool(12, 31)
    r0 = np.linspace(-0.5, 0.5, 12).astype(np.float32)
    L, stored = upload_pool(S, luts, r0=r0)
    # ragged: a total that is no multiple of the warp chunk, empty segments included
    counts = np.array([0, 1, 33, 257, 0, 500, 7, 1000, 2, 0, 64, 3001])
    Q = int(counts.sum())
    dirs = I.directions(Q, 32)
    glyph = np.repeat(np.arange(12, dtype=np.int32), counts)
    seg = np.zeros(13, dtype=np.int64)
    seg[1:] = np.cumsum(counts)
    d = torch.from_numpy(dirs).cuda()
    if mode == "glyph":
        perm = np.random.default_rng(3).permutation(Q)
        dirs, glyph = dirs[perm], glyph[perm]
        d = torch.from_numpy(dirs).cuda()
        out = S.query(L, d, glyph=torch.from_numpy(glyph).cuda(), want=("R", "grad", "normal", "fij"))
    else:
        out = S.query(L, d, seg=torch.from_numpy(seg).cuda(), want=("R", "grad", "normal", "fij"))
    off, Nn = O.make_pool(luts)[1:]
    ref = O.query(stored.reshape(-1, 4), off, Nn, dirs, glyph=glyph, r0=r0.astype(np.float64))
    ok = ~near_edge(ref["fij"], dirs, Nn, glyph)
    assert np.array_equal(out["fij"].cpu().numpy()[ok], ref["fij"][ok])
    check_query(out, ref)


def test_edge_cases(S):
    lut, _ = _config1(9)
    L, stored = upload_pool(S, [lut])
    # Q = 0
    out = S.query(L, torch.empty((0, 3), device="cuda"))
    assert out["R"].numel() == 0
    # zero / inf / nan directions -> NaN outputs and the NONFINITE bit; axis-aligned and tie directions
    special = np.array([[0, 0, 0], [np.inf, 0, 1], [np.nan, 1, 0], [1, 0, 0], [-1, 0, 0], [0, 0, -1],
                        [1, 1, 0], [-1, 1, 1], [0.5, -0.5, 0.5], [-0.0, 0.0, 2.0], [1e-30, 1e-30, 1e-30]],
                       dtype=np.float32)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = S.query(L, torch.from_numpy(special).cuda(), want=("R", "grad", "normal", "fij"), dev_status=st)
    R = out["R"].cpu().numpy()
    assert np.isnan(R[:3]).all() and np.isfinite(R[3:]).all()
    assert st.item() & S.SHM_DEV_NONFINITE
    ref = O.query(stored.reshape(-1, 4), [0], [10], special[3:])
    assert np.array_equal(out["fij"].cpu().numpy()[3:], ref["fij"])
    assert np.abs(R[3:] - ref["R"]).max() <= 1e-5 * np.abs(ref["R"]).max()
    # glyph index out of range -> BOUNDS bit, NaN
    st.zero_()
    bad = torch.tensor([0, 1, -1], dtype=torch.int32, device="cuda")
    out = S.query(L, torch.from_numpy(special[3:6]).cuda(), glyph=bad, dev_status=st)
    R = out["R"].cpu().numpy()
    assert np.isfinite(R[0]) and np.isnan(R[1]) and np.isnan(R[2])
    assert st.item() & S.SHM_DEV_BOUNDS


def test_invalid_arguments_return_status(S):
    lut, _ = _config1(10)
    L, _ = upload_pool(S, [lut])
    bad = S.alloc_lut(1, 10)
    bad.dtype = 7
    with pytest.raises(S.ShmError):
        S.query(bad, torch.zeros((4, 3), device="cuda"))
    with pytest.raises(S.ShmError):
        L2 = S.alloc_lut(1, 10)
        L2.N_uniform = 0  # per-glyph arrays missing
        S.query(L2, torch.zeros((4, 3), device="cuda"))


def test_large_N_precision(S):
    """Planet-scale resolution: the double-float cell coordinate keeps s, t exact at N = 2048."""
    N = 2048
    P = N + 2
    keys = I.fbm_keys(4)
    # a smooth closed-form table: r = x^2 - 0.5 y^3 in chart coordinates on every face, exact derivatives
    u = (np.arange(P) - 0.5) / N
    U, V = np.meshgrid(u, u, indexing="xy")
    X, Y = 2 * U - 1, 2 * V - 1
    rec = np.stack([0.01 * (X ** 2 - 0.5 * Y ** 3), 0.01 * 4 * X / N, 0.01 * (-3 * Y ** 2) / N,
                    np.zeros_like(X)], axis=-1)
    lut = np.broadcast_to(rec, (6, P, P, 4)).copy()
    L, stored = upload_pool(S, [lut], r0=np.array([1.0], np.float32))
    dirs = I.directions(200000, 5)
    d = torch.from_numpy(dirs).cuda()
    out = S.query(L, d, want=("R", "grad", "normal", "fij"))
    ref = O.query(stored.reshape(-1, 4), [0], [N], dirs, r0=np.array([1.0]))
    ok = ~near_edge(ref["fij"], dirs, [N], None)
    assert np.array_equal(out["fij"].cpu().numpy()[ok], ref["fij"][ok])
    check_query(out, ref)


@pytest.mark.parametrize("layout", [0, 1])
def test_vector_and_scalar_io_paths_agree(S, layout):
    """16-byte-aligned directions/outputs take 128-bit loads and stores for full warp rounds; a
    direction view offset by one row (12 B) forces the scalar path.  Results must be identical,
    including the ragged last round."""
    lut, _ = _config1(11)
    L, _ = upload_pool(S, [lut], layout=layout)
    base = torch.from_numpy(I.directions(10001, 12)).cuda()
    d_al = base[1:].clone()          # aligned copy
    d_un = base[1:]                  # offset view: 12-byte shift from a 256-byte-aligned allocation
    assert d_un.data_ptr() % 16 != 0 and d_al.data_ptr() % 16 == 0
    a = S.query(L, d_al, want=("R", "grad", "normal", "chart", "fij"))
    b = S.query(L, d_un, want=("R", "grad", "normal", "chart", "fij"))
    for k in a:
        assert torch.equal(a[k], b[k]), k


def _same(a, b):
    return bool(((a == b) | (torch.isnan(a) & torch.isnan(b))).all())


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_staged_segments_match_unstaged(S, dtype):
    """Per-glyph segments on a small uniform table take the shared-memory staged kernel; glyph ids
    on the same queries take the unstaged one.  Identical results, including queries outside every
    segment (NaN + SHM_DEV_BOUNDS), empty segments and ragged segment lengths."""
    G, N = 9, 20
    luts = [O.bake_sh(N, 6, I.sh_coeffs(1, 6, 500 + g)[0]) for g in range(G)]
    r0 = np.linspace(-0.3, 0.6, G).astype(np.float32)
    L, stored = upload_pool(S, luts, r0=r0, dtype=dtype)
    counts = np.array([1000, 0, 17, 4096, 513, 0, 1, 2047, 300])
    pre, post = 37, 11
    Q = pre + int(counts.sum()) + post
    dirs = I.directions(Q, 501)
    dirs[pre + 5] = 0.0                      # one invalid direction inside a segment
    seg = np.concatenate([[pre], pre + np.cumsum(counts)]).astype(np.int64)
    glyph = np.full(Q, -1, np.int32)
    for g in range(G):
        glyph[seg[g]:seg[g + 1]] = g
    d = torch.from_numpy(dirs).cuda()
    want = ("R", "grad", "normal", "chart", "fij")
    st1 = torch.zeros(1, dtype=torch.int32, device="cuda")
    st2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    a = S.query(L, d, seg=torch.from_numpy(seg).cuda(), want=want, dev_status=st1)
    b = S.query(L, d, glyph=torch.from_numpy(glyph).cuda(), want=want, dev_status=st2)
    for k in want:
        assert _same(a[k], b[k]), k
    assert st1.item() == st2.item() == (S.SHM_DEV_BOUNDS | S.SHM_DEV_NONFINITE)
    # and against the oracle on the covered queries
    off, Ns = O.make_pool(luts)[1:]
    cov = glyph >= 0
    cov[pre + 5] = False
    ref = O.query(stored.reshape(-1, 4), off, Ns, dirs[cov], glyph=glyph[cov], r0=r0.astype(np.float64))
    check_query({k: v[torch.from_numpy(cov).cuda()] for k, v in a.items() if k in ("R", "grad", "normal")}, ref)


def test_staged_glyph_field_size(S):
    """The glyph-field shape (N = 32, f32: 111 KB tables, two CTAs per SM), 512 glyphs."""
    G, N, per = 512, 32, 1024
    coeffs = I.sh_coeffs(G, 8, 510).astype(np.float32)
    lut = S.alloc_lut(G, N)
    S.build_lut(lut, S.Source(kind=S.SHM_SRC_SH, L=8, coeffs=torch.from_numpy(coeffs).cuda(), basis=S.sh_basis(N, 8)))
    dirs = torch.from_numpy(I.directions(G * per, 511)).cuda()
    seg = torch.from_numpy(I.query_glyphs_csr(G, per)).cuda()
    glyph = torch.from_numpy(np.repeat(np.arange(G, dtype=np.int32), per)).cuda()
    a = S.query(lut, dirs, seg=seg, want=("R", "grad", "normal", "fij"))
    b = S.query(lut, dirs, glyph=glyph, want=("R", "grad", "normal", "fij"))
    for k in a:
        assert torch.equal(a[k], b[k]), k
