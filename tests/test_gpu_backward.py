"""GPU parity of the adjoint (shm_query_backward, shm_build_lut_backward) against the FP64 oracle.

Tolerances: dlut is a float32 atomic sum of per-query contributions, so each entry is compared
within 2e-5 of its channel's largest magnitude; ddirs involves the Hermite second derivatives
scaled by N^2 and is compared within 1e-4 of its largest magnitude, away from cell edges (the
patch is only C^1 there, so the one-sided second derivative depends on the chosen cell).
"""
import numpy as np
import pytest
import torch

import oracle as O
import shm_inputs as I
from gpu_common import near_edge, shm, upload_pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return shm()


def _case(seed, N=10, L=4, Q=8192, c00=2.0):
    c = I.sh_coeffs(1, L, seed)[0]
    c[0] += c00
    lut = O.bake_sh(N, L, c)
    dirs = I.directions(Q, seed + 1)
    rng = np.random.default_rng(seed)
    gR = rng.normal(size=Q).astype(np.float32)
    gG = rng.normal(size=(Q, 3)).astype(np.float32)
    gn = rng.normal(size=(Q, 3)).astype(np.float32)
    return lut, dirs, gR, gG, gn


@pytest.mark.parametrize("dtype,layout", [(0, 0), (0, 1), (2, 0)])
def test_query_backward_parity(S, dtype, layout):
    N = 10
    lut, dirs, gR, gG, gn = _case(40, N)
    r0 = np.array([0.3], np.float32)
    L, stored = upload_pool(S, [lut], r0=r0, dtype=dtype, layout=layout)
    dl = S.like_lut(L, dtype=0, layout=0, zero=True)
    t = lambda a: torch.from_numpy(a).cuda()
    ddirs = S.query_backward(L, t(dirs), dl, gR=t(gR), ggrad=t(gG), gnormal=t(gn))
    dref, ddref = O.query_vjp(stored.reshape(-1, 4), [0], [N], dirs, gR=gR, gG=gG, gn=gn, r0=r0.astype(np.float64))
    got = dl.data.view(-1, 4).double().cpu().numpy()
    for ch in range(4):
        scale = np.abs(dref[:, ch]).max()
        assert np.abs(got[:, ch] - dref[:, ch]).max() <= 2e-5 * scale, ch
    ok = ~near_edge(None, dirs, [N], None, eps=1e-4)
    dd = ddirs.double().cpu().numpy()
    scale = np.abs(ddref[ok]).max()
    assert np.abs(dd[ok] - ddref[ok]).max() <= 1e-4 * scale


def test_backward_accumulates_and_segments(S):
    luts = [O.bake_sh(n, 6, I.sh_coeffs(1, 6, 70 + n)[0] + np.eye(1, 49, 0)[0] * 2.0) for n in (4, 12, 31)]
    L, stored = upload_pool(S, luts)
    counts = np.array([100, 0, 3001])
    Q = int(counts.sum())
    dirs = I.directions(Q, 71)
    seg = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    glyph = np.repeat(np.arange(3), counts).astype(np.int32)
    rng = np.random.default_rng(72)
    gR = rng.normal(size=Q).astype(np.float32)
    t = lambda a: torch.from_numpy(a).cuda()
    dl = S.like_lut(L, zero=True)
    S.query_backward(L, t(dirs), dl, gR=t(gR), seg=t(seg), want_ddirs=False)
    S.query_backward(L, t(dirs), dl, gR=t(gR), seg=t(seg), want_ddirs=False)  # accumulates (+=)
    off, Ns = O.make_pool(luts)[1:]
    dref, _ = O.query_vjp(stored.reshape(-1, 4), off, Ns, dirs, gR=gR, glyph=glyph, want_ddirs=False)
    got = dl.data.view(-1, 4).double().cpu().numpy()
    assert np.abs(got - 2 * dref).max() <= 4e-5 * np.abs(2 * dref).max()


def test_dot_product_on_device(S):
    N = 12
    rng = np.random.default_rng(73)
    X = rng.normal(size=(6, N + 2, N + 2, 4))
    L, stored = upload_pool(S, [X])
    dirs = I.directions(20000, 74)
    y = rng.normal(size=20000).astype(np.float32)
    t = lambda a: torch.from_numpy(a).cuda()
    JX = S.query(L, t(dirs), want=("R",))["R"].double()
    dl = S.like_lut(L, zero=True)
    S.query_backward(L, t(dirs), dl, gR=t(y), want_ddirs=False)
    lhs = float((JX * t(y).double()).sum())
    rhs = float((L.data.double() * dl.data.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), 1.0)


@pytest.mark.parametrize("cuda_cores", [False, True])
@pytest.mark.parametrize("N,L,G", [(10, 4, 1), (32, 8, 40), (7, 2, 3), (33, 5, 129), (16, 16, 5)])
def test_build_backward(S, N, L, G, cuda_cores):
    """Adjoint of the bake on both engines vs the oracle's transpose of the linear bake, on sampled
    glyphs (the first six, the last): float32-grade bound 2e-5 of the largest entry.  Odd N (a table
    width not a multiple of the 16-scalar tensor-core chunk), glyph counts across the 128-glyph
    accumulator tiles, and L = 16 (K = 289: two MMAs per accumulator)."""
    rng = np.random.default_rng(N)
    T = 6 * (N + 2) ** 2
    dlut = rng.normal(size=(G, T * 4)).astype(np.float32)
    basis = S.sh_basis(N, L)
    D = S.alloc_lut(G, N)
    D.data.copy_(torch.from_numpy(dlut.ravel()))
    dc = S.build_lut_backward(D, L, basis, cuda_cores=cuda_cores).double().cpu().numpy()
    for g in sorted(set(list(range(min(G, 6))) + [G - 1])):
        ref = O.bake_sh_vjp(N, L, dlut[g].astype(np.float64).reshape(6, N + 2, N + 2, 4))
        assert np.abs(dc[g] - ref).max() <= 2e-5 * np.abs(ref).max(), g


def test_build_backward_engines_agree_at_the_glyph_field_size(S):
    """The glyph field's shape (16,384 glyphs, L = 8, N = 32): the tensor-core adjoint equals the
    CUDA-core one within float32 rounding of the 27,744-term sums, is bit-identical from run to run
    (fixed-order cluster reduction) with and without the deterministic flag, and matches the oracle
    on sampled glyphs."""
    N, L, G = 32, 8, 16384
    T = 6 * (N + 2) ** 2
    g = torch.Generator(device="cuda").manual_seed(9)
    D = S.alloc_lut(G, N)
    D.data.copy_(torch.randn(D.data.numel(), device="cuda", generator=g))
    basis = S.sh_basis(N, L)
    tc1 = S.build_lut_backward(D, L, basis)
    tc2 = S.build_lut_backward(D, L, basis, deterministic=True)
    simt = S.build_lut_backward(D, L, basis, cuda_cores=True, deterministic=True)
    torch.cuda.synchronize()
    assert torch.equal(tc1, tc2)
    scale = simt.abs().max()
    assert float((tc1 - simt).abs().max()) <= 2e-5 * float(scale)
    rows = [0, 1, 127, 128, 4095, 9999, G - 1]
    dl = D.data.view(G, T * 4)
    for r in rows:
        ref = O.bake_sh_vjp(N, L, dl[r].double().cpu().numpy().reshape(6, N + 2, N + 2, 4))
        assert np.abs(tc1[r].double().cpu().numpy() - ref).max() <= 2e-5 * np.abs(ref).max(), r


@pytest.mark.parametrize("dtype,N", [(0, 14), (1, 14), (0, 64), (1, 64)])
def test_segments_and_glyph_ids_agree_with_oracle(S, dtype, N):
    """The reverse pass with CSR segments and with glyph ids on the same queries, both against the
    oracle, accumulating into a non-zero dL/dtable, with queries outside every segment (NaN
    direction gradients, SHM_DEV_BOUNDS) and an empty segment.  N = 14 stages whole tables in the
    segment pass; N = 64 (418 KB tables) reads the footprints from global memory in both."""
    G = 7
    luts = [O.bake_sh(N, 5, I.sh_coeffs(1, 5, 600 + g)[0] + np.eye(1, 36, 0)[0] * 2.0) for g in range(G)]
    r0 = np.linspace(0.0, 0.4, G).astype(np.float32)
    L, stored = upload_pool(S, luts, r0=r0, dtype=dtype)
    counts = np.array([700, 0, 4096, 33, 1500, 2, 9000 if N == 64 else 999])
    pre, post = 5, 9
    Q = pre + int(counts.sum()) + post
    dirs = I.directions(Q, 601)
    seg = np.concatenate([[pre], pre + np.cumsum(counts)]).astype(np.int64)
    glyph = np.full(Q, -1, np.int32)
    for g in range(G):
        glyph[seg[g]:seg[g + 1]] = g
    rng = np.random.default_rng(602)
    gR = rng.normal(size=Q).astype(np.float32)
    gG = rng.normal(size=(Q, 3)).astype(np.float32)
    gn = rng.normal(size=(Q, 3)).astype(np.float32)
    t = lambda a: torch.from_numpy(a).cuda()
    init = torch.from_numpy(rng.normal(size=G * 6 * (N + 2) ** 2 * 4).astype(np.float32)).cuda()
    dl_s, dl_u = S.like_lut(L, dtype=0, layout=0), S.like_lut(L, dtype=0, layout=0)
    dl_s.data.copy_(init)
    dl_u.data.copy_(init)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    dd_s = S.query_backward(L, t(dirs), dl_s, gR=t(gR), ggrad=t(gG), gnormal=t(gn), seg=t(seg), dev_status=st)
    dd_u = S.query_backward(L, t(dirs), dl_u, gR=t(gR), ggrad=t(gG), gnormal=t(gn), glyph=t(glyph))
    assert st.item() & S.SHM_DEV_BOUNDS
    both_nan = torch.isnan(dd_s) & torch.isnan(dd_u)
    assert bool(((dd_s == dd_u) | both_nan).all())          # per-query, no accumulation order involved
    cov = glyph >= 0
    off, Ns = O.make_pool(luts)[1:]
    dref, _ = O.query_vjp(stored.reshape(-1, 4), off, Ns, dirs[cov], gR=gR[cov], gG=gG[cov], gn=gn[cov],
                          glyph=glyph[cov], r0=r0.astype(np.float64), want_ddirs=False)
    base = init.double().cpu().numpy().reshape(-1, 4)
    for dl in (dl_s, dl_u):
        got = dl.data.view(-1, 4).double().cpu().numpy() - base
        for ch in range(4):
            assert np.abs(got[:, ch] - dref[:, ch]).max() <= 2e-5 * np.abs(dref[:, ch]).max() + 4e-7 * np.abs(base[:, ch]).max(), ch


def _det_case(S, N, G, counts, dtype, layout, seed):
    luts = [O.bake_sh(N, 5, I.sh_coeffs(1, 5, seed + g)[0] + np.eye(1, 36, 0)[0] * 2.0) for g in range(G)]
    r0 = np.full(G, 0.25, np.float32)
    L, stored = upload_pool(S, luts, r0=r0, dtype=dtype, layout=layout)
    Q = int(np.sum(counts))
    dirs = I.directions(Q, seed + 100)
    seg = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    rng = np.random.default_rng(seed + 101)
    g = (rng.normal(size=Q).astype(np.float32), rng.normal(size=(Q, 3)).astype(np.float32),
         rng.normal(size=(Q, 3)).astype(np.float32))
    return luts, L, stored, r0, dirs, seg, g



@pytest.mark.parametrize("N,dtype,layout", [(32, 0, 0), (12, 2, 0), (64, 0, 0), (20, 0, 1)])
def test_deterministic_backward(S, N, dtype, layout):
    """SHM_BWD_DETERMINISTIC: bit-identical dlut over repeated runs, the oracle's adjoint within the
    atomic pass's tolerance, the same d/ddirs as the atomic pass.  N = 32 f32 and N = 12 bf16 texel
    tables take the staged kernel, N = 64 (418 KB) and the cell layout read the footprint from
    global memory; segments are ragged (0, 1, 1023, 1024, 1025 and 2500 queries)."""
    counts = np.array([1025, 0, 2500, 1, 1024, 1023])
    luts, L, stored, r0, dirs, seg, (gR, gG, gn) = _det_case(S, N, len(counts), counts, dtype, layout, 300 + N)
    t = lambda a: torch.from_numpy(a).cuda()
    outs = []
    for _ in range(2):
        dl = S.like_lut(L, dtype=0, layout=0, zero=True)
        dd = S.query_backward(L, t(dirs), dl, gR=t(gR), ggrad=t(gG), gnormal=t(gn), seg=t(seg), deterministic=True)
        outs.append((dl.data.clone(), dd))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    dla = S.like_lut(L, dtype=0, layout=0, zero=True)
    dda = S.query_backward(L, t(dirs), dla, gR=t(gR), ggrad=t(gG), gnormal=t(gn), seg=t(seg))
    assert torch.allclose(outs[0][1], dda, rtol=0, atol=1e-6 * float(dda.abs().max()))
    off, Ns = O.make_pool(luts)[1:]
    glyph = np.repeat(np.arange(len(counts)), counts).astype(np.int32)
    dref, _ = O.query_vjp(stored.reshape(-1, 4), off, Ns, dirs, gR=gR, gG=gG, gn=gn, glyph=glyph,
                          r0=r0.astype(np.float64), want_ddirs=False)
    got = outs[0][0].view(-1, 4).double().cpu().numpy()
    for ch in range(4):
        scale = np.abs(dref[:, ch]).max()
        assert np.abs(got[:, ch] - dref[:, ch]).max() <= 2e-5 * scale, ch


def test_deterministic_backward_one_cell(S):
    """Every query of a glyph in the same cell (one long run after the sort): the run's sum in
    query order equals the oracle's."""
    N = 16
    luts, L, stored, r0, _, _, _ = _det_case(S, N, 2, [1, 1], 0, 0, 77)
    Q = 3000
    dirs = np.tile(np.array([[0.31, -0.22, 0.93]], np.float32), (Q, 1))
    seg = np.array([0, Q, Q], np.int64)
    rng = np.random.default_rng(78)
    gR = rng.normal(size=Q).astype(np.float32)
    t = lambda a: torch.from_numpy(a).cuda()
    dl = S.like_lut(L, dtype=0, layout=0, zero=True)
    S.query_backward(L, t(dirs), dl, gR=t(gR), seg=t(seg), deterministic=True, want_ddirs=False)
    off, Ns = O.make_pool(luts)[1:]
    dref, _ = O.query_vjp(stored.reshape(-1, 4), off, Ns, dirs, gR=gR, glyph=np.zeros(Q, np.int32),
                          r0=r0.astype(np.float64), want_ddirs=False)
    got = dl.data.view(-1, 4).double().cpu().numpy()
    assert np.abs(got - dref).max() <= 2e-5 * np.abs(dref).max()


def test_deterministic_needs_segments(S):
    L, _ = upload_pool(S, [O.bake_sh(8, 2, I.sh_coeffs(1, 2, 5)[0])])
    d = torch.from_numpy(I.directions(100, 6)).cuda()
    dl = S.like_lut(L, dtype=0, layout=0, zero=True)
    with pytest.raises(S.ShmError):
        S.query_backward(L, d, dl, gR=torch.ones(100, device="cuda"), glyph=torch.zeros(100, dtype=torch.int32,
                                                                                        device="cuda"),
                         deterministic=True)
    bad = S.alloc_lut(1, 9)  # resolution differs from the table's
    with pytest.raises(S.ShmError):
        S.query_backward(L, d, bad, gR=torch.ones(100, device="cuda"))
