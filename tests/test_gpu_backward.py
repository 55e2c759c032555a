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
    tiles and cluster splits, and L = 16 (K = 289, beyond the tensor-core engine: CUDA cores)."""
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
    """The glyph field's shape (16,384 glyphs, L = 8, N = 32; 27,744-term sums): against the same
    contraction evaluated in float64 (the definition, a float64 matmul of dL/dtable by the float32
    basis) on every entry, the tensor-core adjoint is at least as accurate as the float32 CUDA-core
    contraction (within a factor of two) and within 1e-4 of the largest entry; it is bit-identical
    from run to run (fixed-order cluster reduction) with and without the deterministic flag; and it
    matches the oracle's transpose of the bake on sampled glyphs (2e-5 of the glyph's largest)."""
    N, L, G = 32, 8, 16384
    T = 6 * (N + 2) ** 2
    K = (L + 1) ** 2
    g = torch.Generator(device="cuda").manual_seed(9)
    D = S.alloc_lut(G, N)
    D.data.copy_(torch.randn(D.data.numel(), device="cuda", generator=g))
    basis = S.sh_basis(N, L)
    tc1 = S.build_lut_backward(D, L, basis)
    tc2 = S.build_lut_backward(D, L, basis, deterministic=True)
    simt = S.build_lut_backward(D, L, basis, cuda_cores=True, deterministic=True)
    torch.cuda.synchronize()
    assert torch.equal(tc1, tc2)
    dl = D.data.view(G, T * 4)
    full = basis[:K * T * 4].view(K, T * 4)
    ref = (dl.double() @ full.double().T)
    e_tc = float((tc1.double() - ref).abs().max())
    e_simt = float((simt.double() - ref).abs().max())
    scale = float(ref.abs().max())
    print(f"bake adjoint vs float64: tensor cores {e_tc / scale:.2e}, CUDA cores {e_simt / scale:.2e} of max")
    assert e_tc <= 2.0 * e_simt and e_tc <= 1e-4 * scale
    for r in [0, 1, 127, 128, 4095, 9999, G - 1]:
        oref = O.bake_sh_vjp(N, L, dl[r].double().cpu().numpy().reshape(6, N + 2, N + 2, 4))
        assert np.abs(tc1[r].double().cpu().numpy() - oref).max() <= 2e-5 * np.abs(oref).max(), r


@pytest.mark.parametrize("per_sm", [63.9, 64, 100.5, 128, 131])
def test_build_backward_glyph_group_sizing(S, per_sm):
    """The tensor-core adjoint sizes its glyph groups from the SM count: below 64 glyphs per SM,
    128-row groups with the texel sum split over cluster CTAs; from 64 per SM, groups of 64-128 rows
    that fill whole waves of the SMs (the last group ragged), one wave up to 128 per SM and two above.
    Every glyph against the float64 contraction of the same float32 operands (2e-5 of the largest
    entry), and glyphs at group boundaries against the oracle's transpose of the bake."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    N, L = 7, 4
    G = int(per_sm * sms)
    T = 6 * (N + 2) ** 2
    K = (L + 1) ** 2
    g = torch.Generator(device="cuda").manual_seed(int(per_sm * 10))
    D = S.alloc_lut(G, N)
    D.data.copy_(torch.randn(D.data.numel(), device="cuda", generator=g))
    basis = S.sh_basis(N, L)
    dc = S.build_lut_backward(D, L, basis)
    dl = D.data.view(G, T * 4)
    ref = dl.double() @ basis[:K * T * 4].view(K, T * 4).double().T
    assert float((dc.double() - ref).abs().max()) <= 2e-5 * float(ref.abs().max())
    waves = -(-G // (128 * sms))
    R = 128 if G < 64 * sms else -(-G // (waves * sms))
    dcn = dc.double().cpu().numpy()
    for r in sorted({0, R - 1, R, 2 * R - 1, G // 2, G - R, G - 1} & set(range(G))):
        oref = O.bake_sh_vjp(N, L, dl[r].double().cpu().numpy().reshape(6, N + 2, N + 2, 4))
        assert np.abs(dcn[r] - oref).max() <= 2e-5 * np.abs(oref).max(), r
