"""Parity at the full sizes of the benchmark workloads, in the launch configurations bench.py times,
on sampled outputs the oracle computes one by one.

* Glyph field: 16,384 SH glyphs (L = 8, N = 32) baked by the tensor-core engine, 2^26 queries in
  per-glyph segments (the shared-memory staged query); sampled glyphs are re-baked by the oracle
  from the same float32 coefficients and their sampled queries evaluated there.  The device
  table carries the bake's float32 error (checked separately in test_gpu_build) on top of the
  query's, which the 1e-5 / 1e-4 bars absorb.
* Fit: 1,024 tables of N = 64, 2^24 queries (16,384 per glyph, segments), the fused
  loss + adjoint; the gradient slabs of sampled glyphs depend only on those glyphs' queries and
  targets, whose targets come from the oracle's direct SH evaluation (L = 16).
"""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.fit as OF
import shm_inputs as I
from gpu_common import check_query, near_edge, shm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return shm()


def test_glyph_field_full_size(S):
    G, L, N, per = 16384, 8, 32, 4096
    Q = G * per
    coeffs = I.sh_coeffs(G, L, 20063 + 1).astype(np.float32)
    lut = S.alloc_lut(G, N)
    src = S.Source(kind=S.SHM_SRC_SH, L=L, coeffs=torch.from_numpy(coeffs).cuda(), basis=S.sh_basis(N, L))
    S.build_lut(lut, src, ws=S.build_workspace(lut, src))
    dirs = np.empty((Q, 3), np.float32)
    for s0, d in I.directions_chunked(Q, 20063 + 1 + 7):
        dirs[s0:s0 + len(d)] = d
    seg = torch.from_numpy(I.query_glyphs_csr(G, per)).cuda()
    out = S.query(lut, torch.from_numpy(dirs).cuda(), seg=seg, want=("R", "grad", "normal"))
    rng = np.random.default_rng(11)
    glyphs = np.concatenate([[0, G - 1], rng.choice(G, 6, replace=False)])
    for g in glyphs:
        qs = g * per + rng.choice(per, 250, replace=False)
        ref_lut = O.bake_sh(N, L, coeffs[g].astype(np.float64))
        pool, off, Ns = O.make_pool([ref_lut])
        ref = O.query(pool, off, Ns, dirs[qs])
        idx = torch.from_numpy(qs).cuda()
        check_query({k: v[idx] for k, v in out.items()}, ref)


def test_fit_full_size(S):
    G, N, L, per = 1024, 64, 16, 16384
    Q = G * per
    coeffs = I.sh_coeffs(G, L, 20063 + 5).astype(np.float32)
    lut = S.alloc_lut(G, N, zero=True)
    lut.data.view(G, -1, 4)[:, :, 0] = torch.from_numpy(coeffs[:, 0] * 0.28209479177387814).cuda()[:, None]
    # one earlier Adam-like perturbation so that the derivative channels are not all zero
    rng = np.random.default_rng(12)
    lut.data.add_(torch.from_numpy((1e-3 * rng.standard_normal(lut.data.numel())).astype(np.float32)).cuda())
    dirs = I.directions(Q, 20063 + 5 + 100)
    seg = torch.from_numpy(I.query_glyphs_csr(G, per)).cuda()
    d = torch.from_numpy(dirs).cuda()
    Rt, _, nt = S.sh_eval(L, torch.from_numpy(coeffs).cuda(), d, seg=seg)
    glyphs = [0, 511, G - 1]
    ref_targets = {}
    for g in glyphs:
        sl = slice(g * per, (g + 1) * per)
        R_o, _, n_o = O.sh_eval(L, coeffs[g].astype(np.float64), dirs[sl])
        ref_targets[g] = (R_o.astype(np.float32), n_o.astype(np.float32))
        Rt[sl] = torch.from_numpy(ref_targets[g][0]).cuda()
        nt[sl] = torch.from_numpy(ref_targets[g][1]).cuda()
    dl = S.like_lut(lut, zero=True)
    loss = torch.zeros(1, device="cuda")
    S.fit_backward(lut, d, Rt, nt, dl, w_value=1.0, w_normal=1.0, loss=loss, seg=seg)
    table = lut.data.view(G, -1, 4)
    grads = dl.data.view(G, -1, 4)
    for g in glyphs:
        sl = slice(g * per, (g + 1) * per)
        glut = table[g].double().cpu().numpy().reshape(6, N + 2, N + 2, 4)
        pool, off, Ns = O.make_pool([glut])
        _, dref = OF.loss_and_grad(pool, off, Ns, dirs[sl], ref_targets[g][0].astype(np.float64),
                                   ref_targets[g][1].astype(np.float64), 1.0, 1.0)
        got = grads[g].double().cpu().numpy()
        for ch in range(4):
            assert np.abs(got[:, ch] - dref[:, ch]).max() <= 2e-5 * np.abs(dref[:, ch]).max(), (g, ch)
    assert torch.isfinite(loss).all() and loss.item() > 0


def test_glyph_field_backward_full_size(S):
    """Reverse pass of the glyph field at the bench size (16,384 tcgen05-baked tables, 2^26 queries
    in segments), atomic and deterministic: the gradient slabs of sampled glyphs against the
    oracle's adjoint of those glyphs' queries; the deterministic pass bit-identical over two runs.
    d/ddirs goes through the patch's second derivatives and two chart scalings (d/ds = N d/du, and
    s moves by N/2 per unit of the chart coordinate), so float32 rounding in the Hermite sums grows
    by about N^2: it is compared within 8 N^2 2^-24 of its largest magnitude (4.9e-4 at N = 32)."""
    G, L, N, per = 16384, 8, 32, 4096
    Q = G * per
    coeffs = I.sh_coeffs(G, L, 20063 + 1).astype(np.float32)
    lut = S.alloc_lut(G, N)
    src = S.Source(kind=S.SHM_SRC_SH, L=L, coeffs=torch.from_numpy(coeffs).cuda(), basis=S.sh_basis(N, L))
    S.build_lut(lut, src, ws=S.build_workspace(lut, src))
    dirs = np.empty((Q, 3), np.float32)
    for s0, d in I.directions_chunked(Q, 20063 + 1 + 7):
        dirs[s0:s0 + len(d)] = d
    rng = np.random.default_rng(13)
    up = rng.standard_normal((Q, 7), dtype=np.float32)
    seg = torch.from_numpy(I.query_glyphs_csr(G, per)).cuda()
    d = torch.from_numpy(dirs).cuda()
    u = torch.from_numpy(up).cuda()
    gR, gG, gN = u[:, 0].contiguous(), u[:, 1:4].contiguous(), u[:, 4:7].contiguous()
    res = {}
    for name, det in (("atomic", False), ("det1", True), ("det2", True)):
        dl = S.like_lut(lut, dtype=0, layout=0, zero=True)
        dd = S.query_backward(lut, d, dl, gR=gR, ggrad=gG, gnormal=gN, seg=seg, deterministic=det)
        res[name] = (dl.data.view(G, -1, 4), dd)
    assert torch.equal(res["det1"][0], res["det2"][0]) and torch.equal(res["det1"][1], res["det2"][1])
    table = lut.data.view(G, -1, 4)
    for g in (0, 7777, G - 1):
        sl = slice(g * per, (g + 1) * per)
        pool, off, Ns = O.make_pool([table[g].double().cpu().numpy().reshape(6, N + 2, N + 2, 4)])
        dref, ddref = O.query_vjp(pool, off, Ns, dirs[sl], gR=up[sl, 0], gG=up[sl, 1:4], gn=up[sl, 4:7])
        for name in ("atomic", "det1"):
            got = res[name][0][g].double().cpu().numpy()
            for ch in range(4):
                assert np.abs(got[:, ch] - dref[:, ch]).max() <= 2e-5 * np.abs(dref[:, ch]).max(), (name, g, ch)
            dd = res[name][1][sl].double().cpu().numpy()
            ok = ~near_edge(None, dirs[sl], [N], None, eps=1e-4)
            assert np.abs(dd[ok] - ddref[ok]).max() <= 8 * N * N * 2.0 ** -24 * np.abs(ddref[ok]).max(), (name, g)
