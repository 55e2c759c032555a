"""GPU parity of the staged reverse pass (per-glyph query segments on uniform tables small enough for
shared memory: each glyph's table staged whole, its queries answered from it) against the FP64
oracle.

The cases walk the segment loop through its edges: empty segments between non-empty ones, segments
of 1, 511, 512, 513 and several blocks of queries, queries outside every segment (NaN d/ddirs and
SHM_DEV_BOUNDS), more glyphs than CTAs, each subset of upstream gradients, 16-bit tables and the
fused fit loss; and, on the unstaged pass, lane pairs whose paired gradient reductions straddle
two glyphs of different N.  Tolerances as in the other adjoint tests: dlut within 2e-5 of each
channel's largest magnitude, d/ddirs within 1e-4 of its largest magnitude away from cell edges.
"""
import numpy as np
import pytest
import torch

import oracle as O
import oracle.fit as OF
import shm_inputs as I
from gpu_common import near_edge, shm, upload_pool

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return shm()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _pool(G, N, L, seed):
    return [O.bake_sh(N, L, I.sh_coeffs(1, L, seed + g)[0] + np.eye(1, (L + 1) ** 2, 0)[0] * 2.0) for g in range(G)]


def _segments(counts, head, tail):
    """CSR offsets with `head` queries before the first segment and `tail` after the last."""
    seg = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64) + head
    Q = int(seg[-1]) + tail
    glyph = np.full(Q, -1, np.int32)
    for g in range(len(counts)):
        glyph[seg[g]:seg[g + 1]] = g
    return seg, glyph, Q


def _check_dlut(got, ref, tol=2e-5):
    for ch in range(4):
        scale = np.abs(ref[:, ch]).max()
        assert np.abs(got[:, ch] - ref[:, ch]).max() <= tol * scale, ch


def _check_ddirs(dd, ddref, dirs, N, inside):
    ok = inside & ~near_edge(None, dirs, [N], None, eps=1e-4)
    scale = np.abs(ddref[ok]).max()
    assert np.abs(dd[ok] - ddref[ok]).max() <= 1e-4 * scale
    assert np.isnan(dd[~inside]).all()


@pytest.mark.parametrize("dtype", [0, 1, 2])
def test_staged_backward_segment_edges(S, dtype):
    N, L = 16, 6
    counts = np.array([0, 1, 511, 0, 512, 513, 3 * 512 + 17, 0, 5, 2048])
    G = len(counts)
    luts = _pool(G, N, L, 300)
    Lp, stored = upload_pool(S, luts, dtype=dtype)
    seg, glyph, Q = _segments(counts, head=37, tail=1100)
    dirs = I.directions(Q, 301)
    rng = np.random.default_rng(302)
    gR = rng.normal(size=Q).astype(np.float32)
    gG = rng.normal(size=(Q, 3)).astype(np.float32)
    gn = rng.normal(size=(Q, 3)).astype(np.float32)
    dl = S.like_lut(Lp, dtype=0, layout=0, zero=True)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    dd = S.query_backward(Lp, _t(dirs), dl, gR=_t(gR), ggrad=_t(gG), gnormal=_t(gn), seg=_t(seg), dev_status=st)
    torch.cuda.synchronize()
    assert st.item() & S.SHM_DEV_BOUNDS
    inside = glyph >= 0
    off, Ns = O.make_pool(luts)[1:]
    dref, ddref = O.query_vjp(stored.reshape(-1, 4), off, Ns, dirs[inside], gR=gR[inside], gG=gG[inside],
                              gn=gn[inside], glyph=glyph[inside])
    _check_dlut(dl.data.view(-1, 4).double().cpu().numpy(), dref)
    full = np.full((Q, 3), np.nan)
    full[inside] = ddref
    _check_ddirs(dd.double().cpu().numpy(), full, dirs, N, inside)


@pytest.mark.parametrize("which", ["gR", "ggrad", "gnormal", "gR+gnormal"])
def test_staged_backward_upstream_subsets(S, which):
    """Each subset of upstream gradients: the staged pass against the per-query-glyph pass
    (the general kernel, footprints through L1/L2) and the oracle."""
    N, L, G, per = 12, 4, 7, 1500
    luts = _pool(G, N, L, 310)
    Lp, stored = upload_pool(S, luts)
    Q = G * per
    dirs = I.directions(Q, 311)
    rng = np.random.default_rng(312)
    up = {"gR": rng.normal(size=Q).astype(np.float32), "ggrad": rng.normal(size=(Q, 3)).astype(np.float32),
          "gnormal": rng.normal(size=(Q, 3)).astype(np.float32)}
    use = {k: (k in which.split("+")) for k in up}
    kw = {k: (_t(v) if use[k] else None) for k, v in up.items()}
    seg = I.query_glyphs_csr(G, per)
    glyph = np.repeat(np.arange(G), per).astype(np.int32)
    dl_s = S.like_lut(Lp, zero=True)
    dd_s = S.query_backward(Lp, _t(dirs), dl_s, seg=_t(seg), **kw)
    dl_g = S.like_lut(Lp, zero=True)
    dd_g = S.query_backward(Lp, _t(dirs), dl_g, glyph=_t(glyph), **kw)
    off, Ns = O.make_pool(luts)[1:]
    dref, ddref = O.query_vjp(stored.reshape(-1, 4), off, Ns, dirs, gR=up["gR"] if use["gR"] else None,
                              gG=up["ggrad"] if use["ggrad"] else None, gn=up["gnormal"] if use["gnormal"] else None,
                              glyph=glyph)
    inside = np.ones(Q, bool)
    for dl, dd in ((dl_s, dd_s), (dl_g, dd_g)):
        _check_dlut(dl.data.view(-1, 4).double().cpu().numpy(), dref)
        _check_ddirs(dd.double().cpu().numpy(), ddref, dirs, N, inside)
    # the same per-query arithmetic: d/ddirs agree to rounding between the two kernels
    a, b = dd_s.double().cpu().numpy(), dd_g.double().cpu().numpy()
    assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()


def test_staged_backward_many_glyphs(S):
    """More glyphs than CTAs, ragged and empty segments interleaved: every CTA walks several
    glyphs, restaging the table between them; the deterministic pass agrees too."""
    N, L = 8, 4
    rng = np.random.default_rng(320)
    G = 700
    counts = rng.integers(0, 400, size=G)
    counts[rng.choice(G, 80, replace=False)] = 0
    counts[5], counts[6] = 1024, 2049
    luts = _pool(G, N, L, 1000)
    Lp, stored = upload_pool(S, luts)
    seg, glyph, Q = _segments(counts, head=0, tail=0)
    dirs = I.directions(Q, 321)
    gR = rng.normal(size=Q).astype(np.float32)
    gn = rng.normal(size=(Q, 3)).astype(np.float32)
    dl = S.like_lut(Lp, zero=True)
    dd = S.query_backward(Lp, _t(dirs), dl, gR=_t(gR), gnormal=_t(gn), seg=_t(seg))
    dl_det = S.like_lut(Lp, zero=True)
    S.query_backward(Lp, _t(dirs), dl_det, gR=_t(gR), gnormal=_t(gn), seg=_t(seg), deterministic=True)
    off, Ns = O.make_pool(luts)[1:]
    dref, ddref = O.query_vjp(stored.reshape(-1, 4), off, Ns, dirs, gR=gR, gn=gn, glyph=glyph)
    _check_dlut(dl.data.view(-1, 4).double().cpu().numpy(), dref)
    _check_dlut(dl_det.data.view(-1, 4).double().cpu().numpy(), dref)
    _check_ddirs(dd.double().cpu().numpy(), ddref, dirs, N, np.ones(Q, bool))


def test_staged_fit_backward(S):
    """The fused fit loss on the staged pass (segments) against the per-query-glyph pass and the
    oracle's loss and gradient."""
    G, N, per = 5, 10, 2500
    luts = _pool(G, N, 4, 330)
    Lp, stored = upload_pool(S, luts)
    Q = G * per
    dirs = I.directions(Q, 331)
    glyph = np.repeat(np.arange(G), per).astype(np.int32)
    c = I.sh_coeffs(G, 6, 332)
    Rt, _, nt = O.sh_eval(6, c, dirs, glyph=glyph)
    Rt32, nt32 = Rt.astype(np.float32), nt.astype(np.float32)
    out = {}
    for name, kw in (("seg", {"seg": _t(I.query_glyphs_csr(G, per))}), ("glyph", {"glyph": _t(glyph)})):
        dl = S.like_lut(Lp, zero=True)
        loss = torch.zeros(1, device="cuda")
        S.fit_backward(Lp, _t(dirs), _t(Rt32), _t(nt32), dl, w_value=1.0, w_normal=0.25, loss=loss, **kw)
        out[name] = (loss.item(), dl.data.view(-1, 4).double().cpu().numpy())
    off, Ns = O.make_pool(luts)[1:]
    lref, dref = OF.loss_and_grad(stored.reshape(-1, 4), off, Ns, dirs, Rt32.astype(np.float64),
                                  nt32.astype(np.float64), 1.0, 0.25, glyph=glyph)
    for name, (loss, dl) in out.items():
        assert abs(loss - lref) <= 1e-5 * lref, name
        _check_dlut(dl, dref)


def test_paired_reductions_across_glyphs_of_different_n(S):
    """The unstaged pass (uneven N, per-query glyph ids): lane pairs that straddle two glyphs of
    different resolution (odd segment boundaries), glyph ids outside the pool, non-finite
    directions and a ragged last warp.  dlut against the oracle over the valid queries; d/ddirs
    NaN and the status bits set for the invalid ones."""
    Ns, L = [4, 12, 31, 9], 4
    luts = [O.bake_sh(n, L, I.sh_coeffs(1, L, 340 + k)[0] + np.eye(1, (L + 1) ** 2, 0)[0] * 2.0)
            for k, n in enumerate(Ns)]
    Lp, stored = upload_pool(S, luts)
    counts = [101, 3, 2001, 777]
    glyph = np.repeat(np.arange(4), counts).astype(np.int32)
    Q = len(glyph)  # 2882: not a multiple of 32
    rng = np.random.default_rng(341)
    bad_id = rng.choice(Q, 40, replace=False)
    glyph[bad_id[:20]] = -1
    glyph[bad_id[20:]] = 4
    dirs = I.directions(Q, 342)
    bad_dir = rng.choice(np.setdiff1d(np.arange(Q), bad_id), 10, replace=False)
    dirs[bad_dir[:5]] = np.nan
    dirs[bad_dir[5:]] = 0.0
    gR = rng.normal(size=Q).astype(np.float32)
    gG = rng.normal(size=(Q, 3)).astype(np.float32)
    dl = S.like_lut(Lp, zero=True)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    dd = S.query_backward(Lp, _t(dirs), dl, gR=_t(gR), ggrad=_t(gG), glyph=_t(glyph), dev_status=st)
    torch.cuda.synchronize()
    assert st.item() & S.SHM_DEV_BOUNDS and st.item() & S.SHM_DEV_NONFINITE
    ok = np.ones(Q, bool)
    ok[bad_id] = False
    ok[bad_dir] = False
    off, Ns_ = O.make_pool(luts)[1:]
    dref, ddref = O.query_vjp(stored.reshape(-1, 4), off, Ns_, dirs[ok], gR=gR[ok], gG=gG[ok], glyph=glyph[ok])
    _check_dlut(dl.data.view(-1, 4).double().cpu().numpy(), dref)
    ddn = dd.double().cpu().numpy()
    assert np.isnan(ddn[~ok]).all() and np.isfinite(ddn[ok]).all()
