"""Per-query buffers in page-locked host memory: the kernels read directions (and upstream
gradients) and write outputs directly over the host link.  Results must equal the device-buffer
call bit for bit; pageable host memory is refused before any launch."""
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


def _pool(S, G=20, N=32, L=6, seed=900):
    luts = [O.bake_sh(N, L, I.sh_coeffs(1, L, seed + g)[0]) for g in range(G)]
    return upload_pool(S, luts)[0]


@pytest.mark.parametrize("path", ["segments", "glyph_ids"])
def test_query_host_buffers_match_device(S, path):
    G, per = 20, 2500
    L = _pool(S, G)
    d = torch.from_numpy(I.directions(G * per, 901))
    kw = ({"seg": torch.from_numpy(I.query_glyphs_csr(G, per))} if path == "segments"
          else {"glyph": torch.from_numpy(np.repeat(np.arange(G, dtype=np.int32), per))})
    ref = S.query(L, d.cuda(), **{k: v.cuda() for k, v in kw.items()}, want=("R", "grad", "normal", "fij"))
    dh = d.pin_memory()
    # host directions and host outputs; segments / glyph ids on the host too
    got = S.query(L, dh, **{k: v.pin_memory() for k, v in kw.items()}, want=("R", "grad", "normal", "fij"))
    torch.cuda.synchronize()
    assert all(v.device.type == "cpu" and v.is_pinned() for v in got.values())
    for k in ref:
        assert torch.equal(ref[k].cpu(), got[k]), k
    # mixed: host directions, device outputs
    mixed = S.query(L, dh, **{k: v.cuda() for k, v in kw.items()},
                    out={k: torch.empty_like(v) for k, v in ref.items()})
    torch.cuda.synchronize()
    for k in ref:
        assert torch.equal(ref[k], mixed[k]), k


def test_pageable_host_memory_is_refused(S):
    L = _pool(S, 2)
    d = torch.from_numpy(I.directions(1000, 902))  # pageable
    out = {k: torch.full(s, 7.0, device="cuda") for k, s in (("R", (1000,)), ("grad", (1000, 3)))}
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(S.ShmError):
        S.query(L, d, seg=torch.tensor([0, 500, 1000], dtype=torch.int64).cuda(), out=out, dev_status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and bool((out["R"] == 7.0).all())  # nothing was launched


def test_backward_host_buffers_match_device(S):
    G, per = 20, 2000
    L = _pool(S, G, seed=910)
    Q = G * per
    d = torch.from_numpy(I.directions(Q, 911))
    seg = torch.from_numpy(I.query_glyphs_csr(G, per))
    g = torch.Generator().manual_seed(912)
    gR, gG, gN = torch.randn(Q, generator=g), torch.randn((Q, 3), generator=g), torch.randn((Q, 3), generator=g)
    dl_dev = S.like_lut(L, dtype=S.SHM_F32, layout=S.SHM_LAYOUT_TEXEL, zero=True)
    dd_dev = S.query_backward(L, d.cuda(), dl_dev, gR=gR.cuda(), ggrad=gG.cuda(), gnormal=gN.cuda(), seg=seg.cuda())
    dl_host = S.like_lut(L, dtype=S.SHM_F32, layout=S.SHM_LAYOUT_TEXEL, zero=True)
    dd_host = S.query_backward(L, d.pin_memory(), dl_host, gR=gR.pin_memory(), ggrad=gG.pin_memory(),
                               gnormal=gN.pin_memory(), seg=seg.pin_memory())
    torch.cuda.synchronize()
    assert dd_host.device.type == "cpu" and dd_host.is_pinned()
    assert torch.equal(dd_dev.cpu(), dd_host)
    # atomic accumulation order may differ between the two launches
    a, b = dl_dev.data.cpu().double(), dl_host.data.cpu().double()
    assert float((a - b).abs().max()) <= 1e-5 * float(a.abs().max())


def test_chunked_copy_pipeline_matches_device_step(S):
    """The end-to-end form the glyph-field bench times: glyph chunks whose host-to-device copies run
    on one stream, bake + query on a kernel stream and device-to-host copies on another, ordered by
    per-chunk events only, with consecutive steps overlapping.  Five steps alternate between two
    input sets and two host output sets, reusing the same device buffers, so a missing event shows
    up as outputs mixed from two steps; each output set must equal the plain device step of its
    inputs bit for bit."""
    G, L, N, per, C = 64, 4, 32, 512, 4
    Q, K = G * per, (L + 1) ** 2
    basis = S.sh_basis(N, L)
    lut = S.alloc_lut(G, N)
    seg = torch.from_numpy(I.query_glyphs_csr(G, per)).cuda()
    shapes = (("R", (Q,)), ("grad", (Q, 3)), ("normal", (Q, 3)))
    coeffs_h = [torch.from_numpy(I.sh_coeffs(G, L, 950 + k).astype(np.float32)).pin_memory() for k in range(2)]
    dirs_h = [torch.from_numpy(I.directions(Q, 960 + k)).pin_memory() for k in range(2)]
    outs_h = [{k: torch.full(s, float("nan")).pin_memory() for k, s in shapes} for _ in range(2)]
    coeffs_d = torch.empty((G, K), device="cuda")
    dirs_d = torch.empty((Q, 3), device="cuda")
    out_d = {k: torch.empty(s, device="cuda") for k, s in shapes}
    rec = S.records_per_glyph(N, S.SHM_LAYOUT_TEXEL) * S.record_bytes(S.SHM_F32, S.SHM_LAYOUT_TEXEL) // lut.data.element_size()
    Gc = G // C
    chunks = []
    for c in range(C):
        g0, g1 = c * Gc, (c + 1) * Gc
        lut_c = S.Lut(data=lut.data[g0 * rec:g1 * rec], n_glyphs=Gc, dtype=S.SHM_F32, layout=S.SHM_LAYOUT_TEXEL,
                      N_uniform=N)
        src_c = S.Source(kind=S.SHM_SRC_SH, L=L, coeffs=coeffs_d[g0:g1], basis=basis)
        chunks.append((lut_c, src_c, (seg[g0:g1 + 1] - seg[g0]).contiguous(), g0, g1))
    ws = S.build_workspace(chunks[0][0], chunks[0][1])
    main, h2d, d2h, ks = (torch.cuda.current_stream(), torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream())
    ev_in, ev_q, ev_out = ([torch.cuda.Event() for _ in range(C)] for _ in range(3))
    used = [False] * C
    torch.cuda.synchronize()
    for st in (h2d, d2h, ks):
        st.wait_stream(main)
    for step in range(5):
        sel = step % 2
        for c, (lut_c, src_c, seg_c, g0, g1) in enumerate(chunks):
            q0, q1 = g0 * per, g1 * per
            if used[c]:
                h2d.wait_event(ev_q[c])
            with torch.cuda.stream(h2d):
                dirs_d[q0:q1].copy_(dirs_h[sel][q0:q1], non_blocking=True)
                coeffs_d[g0:g1].copy_(coeffs_h[sel][g0:g1], non_blocking=True)
            ev_in[c].record(h2d)
            ks.wait_event(ev_in[c])
            if used[c]:
                ks.wait_event(ev_out[c])
            S.build_lut(lut_c, src_c, ws=ws, stream=ks)
            out_c = {k: v[q0:q1] for k, v in out_d.items()}
            S.query(lut_c, dirs_d[q0:q1], seg=seg_c, out=out_c, stream=ks)
            ev_q[c].record(ks)
            d2h.wait_event(ev_q[c])
            with torch.cuda.stream(d2h):
                for k in out_c:
                    outs_h[sel][k][q0:q1].copy_(out_c[k], non_blocking=True)
            ev_out[c].record(d2h)
            used[c] = True
    for st in (h2d, d2h, ks):
        main.wait_stream(st)
    torch.cuda.synchronize()
    for sel in range(2):
        lut_r = S.alloc_lut(G, N)
        src_r = S.Source(kind=S.SHM_SRC_SH, L=L, coeffs=coeffs_h[sel].cuda(), basis=basis)
        S.build_lut(lut_r, src_r, ws=S.build_workspace(lut_r, src_r))
        ref = S.query(lut_r, dirs_h[sel].cuda(), seg=seg)
        torch.cuda.synchronize()
        for k in ref:
            assert torch.equal(ref[k].cpu(), outs_h[sel][k]), (sel, k)
