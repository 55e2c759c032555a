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
