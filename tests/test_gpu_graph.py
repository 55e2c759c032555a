"""The library's calls inside CUDA-graph capture: a glyph step (tcgen05 SH bake + staged segment
query) and a reverse pass captured once and replayed give the same bytes as eager calls (no
allocation, no synchronisation and no host work that depends on device data inside the calls)."""
import numpy as np
import pytest
import torch

import shm_inputs as I
from gpu_common import shm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    return shm()


def test_bake_query_backward_replay(S):
    G, L, N, per = 96, 8, 32, 2048
    Q = G * per
    c = torch.from_numpy(I.sh_coeffs(G, L, 950).astype(np.float32)).cuda()
    lut = S.alloc_lut(G, N)
    src = S.Source(kind=S.SHM_SRC_SH, L=L, coeffs=c, basis=S.sh_basis(N, L))
    ws = S.build_workspace(lut, src)
    d = torch.from_numpy(I.directions(Q, 951)).cuda()
    seg = torch.from_numpy(I.query_glyphs_csr(G, per)).cuda()
    gR = torch.from_numpy(np.random.default_rng(952).standard_normal(Q).astype(np.float32)).cuda()
    out = {k: torch.empty(s, device="cuda") for k, s in (("R", (Q,)), ("grad", (Q, 3)), ("normal", (Q, 3)))}
    dl = S.like_lut(lut, zero=True)

    def step():
        S.build_lut(lut, src, ws=ws)
        S.query(lut, d, seg=seg, out=out)
        dl.data.zero_()
        S.query_backward(lut, d, dl, gR=gR, seg=seg, want_ddirs=False, deterministic=True)

    step()  # eager: first-use attributes and tensor maps outside the capture
    torch.cuda.synchronize()
    ref = {k: v.clone() for k, v in out.items()}
    ref_tab, ref_dl = lut.data.clone(), dl.data.clone()
    for v in list(out.values()) + [lut.data, dl.data]:
        v.fill_(float("nan"))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for v in list(out.values()) + [lut.data, dl.data]:
        v.fill_(float("nan"))
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(lut.data, ref_tab)
    for k in ref:
        assert torch.equal(out[k], ref[k]), k
    assert torch.equal(dl.data, ref_dl)  # the deterministic reverse pass: same bits on replay
