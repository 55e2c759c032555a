"""The package's quick-start sequence (alloc_lut, Source, sh_basis, build_lut with a workspace, so
the tensor-core bake, then a segmented query) run with seeded inputs on 64 glyphs and checked
against the oracle on sampled glyphs.

Tolerances: the tensor-core bake keeps each record channel within 4e-6 of its range (test_gpu_build),
and the query on identical bytes is within 1e-5 max|R| and 1e-4 max|grad R| (test_gpu_query).  A
value-channel error e reaches the gradient as about 1.5 N e (the Hermite derivative of a difference),
which at N = 32 is below 1e-4 max|grad R| for these fields.  So the bounds are R 2e-5 max|R|,
gradient 2e-4 max|grad R|, and normals 1e-3.  A dropped term, a wrong sign or a transposed operand
misses these by orders of magnitude.
"""
import numpy as np
import pytest
import torch

import oracle as O
from gpu_common import shm

pytestmark = pytest.mark.gpu


def test_quick_start_sequence():
    S = shm()
    G, L, N, per = 64, 8, 32, 4096
    gen = torch.Generator().manual_seed(20063)
    coeffs = torch.randn(G, (L + 1) ** 2, generator=gen).cuda()
    lut = S.alloc_lut(G, N)
    src = S.Source(kind=S.SHM_SRC_SH, L=L, coeffs=coeffs, basis=S.sh_basis(N, L))
    S.build_lut(lut, src, ws=S.build_workspace(lut, src))

    dirs = torch.nn.functional.normalize(torch.randn(G * per, 3, generator=gen), dim=1).cuda()
    seg = torch.arange(0, G * per + 1, per, device="cuda")
    out = S.query(lut, dirs, seg=seg)
    torch.cuda.synchronize()
    assert set(out) == {"R", "grad", "normal"}
    assert out["R"].shape == (G * per,) and out["grad"].shape == (G * per, 3) and out["normal"].shape == (G * per, 3)
    for v in out.values():
        assert bool(torch.isfinite(v).all())

    c64 = coeffs.double().cpu().numpy()
    d_host = dirs.cpu().numpy()
    picks = (0, 17, 40, G - 1)
    pool, off, Ns = O.make_pool([O.bake_sh(N, L, c64[g]) for g in picks])
    rows = np.concatenate([np.arange(g * per, (g + 1) * per) for g in picks])
    glyph = np.repeat(np.arange(len(picks), dtype=np.int32), per)
    ref = O.query(pool, off, Ns, d_host[rows], glyph=glyph)
    got = {k: v.cpu().numpy().astype(np.float64)[rows] for k, v in out.items()}
    assert np.abs(got["R"] - ref["R"]).max() <= 2e-5 * np.abs(ref["R"]).max()
    assert np.abs(got["grad"] - ref["grad"]).max() <= 2e-4 * np.abs(ref["grad"]).max()
    assert np.abs(got["normal"] - ref["normal"]).max() <= 1e-3
