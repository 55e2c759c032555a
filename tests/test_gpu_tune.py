"""Launch-shape autotuning of shm_query: every shape gives the same results; the fastest is kept
per device, path, dtype and layout, and shm_tune_reset restores the default."""
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


def _same(a, b):
    return all(torch.equal(a[k], b[k]) for k in ("R", "grad", "normal"))


@pytest.mark.parametrize("path", ["glyph_ids", "segments"])
def test_tuned_shapes_give_identical_results(S, path):
    G, N, per = 24, 32, 3000
    luts = [O.bake_sh(N, 6, I.sh_coeffs(1, 6, 700 + g)[0]) for g in range(G)]
    L, _ = upload_pool(S, luts)
    d = torch.from_numpy(I.directions(G * per, 701)).cuda()
    kw = ({"glyph": torch.from_numpy(np.repeat(np.arange(G, dtype=np.int32), per)).cuda()} if path == "glyph_ids"
          else {"seg": torch.from_numpy(I.query_glyphs_csr(G, per)).cuda()})
    S.tune_reset()
    before = S.query(L, d, **kw)
    info = S.tune_query(L, d, reps=2, **kw)
    n_shapes = 4 if path == "glyph_ids" else 3
    assert 0 <= info["chosen"] < n_shapes
    assert all(t > 0 for t in info["times_ms"][:n_shapes])
    assert all(t == -1 for t in info["times_ms"][n_shapes:])
    after = S.query(L, d, **kw)
    assert _same(before, after)
    S.tune_reset()
    assert _same(before, S.query(L, d, **kw))


def test_tune_rejects_bad_arguments(S):
    L, _ = upload_pool(S, [O.bake_sh(8, 4, I.sh_coeffs(1, 4, 710)[0])])
    d = torch.from_numpy(I.directions(100, 711)).cuda()
    with pytest.raises(S.ShmError):
        S.tune_query(L, d, reps=0)
    with pytest.raises(S.ShmError):
        S.tune_query(L, d[:0], reps=1)


def test_l2_fetch_granularity_round_trip(S):
    """shm_l2_fetch_granularity sets the context limit, reports the previous value and leaves query
    results unchanged (it is a fetch-size hint only)."""
    N, per = 32, 5000
    L, _ = upload_pool(S, [O.bake_sh(N, 6, I.sh_coeffs(1, 6, 702)[0])])
    d = torch.from_numpy(I.directions(per, 703)).cuda()
    before = S.query(L, d)
    prev = S.l2_fetch_granularity(-1)
    assert 0 <= prev <= 128
    try:
        assert S.l2_fetch_granularity(32) == prev
        assert S.l2_fetch_granularity(-1) == 32
        assert _same(before, S.query(L, d))
    finally:
        S.l2_fetch_granularity(prev)
    assert S.l2_fetch_granularity(-1) == prev
