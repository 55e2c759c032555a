"""The Python binding's own argument checks (dtype, contiguity, shape), which run before any call
into the library and so need no device: wrong arguments fail with TypeError / ValueError naming the
argument, instead of reaching a kernel."""
import pytest
import torch

import paper_2602_20063_gb300 as S


def _lut(G=3, N=4):
    T = 6 * (N + 2) ** 2
    return S.Lut(data=torch.zeros(G * T * 4), n_glyphs=G, N_uniform=N)


def test_query_checks_its_arguments():
    lut = _lut()
    with pytest.raises(TypeError, match="dirs"):
        S.query(lut, torch.zeros(10, 3, dtype=torch.float64))
    with pytest.raises(ValueError, match="dirs"):
        S.query(lut, torch.zeros(3, 10).t())  # not contiguous
    with pytest.raises(ValueError, match="glyph"):
        S.query(lut, torch.zeros(10, 3), glyph=torch.zeros(9, dtype=torch.int32))
    with pytest.raises(TypeError, match="glyph"):
        S.query(lut, torch.zeros(10, 3), glyph=torch.zeros(10, dtype=torch.int64))
    with pytest.raises(ValueError, match="seg"):
        S.query(lut, torch.zeros(10, 3), seg=torch.zeros(3, dtype=torch.int64))  # needs G + 1 entries


def test_backward_and_fit_check_their_arguments():
    lut, dl = _lut(), _lut()
    with pytest.raises(TypeError, match="gR"):
        S.query_backward(lut, torch.zeros(10, 3), dl, gR=torch.zeros(10, dtype=torch.float64))
    with pytest.raises(ValueError, match="R_target"):
        S.fit_backward(lut, torch.zeros(10, 3), torch.zeros(11), torch.zeros(10, 3), dl)
    with pytest.raises(ValueError, match="n_target"):
        S.fit_backward(lut, torch.zeros(10, 3), torch.zeros(10), torch.zeros(10, 4), dl)


def test_adam_checks_its_arguments():
    p = torch.zeros(8)
    with pytest.raises(TypeError, match="m"):
        S.adam_step(p, torch.zeros(8), torch.zeros(8, dtype=torch.float64), torch.zeros(8), lr=1e-2, step=1)
    with pytest.raises(ValueError, match="v"):
        S.adam_step(p, torch.zeros(8), torch.zeros(8), torch.zeros(7), lr=1e-2, step=1)
