"""PyTorch autograd wrappers over the CUDA query and bake adjoints (argument marshalling only).

``query_fn(table, dirs, lut, seg=None, glyph=None, deterministic=False)`` returns (R, grad, normal)
differentiable with respect to ``table`` (the float32 texel-layout record pool, i.e. ``lut.data``)
and ``dirs``; the backward pass is shm_query_backward (SHM_BWD_DETERMINISTIC when deterministic=True
or torch.are_deterministic_algorithms_enabled(), which needs segments).
``sh_bake_fn(coeffs, basis, lut, L)`` returns the baked table differentiable with respect to the SH
coefficients (backward: shm_build_lut_backward, with a fixed summation order under
deterministic=True or torch's deterministic mode).
Composing the two fits SH coefficients through the table.
"""
from __future__ import annotations

import torch

from . import binding as B


class _Query(torch.autograd.Function):
    @staticmethod
    def forward(ctx, table, dirs, lut, seg, glyph, deterministic):
        if lut.dtype != B.SHM_F32 or lut.layout != B.SHM_LAYOUT_TEXEL:
            raise ValueError("differentiable queries need a float32 texel-layout table")
        view = B.Lut(data=table, n_glyphs=lut.n_glyphs, dtype=lut.dtype, layout=lut.layout,
                     N_uniform=lut.N_uniform, N=lut.N, offset=lut.offset, r0=lut.r0)
        out = B.query(view, dirs.contiguous(), glyph=glyph, seg=seg, want=("R", "grad", "normal"))
        ctx.save_for_backward(table, dirs)
        ctx.lut, ctx.seg, ctx.glyph = view, seg, glyph
        ctx.deterministic = bool(deterministic) or torch.are_deterministic_algorithms_enabled()
        if ctx.deterministic and (seg is None or glyph is not None):
            raise RuntimeError("the deterministic reverse pass of shm_query needs CSR segments (seg), "
                               "not glyph ids: sort the queries by glyph and pass seg")
        return out["R"], out["grad"], out["normal"]

    @staticmethod
    def backward(ctx, gR, gG, gN):
        table, dirs = ctx.saved_tensors
        dl = B.like_lut(ctx.lut, zero=True)
        want_dirs = ctx.needs_input_grad[1]
        c = lambda t: None if t is None else t.contiguous()
        dd = B.query_backward(ctx.lut, dirs.contiguous(), dl, gR=c(gR), ggrad=c(gG), gnormal=c(gN), glyph=ctx.glyph,
                              seg=ctx.seg, want_ddirs=want_dirs, deterministic=ctx.deterministic)
        return (dl.data if ctx.needs_input_grad[0] else None), dd, None, None, None, None


def query_fn(table: torch.Tensor, dirs: torch.Tensor, lut: B.Lut, seg=None, glyph=None, deterministic=False):
    """Differentiable shm_query on a float32 texel table whose records are ``table``."""
    return _Query.apply(table, dirs, lut, seg, glyph, deterministic)


class _ShBake(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coeffs, basis, lut, L, ws, deterministic):
        B.build_lut(lut, B.Source(kind=B.SHM_SRC_SH, L=L, coeffs=coeffs.contiguous(), basis=basis), ws=ws)
        ctx.lut, ctx.L = lut, L
        ctx.deterministic = bool(deterministic) or torch.are_deterministic_algorithms_enabled()
        ctx.save_for_backward(basis)
        return lut.data.clone()

    @staticmethod
    def backward(ctx, gtable):
        (basis,) = ctx.saved_tensors
        D = B.like_lut(ctx.lut, r0=None)
        D.data.copy_(gtable)
        return B.build_lut_backward(D, ctx.L, basis, deterministic=ctx.deterministic), None, None, None, None, None


def sh_bake_fn(coeffs: torch.Tensor, basis: torch.Tensor, lut: B.Lut, L: int, ws: torch.Tensor = None,
               deterministic=False):
    """Differentiable SH bake into ``lut`` (float32 texel layout, uniform N); returns the table records."""
    return _ShBake.apply(coeffs, basis, lut, L, ws, deterministic)
