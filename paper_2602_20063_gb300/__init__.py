"""GB300 (sm_103a) Spherical Hermite Maps: batched evaluation of star-shaped radial functions
through padded cubemap Hermite tables (Abouagour & Garyfallidis, arXiv 2602.20063).

The compute lives in libshm.so (CUDA, C ABI in include/shm.h); this package is its thin
binding plus the autograd wrapper.  See ``binding`` for the entry points.
"""
from .binding import (  # noqa: F401
    SHM_F32, SHM_F16, SHM_BF16, SHM_LAYOUT_TEXEL, SHM_LAYOUT_CELL, SHM_LAYOUT_VALUE,
    SHM_RECON_NEAREST, SHM_RECON_BILINEAR, SHM_RECON_BICUBIC, SHM_RECON_FAST_BICUBIC,
    SHM_SRC_SH, SHM_SRC_SAMPLES, SHM_SRC_BUMPS, SHM_SRC_FBM,
    SHM_DEV_NONFINITE, SHM_DEV_BOUNDS, SHM_DEV_TIMEOUT, SHM_BWD_DETERMINISTIC, SHM_BWD_CUDA_CORES,
    Lut, Source, ShmError, alloc_lut, like_lut, lib, lib_path,
    query, query_binned, query_binned_workspace, query_binned_workspace_bytes, query_binned_bins, query_recon, tune_query, tune_reset, sh_basis, build_lut, build_workspace, build_workspace_bytes, pack_lut, lut_bounds, build_mip, mip_like, mip_chain, query_backward, build_lut_backward, sh_eval, fit_backward, adam_step,
    make_camera, make_raycast_params, objects_tensor, raycast, raycast_noalloc, raycast_workspace_bytes, raycast_query_count,
    records_per_glyph, record_bytes, l2_fetch_granularity,
)
from .autograd import query_fn, sh_bake_fn  # noqa: F401
