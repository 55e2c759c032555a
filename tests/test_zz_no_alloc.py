"""shm_raycast_noalloc: the ray caster for callers that cannot allocate device memory when they
render (an application that owns the GPU memory budget through its own pool, or a frame loop in
which cudaMalloc would synchronise the device).  Its workspace is a static device array inside
libshm.so.  Checked through the C ABI against shm_raycast (caller workspace) on two calls in a
row, so that the second call also shows that state left in the shared array by the first one does
not leak into its result; oversized requests are refused before any launch.

This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

import shm_inputs as I

pytestmark = pytest.mark.gpu


def _shm():
    from paper_2602_20063_gb300 import build as B
    B.build()
    import paper_2602_20063_gb300 as S
    L = S.lib()
    L.shm_raycast_noalloc.restype = C.c_int
    L.shm_raycast_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    return S, L


def _scene(S, n, seed, N=24):
    counts, offs, mu, amp, width = I.bump_params(n, seed)
    lut = S.alloc_lut(n, N, r0=[1.0] * n)
    S.build_lut(lut, S.Source(kind=S.SHM_SRC_BUMPS, bump_offset=torch.from_numpy(offs).cuda(),
                              mu=torch.from_numpy(mu.astype(np.float32)).cuda(),
                              amp=torch.from_numpy(amp.astype(np.float32)).cuda(),
                              width=torch.from_numpy(width.astype(np.float32)).cuda()))
    rmax = S.lut_bounds(lut)
    side = int(round(n ** (1 / 3)))
    g = (np.arange(side) - (side - 1) / 2) * 2.6
    centres = np.array([[x, y, z] for x in g for y in g for z in g])[:n]
    objs = S.objects_tensor(centres, np.ones(n), rmax.cpu().numpy(), np.arange(n))
    return lut, objs


def _camera(S, W, H, eye):
    eye = np.asarray(eye, dtype=np.float64)
    fwd = -eye / np.linalg.norm(eye)
    right = np.cross(fwd, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    return S.make_camera(eye, fwd, right, up, 45.0, W, H)


def _outputs(W, H):
    return ({"rgba": torch.full((H, W, 4), -7.0, device="cuda"), "depth": torch.full((H, W), -7.0, device="cuda"),
             "normal": torch.full((H, W, 3), -7.0, device="cuda"),
             "obj_id": torch.full((H, W), -7, dtype=torch.int32, device="cuda")},
            torch.zeros(1, dtype=torch.int32, device="cuda"))


def _device_memory():
    """(free device bytes as the driver reports them, bytes held by torch's allocator)."""
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()


def _noalloc(S, L, lut, objs, n, cam, prm, bufs=None):
    out, st = bufs if bufs is not None else _outputs(cam.W, cam.H)
    rc = L.shm_raycast_noalloc(C.byref(lut.c()), objs.data_ptr(), n, C.byref(cam), C.byref(prm),
                               out["rgba"].data_ptr(), out["depth"].data_ptr(), out["normal"].data_ptr(),
                               out["obj_id"].data_ptr(), st.data_ptr(),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out, st


def _same(a, b):
    assert torch.equal(a["obj_id"], b["obj_id"])
    hit = a["obj_id"] >= 0
    for k in ("rgba", "depth", "normal"):
        x, y = a[k][hit], b[k][hit]
        assert torch.allclose(x, y, rtol=2e-5, atol=2e-5), k
    assert torch.all(torch.isinf(a["depth"][~hit])) and torch.all(torch.isinf(b["depth"][~hit]))


def test_noalloc_matches_workspace_entry_point_twice():
    S, L = _shm()
    prm = S.make_raycast_params()
    # two different scenes in a row: the second call starts from the first call's leftover scratch
    for k, (n, seed, W, H, eye) in enumerate(((27, 11, 320, 200, (3.0, 4.0, 14.0)),
                                              (64, 12, 480, 270, (-5.0, 2.0, 16.0)))):
        lut, objs = _scene(S, n, seed)
        cam = _camera(S, W, H, eye)
        ref = S.raycast(lut, objs, n, cam, prm)
        bufs = _outputs(W, H)
        before = _device_memory()
        rc, out, st = _noalloc(S, L, lut, objs, n, cam, prm, bufs)
        after = _device_memory()
        assert rc == 0, rc
        assert st.item() == 0
        if k == 1:
            # the first call on the device may have set up the library's static array; from then on
            # a call allocates nothing, neither through the driver nor through torch's pool
            assert after == before, (before, after)
        assert (ref["obj_id"] >= 0).float().mean() > 0.05
        _same(out, ref)
        del ref, bufs, out, st  # released before the next call's "before" reading


def test_noalloc_python_wrapper():
    """The binding's raycast_noalloc gives the same image as shm_raycast with a caller workspace."""
    S, _ = _shm()
    prm = S.make_raycast_params()
    lut, objs = _scene(S, 27, 14)
    cam = _camera(S, 256, 160, (2.0, -3.0, 13.0))
    ref = S.raycast(lut, objs, 27, cam, prm)
    out = S.raycast_noalloc(lut, objs, 27, cam, prm)
    torch.cuda.synchronize()
    _same(out, ref)


def test_noalloc_full_hd_capacity_and_refusal():
    S, L = _shm()
    n = 512
    lut, objs = _scene(S, n, 13, N=16)
    prm = S.make_raycast_params(march=16, bisect=8, newton=2)
    cam = _camera(S, 1920, 1080, (0.0, 0.0, 40.0))
    assert S.raycast_workspace_bytes(n, 1920, 1080) <= 16 * 1024 * 1024
    ref = S.raycast(lut, objs, n, cam, prm)
    rc, out, _ = _noalloc(S, L, lut, objs, n, cam, prm)
    torch.cuda.synchronize()
    assert rc == 0
    _same(out, ref)
    # beyond the static capacity: refused on the host with SHM_ERR_WORKSPACE, nothing launched
    big = _camera(S, 3840, 2160, (0.0, 0.0, 40.0))
    rc, out, _ = _noalloc(S, L, lut, objs, n, big, prm)
    torch.cuda.synchronize()
    assert rc == 3
    assert torch.all(out["obj_id"] == -7)
