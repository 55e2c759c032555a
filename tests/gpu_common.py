"""Helpers shared by the GPU parity tests: device tables made from oracle tables, tolerances."""
import numpy as np
import torch

import oracle as O
import shm_inputs as I


def shm():
    from paper_2602_20063_gb300 import build as B
    B.build()
    import paper_2602_20063_gb300 as S
    S.lib()
    return S


def upload_pool(S, luts, r0=None, dtype=0, layout=0):
    """Oracle float64 glyph tables -> float32 texel pool on the device (same bytes the oracle gets
    back through ``stored_f64``), then packed on the device into (dtype, layout)."""
    Ns = [l.shape[1] - 2 for l in luts]
    uniform = len(set(Ns)) == 1
    lut32 = S.alloc_lut(len(luts), Ns[0] if uniform else Ns, 0, 0, r0=r0)
    host = np.concatenate([np.asarray(l, dtype=np.float32).reshape(-1) for l in luts])
    lut32.data.copy_(torch.from_numpy(host))
    if dtype == 0 and layout == 0:
        return lut32, host.astype(np.float64)
    dst = S.like_lut(lut32, dtype=dtype, layout=layout)
    S.pack_lut(lut32, dst)
    if dtype == 1:
        stored = O.quantize_f16(host)
    elif dtype == 2:
        stored = O.quantize_bf16(host)
    else:
        stored = host.astype(np.float64)
    return dst, stored


def oracle_pool_meta(luts):
    pool, off, Ns = O.make_pool(luts)
    return off, Ns


def near_edge(fij_o, dirs, Ns, glyph, eps=1e-6):
    """Queries within eps of a cell edge or a face tie: indices may legitimately differ."""
    d = dirs.astype(np.float64)
    a = np.sort(np.abs(d), axis=1)
    tie = (a[:, 2] - a[:, 1]) <= eps * a[:, 2]
    k = np.argmax(np.abs(d), axis=1)
    m = np.abs(d[np.arange(len(d)), k])
    N = np.asarray(Ns)[glyph] if glyph is not None else np.full(len(d), Ns[0])
    edge = np.zeros(len(d), dtype=bool)
    for ax in (1, 2):
        q = d[np.arange(len(d)), (k + ax) % 3] / m
        x = (q + 1.0) / 2.0 * N + 0.5
        fr = x - np.floor(x)
        edge |= (fr < eps * N) | (fr > 1 - eps * N)
    return tie | edge


def check_query(out_gpu, ref, tol_scale=1.0, mask=None):
    """Value <= 1e-5 max|R|, gradient <= 1e-4 max|grad R|; normal within the propagated bound."""
    R = out_gpu["R"].double().cpu().numpy()
    G = out_gpu["grad"].double().cpu().numpy()
    if mask is None:
        mask = np.ones(len(R), dtype=bool)
    maxR = np.abs(ref["R"]).max()
    maxG = np.linalg.norm(ref["grad"], axis=1).max()
    tR, tG = 1e-5 * maxR * tol_scale, 1e-4 * maxG * tol_scale
    eR = np.abs(R - ref["R"])[mask].max()
    eG = np.abs(G - ref["grad"])[mask].max()
    assert eR <= tR, (eR, tR)
    assert eG <= tG, (eG, tG)
    if "normal" in out_gpu:
        Nn = out_gpu["normal"].double().cpu().numpy()
        mlen = np.sqrt(ref["R"] ** 2 + (ref["grad"] ** 2).sum(1))
        bound = 2.0 * (tR + tG) / np.maximum(mlen, 1e-30) + 1e-6
        err = np.abs(Nn - ref["normal"]).max(1)
        assert np.all((err <= bound)[mask]), (err / bound)[mask].max()
    return eR / maxR, eG / maxG
