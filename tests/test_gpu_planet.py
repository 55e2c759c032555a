"""End-to-end parity of the procedural planet at full resolution (N = 2048, table 403 MB): device fBm
bake + device query versus the oracle evaluating each sampled query from the procedural source
itself (the 4 x 4 fBm samples around the query's cell -> central-difference records of the four
corners -> Hermite reconstruction -> S^2 gradient -> normal), without the oracle baking the table.

Tolerance: value <= 1e-5 max|R|.  Gradient: the finite-difference channels difference float32
samples, so a per-sample evaluation error eps_S reaches the chart gradient amplified by N:
|d grad| <= 1e-4 max|grad R| + 3 N eps_S (rho/2 <= 0.87 times the Hermite slope weights); eps_S is
bounded by the float32 rounding of the noise position, measured here against the float64 oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import shm_inputs as I
from gpu_common import shm

pytestmark = pytest.mark.gpu

N = 2048


@pytest.fixture(scope="module")
def planet():
    S = shm()
    keys = I.fbm_keys(20063 + 3)
    lut = S.alloc_lut(1, N, r0=[1.0])
    S.build_lut(lut, S.Source(kind=S.SHM_SRC_FBM, octaves=8, keys=torch.from_numpy(keys.view(np.int32)).cuda(),
                              base_freq=2.0, lacunarity=2.0, gain=0.5, amplitude=0.02))
    return S, lut, keys


def _oracle_query_from_source(keys, d):
    """One query evaluated from the fBm source by the oracle (records baked locally)."""
    w = d / np.linalg.norm(d)
    f, u, v = O.face_uv(d)
    i, s = O.cell(N, u)
    j, t = O.cell(N, v)
    samp = np.zeros((4, 4))  # texels i-1..i+2, j-1..j+2
    for b in range(4):
        for a in range(4):
            wt = O.dir_tilde(f, O.texel_centre(i - 1 + a, N), O.texel_centre(j - 1 + b, N))
            samp[b, a] = 0.02 * O.fbm(wt / np.linalg.norm(wt), keys)
    mini = np.zeros((2, 2, 4))
    for bb in range(2):
        for aa in range(2):
            y, x = bb + 1, aa + 1
            mini[bb, aa] = [samp[y, x], (samp[y, x + 1] - samp[y, x - 1]) / 2, (samp[y + 1, x] - samp[y - 1, x]) / 2,
                            (samp[y + 1, x + 1] - samp[y - 1, x + 1] - samp[y + 1, x - 1] + samp[y - 1, x - 1]) / 4]
    h = O.hermite_eval(mini, 0, 0, 0, s, t)  # a 2 x 2 patch: padded width 2
    R = 1.0 + h[0]
    g = O.s2_gradient(f, u, v, N * h[1], N * h[2])
    return R, g, O.normal(w, R, g)


def test_planet_sampled_queries_full_resolution(planet):
    S, lut, keys = planet
    Q = 1 << 20
    dirs = I.directions(Q, 20063 + 33)
    out = S.query(lut, torch.from_numpy(dirs).cuda())
    R = out["R"].double().cpu().numpy()
    G = out["grad"].double().cpu().numpy()
    Nn = out["normal"].double().cpu().numpy()
    rng = np.random.default_rng(7)
    idx = rng.choice(Q, 1500, replace=False)
    ref = [_oracle_query_from_source(keys, dirs[q].astype(np.float64)) for q in idx]
    Rr = np.array([r[0] for r in ref])
    Gr = np.array([r[1] for r in ref])
    Nr = np.array([r[2] for r in ref])
    maxG = np.linalg.norm(Gr, axis=1).max()
    eR = np.abs(R[idx] - Rr).max()
    eG = np.abs(G[idx] - Gr).max()
    eN = np.abs(Nn[idx] - Nr).max()
    eps_S = 2e-8  # float32 noise-position rounding, amplitude 0.02 (see test_fbm_planet_sampled_texels)
    print(f"planet N=2048: max|dR| {eR:.3e}, max|dgrad| {eG:.3e} (max|grad| {maxG:.3f}), max|dn| {eN:.3e}")
    assert eR <= 1e-5 * np.abs(Rr).max()
    assert eG <= 1e-4 * maxG + 3 * N * eps_S
    assert eN <= 2e-3
