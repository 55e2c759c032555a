"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds random-number generation and input shapes only: no step of the
Spherical Hermite Map method (no chart mapping, no SH evaluation, no Hermite
reconstruction, no noise or bump evaluation) lives here, so that both sides of
every parity test consume identical input bytes while sharing none of the
arithmetic under test.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014).  Stream ``seed`` yields z_k = mix64(seed + k*GAMMA)
for k = 1, 2, ...; uniforms are the top 53 bits times 2^-53.

Input recipes (workload shapes follow the paper's experiments, section 4):
  * directions: uniform on S^2 via z = 2U-1, phi = 2*pi*U', computed in float64
    and stored float32 (the paper samples "uniform random directions", §4.2).
  * SH coefficients: c_lm = N(0,1)/(l+1)^2 (Box-Muller), c_00 += 2.5 so that the
    radius stays positive (§4.1 uses a fixed-seed L=8 glyph).
  * Gaussian bumps: 8..64 bumps per object, centres uniform on S^2, amplitude
    U[-0.2, 0.2], width U[0.05, 0.4] rad (radial depth-map impostors, §4.9).
  * fBm keys: per-octave 3 x uint32 lattice keys for the value-noise hash
    (procedural planet, §4.10).
"""
from __future__ import annotations

import math
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 20063


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class SplitMix64:
    """Vectorised SplitMix64 stream; ``pos`` counts outputs drawn so far."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.pos = 0

    def u64(self, n: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            k = np.arange(self.pos + 1, self.pos + 1 + n, dtype=np.uint64)
            out = _mix64(self.seed + k * GAMMA)
        self.pos += n
        return out

    def uniform(self, n: int) -> np.ndarray:
        """U[0,1) doubles from the top 53 bits."""
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """N(0,1) by Box-Muller from two uniforms (first uses 1-U to avoid log 0)."""
        u = self.uniform(2 * n).reshape(n, 2)
        return np.sqrt(-2.0 * np.log(1.0 - u[:, 0])) * np.cos(2.0 * math.pi * u[:, 1])

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Integers in [lo, hi] (inclusive) by the multiply-shift of a 53-bit uniform."""
        return lo + np.floor(self.uniform(n) * (hi - lo + 1)).astype(np.int64)


def sub_seed(seed: int, *tags: int) -> int:
    """Deterministic child seed: SplitMix64-mix the parent seed with integer tags."""
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for t in tags:
            s = _mix64(np.array([s + np.uint64(t & 0xFFFFFFFFFFFFFFFF) * GAMMA + GAMMA], dtype=np.uint64))[0]
    return int(s)


def directions(n: int, seed: int) -> np.ndarray:
    """[n][3] float32 directions uniform on S^2 (float64 construction, float32 storage)."""
    u = SplitMix64(seed).uniform(2 * n).reshape(n, 2)
    z = 2.0 * u[:, 0] - 1.0
    phi = 2.0 * math.pi * u[:, 1]
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    out = np.empty((n, 3), dtype=np.float32)
    out[:, 0] = rxy * np.cos(phi)
    out[:, 1] = rxy * np.sin(phi)
    out[:, 2] = z
    return out


def directions_chunked(n: int, seed: int, chunk: int = 1 << 24):
    """Yield (start, [m][3] float32) chunks of ``directions(n, seed)``; identical bytes."""
    st = SplitMix64(seed)
    start = 0
    while start < n:
        m = min(chunk, n - start)
        u = st.uniform(2 * m).reshape(m, 2)
        z = 2.0 * u[:, 0] - 1.0
        phi = 2.0 * math.pi * u[:, 1]
        rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
        out = np.empty((m, 3), dtype=np.float32)
        out[:, 0] = rxy * np.cos(phi)
        out[:, 1] = rxy * np.sin(phi)
        out[:, 2] = z
        yield start, out
        start += m


def sh_count(L: int) -> int:
    return (L + 1) * (L + 1)


def sh_coeffs(G: int, L: int, seed: int) -> np.ndarray:
    """[G][(L+1)^2] float64: c_lm = N(0,1)/(l+1)^2, c_00 += 2.5; index l*l + l + m."""
    K = sh_count(L)
    c = SplitMix64(seed).normal(G * K).reshape(G, K)
    l_of = np.array([int(math.isqrt(k)) for k in range(K)], dtype=np.float64)
    c = c / (l_of + 1.0) ** 2
    c[:, 0] += 2.5
    return c


def bump_params(n_objects: int, seed: int, count_range=(8, 64),
                amp_range=(-0.2, 0.2), width_range=(0.05, 0.4)):
    """Gaussian-bump parameters for ``n_objects`` star-shaped objects.

    Returns (counts[n] int32, offsets[n+1] int64, mu[B][3] f64, amp[B] f64, width[B] f64)
    where the bumps of object o are rows offsets[o]:offsets[o+1].
    """
    st = SplitMix64(seed)
    counts = st.integers(n_objects, count_range[0], count_range[1]).astype(np.int32)
    offsets = np.zeros(n_objects + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(counts)
    B = int(offsets[-1])
    mu = directions(B, sub_seed(seed, 1)).astype(np.float64)
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    u = SplitMix64(sub_seed(seed, 2)).uniform(2 * B).reshape(B, 2)
    amp = amp_range[0] + (amp_range[1] - amp_range[0]) * u[:, 0]
    width = width_range[0] + (width_range[1] - width_range[0]) * u[:, 1]
    return counts, offsets, mu, amp, width


def fbm_keys(seed: int, octaves: int = 8) -> np.ndarray:
    """[octaves][3] uint32 lattice keys for the value-noise hash, one triple per octave."""
    return (SplitMix64(seed).u64(3 * octaves) >> np.uint64(32)).astype(np.uint32).reshape(octaves, 3)


def uneven_N(n_objects: int, seed: int, choices=(16, 32, 64, 128)) -> np.ndarray:
    """Per-object interior face resolution drawn uniformly from ``choices``."""
    idx = SplitMix64(seed).integers(n_objects, 0, len(choices) - 1)
    return np.asarray(choices, dtype=np.int32)[idx]


def query_glyphs_csr(G: int, per_glyph: int):
    """CSR segments for ``per_glyph`` contiguous queries per glyph: seg[G+1] int64."""
    return (np.arange(G + 1, dtype=np.int64) * per_glyph)


def random_glyph_ids(Q: int, G: int, seed: int) -> np.ndarray:
    return SplitMix64(seed).integers(Q, 0, G - 1).astype(np.int32)
