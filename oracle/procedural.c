/*
 * Oracle (test infrastructure only): synthetic radial functions standing in for the paper's
 * application scenes (§4.9 radial depth-map impostors, §4.10 procedural planets), whose
 * meshes and terrain recipes are not published.
 *
 * Gaussian bumps: R(w) = 1 + sum_k a_k exp(-|w - mu_k|^2 / (2 w_k^2)).  For unit vectors
 *   |w - mu|^2 / 2 = 1 - w.mu, so this is the "width w_k radians" bump exp(-(1 - w.mu)/w_k^2),
 *   written in the chord form that stays accurate when w is close to mu.
 * Value-noise fBm (§4.10 names Perlin/Simplex/fBm; the octave noise is not specified):
 *   lattice values from the PCG3D hash (Jarzynski & Olano, "Hash Functions for GPU Rendering",
 *   JCGT 9(3), 2020) of the integer lattice point plus a per-octave key, mapped to [-1, 1);
 *   quintic fade 6t^5 - 15t^4 + 10t^3; trilinear blend; fBm = sum_o gain^o noise(w f0 lac^o).
 */
#include <math.h>
#include "oracle.h"

double shmo_bumps(const double w[3], int nb, const double* mu, const double* amp, const double* width)
{
    double r = 1.0;
    for (int k = 0; k < nb; ++k) {
        double dx = w[0] - mu[3 * k], dy = w[1] - mu[3 * k + 1], dz = w[2] - mu[3 * k + 2];
        double chord2 = dx * dx + dy * dy + dz * dz;
        r += amp[k] * exp(-chord2 / (2.0 * width[k] * width[k]));
    }
    return r;
}

void shmo_pcg3d(uint32_t v[3])
{
    for (int q = 0; q < 3; ++q) v[q] = v[q] * 1664525u + 1013904223u;
    v[0] += v[1] * v[2];
    v[1] += v[2] * v[0];
    v[2] += v[0] * v[1];
    for (int q = 0; q < 3; ++q) v[q] ^= v[q] >> 16;
    v[0] += v[1] * v[2];
    v[1] += v[2] * v[0];
    v[2] += v[0] * v[1];
}

static double lattice(int64_t ix, int64_t iy, int64_t iz, const uint32_t key[3])
{
    uint32_t v[3] = {(uint32_t)ix + key[0], (uint32_t)iy + key[1], (uint32_t)iz + key[2]};
    shmo_pcg3d(v);
    return (double)(v[0] >> 8) * (2.0 / 16777216.0) - 1.0;
}

static double fade(double t) { return t * t * t * (t * (t * 6.0 - 15.0) + 10.0); }

double shmo_value_noise(const double p[3], const uint32_t key[3])
{
    double fl[3], w[3];
    int64_t i0[3];
    for (int q = 0; q < 3; ++q) {
        fl[q] = floor(p[q]);
        i0[q] = (int64_t)fl[q];
        w[q] = fade(p[q] - fl[q]);
    }
    double acc = 0.0;
    for (int c = 0; c < 8; ++c) {
        int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        double wt = (dx ? w[0] : 1.0 - w[0]) * (dy ? w[1] : 1.0 - w[1]) * (dz ? w[2] : 1.0 - w[2]);
        acc += wt * lattice(i0[0] + dx, i0[1] + dy, i0[2] + dz, key);
    }
    return acc;
}

double shmo_fbm(const double w[3], int octaves, const uint32_t* keys, double base_freq,
                double lacunarity, double gain)
{
    double sum = 0.0, freq = base_freq, ampl = 1.0;
    for (int o = 0; o < octaves; ++o) {
        double p[3] = {w[0] * freq, w[1] * freq, w[2] * freq};
        sum += ampl * shmo_value_noise(p, keys + 3 * o);
        freq *= lacunarity;
        ampl *= gain;
    }
    return sum;
}
