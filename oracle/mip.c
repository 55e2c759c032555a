/*
 * Oracle (test infrastructure only): mip levels of a Spherical Hermite Map (§4.7, Table lod).
 *
 * Derivative-consistent level (the paper: filter the scalar field, then recompute the derivative
 * channels from the filtered values by finite differences in (u,v)).  Reading used here: the
 * coarse table has resolution Nc = Nf/2 on the same cell-centred chart; its sample at coarse texel
 * (ic, jc) of face f (gutter and one-texel bake margin included) is the mean of the fine table's
 * interpolated radius (query.c) at the four fine texel centres the coarse texel covers, fine
 * indices 2ic-1, 2ic along u and 2jc-1, 2jc along v (children outside the face are directions on
 * a neighbouring face, served by that face); the records then follow from the central-difference
 * bake of bake.c.
 * Naive level (hardware mipmapping of all four RGBA channels, the paper's comparison): each coarse
 * record is the mean of its four fine child records, indices clamped to the padded fine face.
 */
#include <math.h>
#include <stdlib.h>
#include "oracle.h"

/* Direction a + X b + Y c of fine texel (i, j) of face f with X = 2u_i - 1 = (2i - 1 - N)/N formed
 * from the integer numerator: near cube corners two children sit exactly on a cube edge
 * (|X| = |Y|), and the face choice there must see the exact tie (ties -> lowest axis, §3.2
 * reading), which 2 * ((i - 1/2)/N) - 1 can break by one rounding. */
static void child_dir(int f, int i, int j, int N, double wt[3])
{
    double a[3], b[3], c[3];
    shmo_face_frame(f, a, b, c);
    const double X = (double)(2 * i - 1 - N) / (double)N, Y = (double)(2 * j - 1 - N) / (double)N;
    for (int q = 0; q < 3; ++q) wt[q] = a[q] + X * b[q] + Y * c[q];
}

void shmo_mip_samples(const double* fine, int Nf, double r0, double* samples)
{
    int Nc = Nf / 2, S = Nc + 4;
    for (int f = 0; f < 6; ++f)
        for (int jj = 0; jj < S; ++jj)
            for (int ii = 0; ii < S; ++ii) {
                int ic = ii - 1, jc = jj - 1;
                double acc = 0.0;
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) {
                        int i_f = 2 * ic - 1 + a, j_f = 2 * jc - 1 + b;
                        double wt[3];
                        child_dir(f, i_f, j_f, Nf, wt);
                        shmo_query_out o;
                        shmo_query_one(fine, Nf, r0, wt, &o);
                        acc += o.R;
                    }
                samples[((size_t)f * S + jj) * S + ii] = acc / 4.0;
            }
}

void shmo_mip_naive(const double* fine, int Nf, double* coarse)
{
    int Nc = Nf / 2, Pf = Nf + 2, Pc = Nc + 2;
    for (int f = 0; f < 6; ++f)
        for (int jc = 0; jc < Pc; ++jc)
            for (int ic = 0; ic < Pc; ++ic)
                for (int ch = 0; ch < 4; ++ch) {
                    double acc = 0.0;
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a) {
                            int i_f = 2 * ic - 1 + a, j_f = 2 * jc - 1 + b;
                            if (i_f < 0) i_f = 0;
                            if (j_f < 0) j_f = 0;
                            if (i_f > Pf - 1) i_f = Pf - 1;
                            if (j_f > Pf - 1) j_f = Pf - 1;
                            acc += fine[(((size_t)f * Pf + j_f) * Pf + i_f) * 4 + ch];
                        }
                    coarse[(((size_t)f * Pc + jc) * Pc + ic) * 4 + ch] = acc / 4.0;
                }
}
