/*
 * cube_oracle.c -- plain, slow, single-threaded CPU oracle of cube-map
 * texture sampling and of its texture gradient: the second workload of the
 * gradient-accumulation study, NvDiffRec's learning of a specular cube map
 * from rendered images (Sec. VI, "Workloads").  Each pixel samples the cube
 * map in its reflection direction; the backward adds the pixel's upstream
 * gradient, weighted by the bilinear tap weights, into the gradient of the
 * four texels it read.  Neighbouring pixels read overlapping texels, so the
 * accumulation is the contended scatter-add the paper studies, with
 * destinations that differ between the lanes of a warp (Sec. V-A1).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU legs load this library.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Definitions (the paper relies on NvDiffRec for them; the conventions are
 * OpenGL's cube-map conventions):
 *   - face: the major axis of d (|x| >= |y| and |x| >= |z| -> x; else
 *     |y| >= |z| -> y; else z), positive when that component is >= 0;
 *     faces +x, -x, +y, -y, +z, -z are 0..5;
 *   - (sc, tc) and ma per face: +x (-z, -y, |x|), -x (+z, -y, |x|),
 *     +y (+x, +z, |y|), -y (+x, -z, |y|), +z (+x, -y, |z|), -z (-x, -y, |z|);
 *     s = (sc / ma + 1) / 2, t = (tc / ma + 1) / 2;
 *   - bilinear filtering at texel centres: u = s R - 1/2, v = t R - 1/2,
 *     taps (floor u + {0,1}, floor v + {0,1}) clamped to the face, weights
 *     (1 - fu)(1 - fv), fu (1 - fv), (1 - fu) fv, fu fv with fu = u - floor u;
 *   - a zero direction is a pixel without a sample (output 0, no gradient).
 * Precision reading: the texel coordinates decide which texels a pixel
 * touches (integers), so they are computed in FP32 with exactly the IEEE
 * operations listed above, in that order (division, add, multiply by 1/2,
 * multiply by R, subtract 1/2, floor, subtract); the kernels do the same.
 * Weights and all sums are FP64.
 * Texture layout: [6][R][R][4] floats (texel (face, row v, column u); RGB
 * and one unused channel); gradients [6][R][R][3] here.
 *
 * Pins (CPU tests): face = major axis by brute force; axis directions hit
 * the face centre; coordinates are the central projection onto the face
 * (each of s, t is +-1/2 of one minor component over the major one);
 * constant textures sample exactly; a worked example on face +x; the
 * backward equals the exact difference quotient of the forward; the
 * gradient sum rule.  Parity unpinned: which sign and which minor axis each
 * face gives to s and t (the OpenGL table above).  Any consistent choice is
 * an equally valid cube map; nothing independent of the table fixes it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int face;
    int tx[4], ty[4];  /* tap texels (column, row) */
    double w[4];       /* tap weights */
} cube_taps_t;

/* Returns 0 for a zero direction (no sample). */
static int cube_taps(float dx, float dy, float dz, int R, cube_taps_t* out) {
    const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    float sc, tc, ma;
    int face;
    if (ax >= ay && ax >= az) {
        ma = ax;
        face = dx >= 0.0f ? 0 : 1;
        sc = dx >= 0.0f ? -dz : dz;
        tc = -dy;
    } else if (ay >= az) {
        ma = ay;
        face = dy >= 0.0f ? 2 : 3;
        sc = dx;
        tc = dy >= 0.0f ? dz : -dz;
    } else {
        ma = az;
        face = dz >= 0.0f ? 4 : 5;
        sc = dz >= 0.0f ? dx : -dx;
        tc = -dy;
    }
    if (!(ma > 0.0f)) return 0;
    /* FP32, one rounding per operation (volatile keeps each step a float) */
    volatile float qs = sc / ma, qt = tc / ma;
    volatile float s1 = qs + 1.0f, t1 = qt + 1.0f;
    volatile float ss = s1 * 0.5f, tt = t1 * 0.5f;
    volatile float su = ss * (float)R, tv = tt * (float)R;
    volatile float u = su - 0.5f, v = tv - 0.5f;
    const float fu0 = floorf(u), fv0 = floorf(v);
    const float fu = u - fu0, fv = v - fv0;
    const int x0 = (int)fu0, y0 = (int)fv0;
    for (int k = 0; k < 4; ++k) {
        int x = x0 + (k & 1), y = y0 + (k >> 1);
        out->tx[k] = x < 0 ? 0 : (x > R - 1 ? R - 1 : x);
        out->ty[k] = y < 0 ? 0 : (y > R - 1 ? R - 1 : y);
    }
    const double a = (double)fu, b = (double)fv;
    out->w[0] = (1.0 - a) * (1.0 - b);
    out->w[1] = a * (1.0 - b);
    out->w[2] = (1.0 - a) * b;
    out->w[3] = a * b;
    out->face = face;
    return 1;
}

/* Per direction: face (-1 without a sample), the 4 tap texels as linear
 * texel indices face*R*R + row*R + column, and their weights. */
void orc_cube_taps(long long n, const float* dirs, int R, int* face, long long* texel, double* w) {
    for (long long i = 0; i < n; ++i) {
        cube_taps_t t;
        if (!cube_taps(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], R, &t)) {
            face[i] = -1;
            for (int k = 0; k < 4; ++k) {
                texel[4 * i + k] = -1;
                w[4 * i + k] = 0.0;
            }
            continue;
        }
        face[i] = t.face;
        for (int k = 0; k < 4; ++k) {
            texel[4 * i + k] = ((long long)t.face * R + t.ty[k]) * R + t.tx[k];
            w[4 * i + k] = t.w[k];
        }
    }
}

/* out[i][c] = sum_k w_k tex[tap_k][c]; scale[i][c] = sum_k |w_k tex[tap_k][c]|. */
void orc_cube_forward(long long n, const float* dirs, int R, const float* tex, double* out, double* scale) {
    for (long long i = 0; i < n; ++i) {
        cube_taps_t t;
        for (int c = 0; c < 3; ++c) {
            out[3 * i + c] = 0.0;
            scale[3 * i + c] = 0.0;
        }
        if (!cube_taps(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], R, &t)) continue;
        for (int k = 0; k < 4; ++k) {
            const float* tx = tex + 4 * (((size_t)t.face * R + t.ty[k]) * R + t.tx[k]);
            for (int c = 0; c < 3; ++c) {
                const double term = t.w[k] * (double)tx[c];
                out[3 * i + c] += term;
                scale[3 * i + c] += fabs(term);
            }
        }
    }
}

/* grad[texel][c] += sum over pixels and taps of w_k dL[i][c] (grad [6][R][R][3],
 * not cleared); gscale[texel][c] += the absolute values of the terms. */
void orc_cube_backward(long long n, const float* dirs, const float* dL, int R, double* grad, double* gscale) {
    for (long long i = 0; i < n; ++i) {
        cube_taps_t t;
        if (!cube_taps(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], R, &t)) continue;
        for (int k = 0; k < 4; ++k) {
            const size_t o = 3 * (((size_t)t.face * R + t.ty[k]) * R + t.tx[k]);
            for (int c = 0; c < 3; ++c) {
                const double term = t.w[k] * (double)dL[3 * i + c];
                grad[o + c] += term;
                gscale[o + c] += fabs(term);
            }
        }
    }
}
