/*
 * gsr_oracle.c -- plain, slow, single-threaded FP64 CPU oracle of the
 * tile-based Gaussian-splat rasterizer whose backward pass the paper studies.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg load this library.  It shares no code, header, table or
 * constant generator with the CUDA library: every formula below is written out
 * independently from its definition.
 *
 * What the paper fixes (DISTWAR, arXiv 2401.05345):
 *   - the gradient computation step: one thread per pixel iterates the
 *     pixel's list of primitives, skips primitives that fail per-pixel
 *     conditions, computes the gradient of every parameter of each remaining
 *     primitive and accumulates it into the primitive's gradient buffer
 *     (Sec. III-A, Fig. "Outline of the gradient computation step");
 *   - warp-level reduction only changes WHERE the per-primitive sum is formed,
 *     never its value (Sec. V-A1/V-A2: the reduction routine directly replaces
 *     the atomic adds).  Hence the oracle is the plain definition of the
 *     rendered image and of its exact gradient, summed in FP64.
 * What the paper leaves to the 3DGS rasterizer it evaluates (Sec. VI,
 * "Workloads"; Sec. II-C): projection, EWA covariance, SH colour, tile binning
 * and front-to-back alpha compositing.  Those are written out here from their
 * mathematical definitions with the 3DGS constants (near plane 0.2, screen-
 * space dilation 0.3, 3-sigma radius, eigenvalue floor 0.1, frustum clamp 1.3,
 * alpha cap 0.99, alpha floor 1/255, transmittance stop 1e-4, SH offset 0.5).
 * Constants that the rasterizer stores as FP32 are taken at their FP32 value.
 *
 * Precision readings: the oracle computes in FP64 on inputs given as FP32
 * values.  Where a floating-point comparison decides a discrete outcome (skip,
 * stop, clamp, radius ceiling), the FP32 kernel may legitimately decide the
 * other way when the FP64 value lies within the FP32 rounding error of the
 * boundary.  The oracle detects those decisions from a first-order FP32 error
 * bound, re-evaluates the pixel with the decision flipped and reports the
 * difference as an allowance: both outcomes are valid results.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define F32(x) ((double)(float)(x))
static const double EPS32 = 5.9604644775390625e-08; /* 2^-24, FP32 unit roundoff */

/* 3DGS rasterizer constants (FP32 values). */
#define K_DILATION  F32(0.3)
#define K_ALPHA_MAX F32(0.99)
#define K_ALPHA_MIN ((double)(1.0f / 255.0f))
#define K_T_MIN     F32(0.0001)
#define K_FRUSTUM   F32(1.3)
#define K_LAMBDA_FLOOR F32(0.1)
#define K_SH_OFFSET 0.5
#define AMBIG_SAFETY 8.0

typedef struct {
    int width, height;
    double view[12];        /* row-major [R | t], world -> camera */
    double fx, fy, cx, cy;
    double tan_fovx, tan_fovy;
    double campos[3];
    double znear;
} orc_camera;

/* ------------------------------------------------------------------ */
/* integer helpers                                                     */
/* ------------------------------------------------------------------ */
static long long floordiv_ll(long long a, long long b) {
    long long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q -= 1;
    return q;
}
static long long clamp_ll(long long x, long long lo, long long hi) {
    return x < lo ? lo : (x > hi ? hi : x);
}

/* Tile rectangle [x0,x1) x [y0,y1) touched by a splat of integer radius r
 * centred at (u,v): the 3DGS bounding-box rule, written with floor(u) so the
 * result is exact integer arithmetic.  Returns the number of tiles. */
static long long tile_rect(double u, double v, int r, int W, int H, int tw, int th,
                           long long* x0, long long* x1, long long* y0, long long* y1) {
    long long gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    long long fu = (long long)floor(u), fv = (long long)floor(v);
    *x0 = clamp_ll(floordiv_ll(fu - r, tw), 0, gx);
    *x1 = clamp_ll(floordiv_ll(fu + r + tw - 1, tw), 0, gx);
    *y0 = clamp_ll(floordiv_ll(fv - r, th), 0, gy);
    *y1 = clamp_ll(floordiv_ll(fv + r + th - 1, th), 0, gy);
    long long n = (*x1 - *x0) * (*y1 - *y0);
    return n > 0 ? n : 0;
}

/* ------------------------------------------------------------------ */
/* real spherical harmonics up to degree 3 (3DGS sign convention)       */
/* ------------------------------------------------------------------ */
/* Normalisation constants of the orthonormal real SH basis, from
 * N_lm = sqrt((2l+1)/(4 pi) * (l-|m|)!/(l+|m|)!) times the polynomial factor. */
static void sh_consts(double c[16]) {
    const double pi = 3.14159265358979323846;
    const double rpi = sqrt(pi);
    c[0] = 1.0 / (2.0 * rpi);
    c[1] = sqrt(3.0) / (2.0 * rpi);
    c[2] = sqrt(15.0) / (2.0 * rpi);     /* xy, yz, xz */
    c[3] = sqrt(5.0) / (4.0 * rpi);      /* 2z^2 - x^2 - y^2 */
    c[4] = sqrt(15.0) / (4.0 * rpi);     /* x^2 - y^2 */
    c[5] = sqrt(35.0 / 2.0) / (4.0 * rpi); /* y(3x^2-y^2), x(x^2-3y^2) */
    c[6] = sqrt(105.0) / (2.0 * rpi);    /* xyz */
    c[7] = sqrt(21.0 / 2.0) / (4.0 * rpi); /* y(4z^2-x^2-y^2), x(4z^2-x^2-y^2) */
    c[8] = sqrt(7.0) / (4.0 * rpi);      /* z(2z^2-3x^2-3y^2) */
    c[9] = sqrt(105.0) / (4.0 * rpi);    /* z(x^2-y^2) */
}

/* Basis values Y[0..(deg+1)^2) and, if dY != NULL, their gradients
 * dY[k*3 + {0,1,2}] with respect to (x,y,z) treated as free variables. */
static void sh_eval(int deg, const double d[3], double* Y, double* dY) {
    double c[16];
    sh_consts(c);
    const double x = d[0], y = d[1], z = d[2];
    int n = (deg + 1) * (deg + 1);
    double g[16][3];
    memset(g, 0, sizeof(g));
    Y[0] = c[0];
    if (deg >= 1) {
        Y[1] = -c[1] * y;  g[1][1] = -c[1];
        Y[2] = c[1] * z;   g[2][2] = c[1];
        Y[3] = -c[1] * x;  g[3][0] = -c[1];
    }
    if (deg >= 2) {
        Y[4] = c[2] * x * y;    g[4][0] = c[2] * y; g[4][1] = c[2] * x;
        Y[5] = -c[2] * y * z;   g[5][1] = -c[2] * z; g[5][2] = -c[2] * y;
        Y[6] = c[3] * (2 * z * z - x * x - y * y);
        g[6][0] = -2 * c[3] * x; g[6][1] = -2 * c[3] * y; g[6][2] = 4 * c[3] * z;
        Y[7] = -c[2] * x * z;   g[7][0] = -c[2] * z; g[7][2] = -c[2] * x;
        Y[8] = c[4] * (x * x - y * y);
        g[8][0] = 2 * c[4] * x; g[8][1] = -2 * c[4] * y;
    }
    if (deg >= 3) {
        Y[9] = -c[5] * y * (3 * x * x - y * y);
        g[9][0] = -c[5] * 6 * x * y; g[9][1] = -c[5] * (3 * x * x - 3 * y * y);
        Y[10] = c[6] * x * y * z;
        g[10][0] = c[6] * y * z; g[10][1] = c[6] * x * z; g[10][2] = c[6] * x * y;
        Y[11] = -c[7] * y * (4 * z * z - x * x - y * y);
        g[11][0] = -c[7] * y * (-2 * x); g[11][1] = -c[7] * (4 * z * z - x * x - 3 * y * y);
        g[11][2] = -c[7] * y * 8 * z;
        Y[12] = c[8] * z * (2 * z * z - 3 * x * x - 3 * y * y);
        g[12][0] = c[8] * z * (-6 * x); g[12][1] = c[8] * z * (-6 * y);
        g[12][2] = c[8] * (6 * z * z - 3 * x * x - 3 * y * y);
        Y[13] = -c[7] * x * (4 * z * z - x * x - y * y);
        g[13][0] = -c[7] * (4 * z * z - 3 * x * x - y * y); g[13][1] = -c[7] * x * (-2 * y);
        g[13][2] = -c[7] * x * 8 * z;
        Y[14] = c[9] * z * (x * x - y * y);
        g[14][0] = c[9] * z * 2 * x; g[14][1] = -c[9] * z * 2 * y; g[14][2] = c[9] * (x * x - y * y);
        Y[15] = -c[5] * x * (x * x - 3 * y * y);
        g[15][0] = -c[5] * (3 * x * x - 3 * y * y); g[15][1] = -c[5] * x * (-6 * y);
    }
    if (dY)
        for (int k = 0; k < n; ++k)
            for (int a = 0; a < 3; ++a) dY[k * 3 + a] = g[k][a];
}

void orc_sh_basis(int deg, const double* dir, double* out) { sh_eval(deg, dir, out, NULL); }
void orc_sh_basis_grad(int deg, const double* dir, double* out) {
    double Y[16];
    sh_eval(deg, dir, Y, out);
}

/* ------------------------------------------------------------------ */
/* per-Gaussian projection (forward quantities)                         */
/* ------------------------------------------------------------------ */
typedef struct {
    int culled;            /* 1: behind the near plane, degenerate, or off-screen */
    double p[3];           /* camera-space mean */
    double qn[4], qnorm;   /* normalised quaternion (w,x,y,z) and |q| */
    double R[9];           /* rotation of qn */
    double M[9];           /* R diag(s) */
    double S3[9];          /* 3D covariance M M^T */
    double tx, ty;         /* x/z and y/z after the frustum clamp */
    int clx, cly;          /* 1 where the clamp is active */
    double J[6];           /* 2x3 Jacobian of the projection */
    double Tm[6];          /* J W (W = camera rotation) */
    double a, b, c;        /* 2D covariance after dilation: [[a,b],[b,c]] */
    double det;
    double conic[3];       /* (A,B,C): inverse covariance [[A,B],[B,C]] */
    double u, v;
    double radius_real;    /* 3 sqrt(lambda_max) */
    int radius;
    double dir[3], dist;   /* view direction of the SH colour */
    double raw[3];         /* SH sum + 0.5 before the clamp at zero */
    double rgb[3];
    int pp_ambig;          /* an integer output may legitimately differ in FP32 */
    int bp_ambig;          /* a derivative branch may legitimately differ in FP32 */
} gauss_t;

static void quat_to_rot(const double q[4], double R[9]) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

static void project_one(const orc_camera* cam, int sh_deg, const double* mean, const double* scale,
                        const double* quat, const double* feat, int tw, int th, gauss_t* G) {
    memset(G, 0, sizeof(*G));
    const double* V = cam->view;
    double pabs = 0.0;
    for (int i = 0; i < 3; ++i) {
        G->p[i] = V[4 * i] * mean[0] + V[4 * i + 1] * mean[1] + V[4 * i + 2] * mean[2] + V[4 * i + 3];
        if (i == 2)
            pabs = fabs(V[8] * mean[0]) + fabs(V[9] * mean[1]) + fabs(V[10] * mean[2]) + fabs(V[11]);
    }
    const double z = G->p[2];
    /* near-plane cull */
    double ez = 4.0 * EPS32 * pabs;
    if (fabs(z - cam->znear) <= AMBIG_SAFETY * ez) G->pp_ambig = 1;
    if (z <= cam->znear) { G->culled = 1; return; }

    /* rotation and 3D covariance, Sigma = R S S^T R^T */
    double qn2 = quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3];
    G->qnorm = sqrt(qn2);
    for (int i = 0; i < 4; ++i) G->qn[i] = quat[i] / G->qnorm;
    quat_to_rot(G->qn, G->R);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) G->M[3 * i + j] = G->R[3 * i + j] * scale[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += G->M[3 * i + k] * G->M[3 * j + k];
            G->S3[3 * i + j] = s;
        }

    /* local affine approximation of the projection (EWA splatting) */
    const double limx = K_FRUSTUM * cam->tan_fovx, limy = K_FRUSTUM * cam->tan_fovy;
    double xz = G->p[0] / z, yz = G->p[1] / z;
    G->clx = (xz < -limx || xz > limx);
    G->cly = (yz < -limy || yz > limy);
    if (fabs(fabs(xz) - limx) <= AMBIG_SAFETY * 8.0 * EPS32 * limx) G->bp_ambig = 1;
    if (fabs(fabs(yz) - limy) <= AMBIG_SAFETY * 8.0 * EPS32 * limy) G->bp_ambig = 1;
    G->tx = xz < -limx ? -limx : (xz > limx ? limx : xz);
    G->ty = yz < -limy ? -limy : (yz > limy ? limy : yz);
    const double fx = cam->fx, fy = cam->fy;
    G->J[0] = fx / z; G->J[1] = 0.0; G->J[2] = -fx * G->tx / z;
    G->J[3] = 0.0;    G->J[4] = fy / z; G->J[5] = -fy * G->ty / z;
    for (int r = 0; r < 2; ++r)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += G->J[3 * r + k] * V[4 * k + j];
            G->Tm[3 * r + j] = s;
        }
    double S2[4];
    for (int r = 0; r < 2; ++r)
        for (int q = 0; q < 2; ++q) {
            double s = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) s += G->Tm[3 * r + i] * G->S3[3 * i + j] * G->Tm[3 * q + j];
            S2[2 * r + q] = s;
        }
    G->a = S2[0] + K_DILATION;
    G->b = S2[1];
    G->c = S2[3] + K_DILATION;
    G->det = G->a * G->c - G->b * G->b;
    if (G->det <= 0.0) { G->culled = 1; return; }
    G->conic[0] = G->c / G->det;
    G->conic[1] = -G->b / G->det;
    G->conic[2] = G->a / G->det;

    /* screen position: pixel centres at integer coordinates */
    G->u = fx * G->p[0] / z + cam->cx;
    G->v = fy * G->p[1] / z + cam->cy;

    /* 3-sigma radius of the larger eigenvalue */
    double mid = 0.5 * (G->a + G->c);
    double disc = mid * mid - G->det;
    double dfl = disc > K_LAMBDA_FLOOR ? disc : K_LAMBDA_FLOOR;
    double lam = mid + sqrt(dfl);
    G->radius_real = 3.0 * sqrt(lam);
    G->radius = (int)ceil(G->radius_real);
    {
        /* FP32 error of lambda: cancellation in mid^2 - det, then the sqrt */
        double e_lam = EPS32 * (16.0 + 4.0 * mid * mid / (sqrt(dfl) * lam));
        double e_r = 0.5 * e_lam + 4.0 * EPS32;
        double fr = G->radius_real - floor(G->radius_real);
        double dist_int = fr < 0.5 ? fr : 1.0 - fr;
        if (dist_int <= AMBIG_SAFETY * e_r * G->radius_real) G->pp_ambig = 1;
    }
    /* off-screen cull on the tile rectangle; floor(u) may differ in FP32 */
    long long x0, x1, y0, y1;
    long long nt = tile_rect(G->u, G->v, G->radius, cam->width, cam->height, tw, th, &x0, &x1, &y0, &y1);
    {
        double eu = 8.0 * EPS32 * (fabs(fx * G->p[0] / z) + fabs(cam->cx) + 1.0);
        double ev = 8.0 * EPS32 * (fabs(fy * G->p[1] / z) + fabs(cam->cy) + 1.0);
        double fu = G->u - floor(G->u), fv = G->v - floor(G->v);
        int near_u = (fu <= AMBIG_SAFETY * eu) || (1.0 - fu <= AMBIG_SAFETY * eu);
        int near_v = (fv <= AMBIG_SAFETY * ev) || (1.0 - fv <= AMBIG_SAFETY * ev);
        if (near_u || near_v) {
            for (int du = -1; du <= 1; ++du)
                for (int dv = -1; dv <= 1; ++dv) {
                    if ((du && !near_u) || (dv && !near_v)) continue;
                    long long a0, a1, b0, b1;
                    long long n2 = tile_rect(G->u + du, G->v + dv, G->radius, cam->width, cam->height,
                                             tw, th, &a0, &a1, &b0, &b1);
                    if ((n2 == 0) != (nt == 0)) G->pp_ambig = 1;
                }
        }
    }
    if (nt == 0) { G->culled = 1; return; }

    /* colour: SH evaluated along the viewing direction, +0.5, clamped at 0 */
    double d[3];
    for (int i = 0; i < 3; ++i) d[i] = mean[i] - cam->campos[i];
    G->dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int i = 0; i < 3; ++i) G->dir[i] = d[i] / G->dist;
    if (sh_deg < 0) {
        for (int ch = 0; ch < 3; ++ch) { G->raw[ch] = feat[ch]; G->rgb[ch] = feat[ch]; }
    } else {
        double Y[16];
        sh_eval(sh_deg, G->dir, Y, NULL);
        int K = (sh_deg + 1) * (sh_deg + 1);
        for (int ch = 0; ch < 3; ++ch) {
            double s = 0, sabs = 0;
            for (int k = 0; k < K; ++k) { s += Y[k] * feat[3 * k + ch]; sabs += fabs(Y[k] * feat[3 * k + ch]); }
            G->raw[ch] = s + K_SH_OFFSET;
            G->rgb[ch] = G->raw[ch] > 0.0 ? G->raw[ch] : 0.0;
            if (fabs(G->raw[ch]) <= AMBIG_SAFETY * 16.0 * EPS32 * (sabs + 0.5)) G->bp_ambig = 1;
        }
    }
}

/* Projection of N Gaussians (3DGS "preprocess").  Culled Gaussians get
 * radius 0 and zeros elsewhere.  sh_deg = -1: feat holds RGB colours [N,3];
 * otherwise SH coefficients [N,(deg+1)^2,3].  Returns the number visible. */
int orc_preprocess(int N, int sh_deg, const double* mean, const double* scale, const double* quat,
                   const double* opacity, const double* feat, const orc_camera* cam, int tw, int th,
                   double* uv, double* conic, double* rgb, double* depth, int* radius,
                   int* pp_ambig, int* bp_ambig) {
    int K = sh_deg < 0 ? 1 : (sh_deg + 1) * (sh_deg + 1);
    int visible = 0;
    (void)opacity;
    for (int i = 0; i < N; ++i) {
        gauss_t G;
        project_one(cam, sh_deg, mean + 3 * i, scale + 3 * i, quat + 4 * i, feat + 3 * K * i, tw, th, &G);
        if (pp_ambig) pp_ambig[i] = G.pp_ambig;
        if (bp_ambig) bp_ambig[i] = G.bp_ambig;
        if (G.culled) {
            uv[2 * i] = uv[2 * i + 1] = 0;
            conic[3 * i] = conic[3 * i + 1] = conic[3 * i + 2] = 0;
            rgb[3 * i] = rgb[3 * i + 1] = rgb[3 * i + 2] = 0;
            depth[i] = 0;
            radius[i] = 0;
            continue;
        }
        ++visible;
        uv[2 * i] = G.u; uv[2 * i + 1] = G.v;
        for (int k = 0; k < 3; ++k) { conic[3 * i + k] = G.conic[k]; rgb[3 * i + k] = G.rgb[k]; }
        depth[i] = G.p[2];
        radius[i] = G.radius;
    }
    return visible;
}

/* ------------------------------------------------------------------ */
/* tile binning: keys, stable sort, per-tile ranges                     */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t key; uint64_t order; uint32_t val; } kv_t;
static int kv_cmp(const void* pa, const void* pb) {
    const kv_t* a = (const kv_t*)pa; const kv_t* b = (const kv_t*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->order != b->order) return a->order < b->order ? -1 : 1;
    return 0;
}

static uint32_t f32_bits(double x) {
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* Number of (tile, Gaussian) entries: the duplicated key count. */
long long orc_bin_count(int N, const double* uv, const int* radius, int W, int H, int tw, int th) {
    long long total = 0;
    for (int i = 0; i < N; ++i) {
        if (radius[i] <= 0) continue;
        long long x0, x1, y0, y1;
        total += tile_rect(uv[2 * i], uv[2 * i + 1], radius[i], W, H, tw, th, &x0, &x1, &y0, &y1);
    }
    return total;
}

/* Keys (tile_id << 32 | FP32 bits of depth) emitted per Gaussian in id order,
 * tiles row-major inside each rectangle; sorted stably (ties keep emission
 * order, i.e. Gaussian id); ranges[2t], ranges[2t+1] = [start, end) of tile t
 * in the sorted list, 0,0 for empty tiles.  keys/vals sized orc_bin_count. */
int orc_bin(int N, const double* uv, const double* depth, const int* radius, int W, int H, int tw,
            int th, uint64_t* keys, uint32_t* vals, uint32_t* ranges) {
    long long n = orc_bin_count(N, uv, radius, W, H, tw, th);
    long long gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    kv_t* buf = (kv_t*)malloc(sizeof(kv_t) * (size_t)(n > 0 ? n : 1));
    if (!buf) return -1;
    long long w = 0;
    for (int i = 0; i < N; ++i) {
        if (radius[i] <= 0) continue;
        long long x0, x1, y0, y1;
        tile_rect(uv[2 * i], uv[2 * i + 1], radius[i], W, H, tw, th, &x0, &x1, &y0, &y1);
        for (long long y = y0; y < y1; ++y)
            for (long long x = x0; x < x1; ++x) {
                uint64_t tile = (uint64_t)(y * gx + x);
                buf[w].key = (tile << 32) | (uint64_t)f32_bits(depth[i]);
                buf[w].order = (uint64_t)w;
                buf[w].val = (uint32_t)i;
                ++w;
            }
    }
    qsort(buf, (size_t)n, sizeof(kv_t), kv_cmp);
    for (long long k = 0; k < gx * gy; ++k) ranges[2 * k] = ranges[2 * k + 1] = 0;
    for (long long k = 0; k < n; ++k) {
        keys[k] = buf[k].key;
        vals[k] = buf[k].val;
        uint32_t t = (uint32_t)(buf[k].key >> 32);
        if (k == 0 || (uint32_t)(buf[k - 1].key >> 32) != t) ranges[2 * t] = (uint32_t)k;
        if (k == n - 1 || (uint32_t)(buf[k + 1].key >> 32) != t) ranges[2 * t + 1] = (uint32_t)(k + 1);
    }
    free(buf);
    return 0;
}

/* ------------------------------------------------------------------ */
/* per-pixel compositing and its exact gradient                        */
/* ------------------------------------------------------------------ */
enum { D_SIGMA = 1, D_CAP = 2, D_FLOOR = 3, D_STOP = 4 };

typedef struct {
    int pos;               /* position in the tile list */
    uint32_t id;
    double alpha, T, G, dx, dy;
    int clamped;
    double e_a;            /* FP32 relative error bound of alpha */
} contrib_t;

typedef struct { int pos, kind; } ambig_t;

typedef struct {
    int W, H;
    const double *uv, *conic, *opac, *rgb, *bg;
} scene2d_t;

/* Front-to-back walk over one pixel's list: the forward rule of the rasterizer.
 * Returns the number of contributors written to cs.  flip_pos/flip_kind force
 * the opposite outcome of one decision; amb (if not NULL) records decisions
 * whose FP64 value lies within the FP32 error bound of their boundary. */
static int walk_pixel(const scene2d_t* S, double px, double py, const uint32_t* list, int n,
                      int flip_pos, int flip_kind, contrib_t* cs, double out[3], double* T_final,
                      int* last, double* e_T_final, ambig_t* amb, int* namb) {
    double T = 1.0, eT = 0.0, C[3] = {0, 0, 0};
    int nc = 0, lst = 0;
    if (namb) *namb = 0;
    for (int k = 0; k < n; ++k) {
        uint32_t g = list[k];
        const double u = S->uv[2 * g], v = S->uv[2 * g + 1];
        const double A = S->conic[3 * g], B = S->conic[3 * g + 1], Cc = S->conic[3 * g + 2];
        const double o = S->opac[g];
        double dx = u - px, dy = v - py;
        double sA = 0.5 * A * dx * dx, sC = 0.5 * Cc * dy * dy, sB = B * dx * dy;
        double sig = sA + sC + sB;
        double ssum = fabs(sA) + fabs(sC) + fabs(sB);
        double e_sig = 6.0 * EPS32 * ssum +
                       EPS32 * (fabs(u) * fabs(A * dx + B * dy) + fabs(v) * fabs(B * dx + Cc * dy));
        int neg = sig < 0.0;
        if (flip_pos == k && flip_kind == D_SIGMA) neg = !neg;
        else if (amb && fabs(sig) < AMBIG_SAFETY * e_sig) { amb[*namb].pos = k; amb[*namb].kind = D_SIGMA; ++*namb; }
        if (neg) continue;
        double Gv = exp(-sig);
        double e_a = e_sig + 4.0 * EPS32 * (1.0 + fabs(sig)) + EPS32;
        double oG = o * Gv;
        int clamped = oG > K_ALPHA_MAX;
        if (flip_pos == k && flip_kind == D_CAP) clamped = !clamped;
        else if (amb && fabs(oG - K_ALPHA_MAX) <= AMBIG_SAFETY * e_a * K_ALPHA_MAX) { amb[*namb].pos = k; amb[*namb].kind = D_CAP; ++*namb; }
        double alpha = clamped ? K_ALPHA_MAX : oG;
        int skip = alpha < K_ALPHA_MIN;
        if (flip_pos == k && flip_kind == D_FLOOR) skip = !skip;
        else if (amb && fabs(alpha - K_ALPHA_MIN) <= AMBIG_SAFETY * e_a * alpha) { amb[*namb].pos = k; amb[*namb].kind = D_FLOOR; ++*namb; }
        if (skip) continue;
        double Tn = T * (1.0 - alpha);
        double eTn = eT + (clamped ? 0.0 : e_a * alpha / (1.0 - alpha)) + 2.0 * EPS32;
        int stop = Tn < K_T_MIN;
        if (flip_pos == k && flip_kind == D_STOP) stop = !stop;
        else if (amb && fabs(Tn - K_T_MIN) <= AMBIG_SAFETY * eTn * K_T_MIN) { amb[*namb].pos = k; amb[*namb].kind = D_STOP; ++*namb; }
        if (stop) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += S->rgb[3 * g + ch] * alpha * T;
        contrib_t* c = &cs[nc++];
        c->pos = k; c->id = g; c->alpha = alpha; c->T = T; c->G = Gv; c->dx = dx; c->dy = dy;
        c->clamped = clamped; c->e_a = clamped ? 0.0 : e_a;
        T = Tn;
        eT = eTn;
        lst = k + 1;
    }
    for (int ch = 0; ch < 3; ++ch) out[ch] = C[ch] + T * S->bg[ch];
    *T_final = T;
    *last = lst;
    if (e_T_final) *e_T_final = eT;
    return nc;
}

/* Exact gradient of one pixel's colour: for contributor j (front-to-back
 * index), with g = dL/d(pixel colour), T_j the transmittance in front of j:
 *   dL/dc_j     = alpha_j T_j g
 *   dL/dalpha_j = T_j (c_j . g) - [sum_{k>j} (c_k . g) alpha_k T_k + T_final (bg . g)] / (1 - alpha_j)
 *   alpha = o exp(-sigma) (unclamped): dL/do = G dL/dalpha, dL/dsigma = -o G dL/dalpha
 *   sigma = A dx^2/2 + B dx dy + C dy^2/2 with (dx,dy) = (u,v) - pixel
 * The 9 values per contributor are (u, v, A, B, C, o, r, g, b).  mag receives
 * the same chain evaluated on absolute values (the scale of the terms). */
static void pixel_grads(const scene2d_t* S, const contrib_t* cs, int nc, double T_final, const double g[3],
                        double* grads /* nc x 9 */, double* mags /* nc x 9 or NULL */) {
    const double* bg = S->bg;
    double Sf = T_final * (bg[0] * g[0] + bg[1] * g[1] + bg[2] * g[2]);
    double Sa = T_final * (fabs(bg[0] * g[0]) + fabs(bg[1] * g[1]) + fabs(bg[2] * g[2]));
    for (int j = nc - 1; j >= 0; --j) {
        const contrib_t* c = &cs[j];
        uint32_t id = c->id;
        const double* col = S->rgb + 3 * id;
        const double A = S->conic[3 * id], B = S->conic[3 * id + 1], Cc = S->conic[3 * id + 2];
        const double o = S->opac[id];
        double cg = col[0] * g[0] + col[1] * g[1] + col[2] * g[2];
        double cga = fabs(col[0] * g[0]) + fabs(col[1] * g[1]) + fabs(col[2] * g[2]);
        double inv = 1.0 / (1.0 - c->alpha);
        double dalpha = c->T * cg - Sf * inv;
        double malpha = c->T * cga + Sa * inv;
        Sf += cg * c->alpha * c->T;
        Sa += cga * c->alpha * c->T;
        double dopa = 0, dsig = 0, mopa = 0, msig = 0;
        if (!c->clamped) {
            dopa = c->G * dalpha;
            dsig = -o * c->G * dalpha;
            mopa = c->G * malpha;
            msig = o * c->G * malpha;
        }
        double* gr = grads + 9 * j;
        gr[0] = (A * c->dx + B * c->dy) * dsig;
        gr[1] = (B * c->dx + Cc * c->dy) * dsig;
        gr[2] = 0.5 * c->dx * c->dx * dsig;
        gr[3] = c->dx * c->dy * dsig;
        gr[4] = 0.5 * c->dy * c->dy * dsig;
        gr[5] = dopa;
        for (int ch = 0; ch < 3; ++ch) gr[6 + ch] = c->alpha * c->T * g[ch];
        if (mags) {
            double* mg = mags + 9 * j;
            mg[0] = (fabs(A * c->dx) + fabs(B * c->dy)) * msig;
            mg[1] = (fabs(B * c->dx) + fabs(Cc * c->dy)) * msig;
            mg[2] = 0.5 * c->dx * c->dx * msig;
            mg[3] = fabs(c->dx * c->dy) * msig;
            mg[4] = 0.5 * c->dy * c->dy * msig;
            mg[5] = mopa;
            for (int ch = 0; ch < 3; ++ch) mg[6 + ch] = fabs(c->alpha * c->T * g[ch]);
        }
    }
}

/*
 * Forward render and backward pass of one view, pixel by pixel (the
 * gradient-computation step of Sec. III-A; per-tile lists as in 3DGS).
 *
 * Inputs: ranges [2*tiles], point_list, 2D splat parameters (uv [N,2],
 * conic [N,3], opacity [N], rgb [N,3]) as FP64 copies of the kernel's FP32
 * inputs, bg [3], dL_dimage [3,H,W] (NULL: forward only).
 * Outputs: image [3,H,W], final_T [H*W], n_contrib [H*W] (1-based list
 * position of the last contributor, 0 if none);
 * grad2d [N,9] (u, v, A, B, C, o, r, g, b) accumulated exactly in FP64;
 * gscale [N,9]: sum over pixels of the terms' absolute chain values, widened
 *   by max(1, 8 b / 1e-5) where b is the pixel's FP32 error-bound factor
 *   (transmittance recovered through alpha near 1 amplifies FP32 rounding);
 * glit [N,9]: the same sum without widening;
 * gallow [N,9], iallow [3,H,W], tallow [H*W]: allowance from decisions that
 *   FP32 may take the other way (difference between both outcomes);
 * nc_alt [H*W]: n_contrib under the flipped decision (-1 if none);
 * pix_ambig [H*W]: count of such decisions in the pixel;
 * pix_widen [H*W]: the pixel's widening factor max(1, 8 b / 1e-5);
 * terr [H*W]: first-order FP32 relative error bound of final_T;
 * n_active [H*W]: number of contributing splats of the pixel.
 * tile_mask [tiles] (may be NULL = all): only tiles with a non-zero entry are
 * evaluated (sampled comparisons); other pixels' outputs are left untouched.
 * Any output pointer may be NULL.  Returns 0, or -1 on allocation failure.
 */
int orc_render(int W, int H, int tw, int th, const uint32_t* ranges, const uint32_t* point_list, int N,
               const double* uv, const double* conic, const double* opacity, const double* rgb,
               const double* bg, const float* dL_dimage, const uint8_t* tile_mask, double* image,
               double* final_T, int* n_contrib, double* grad2d, double* gscale, double* glit,
               double* gallow, double* iallow, double* tallow, int* nc_alt, int* pix_ambig,
               double* pix_widen, double* terr, int* n_active) {
    scene2d_t S = {W, H, uv, conic, opacity, rgb, bg};
    long long gx = (W + tw - 1) / tw, gy = (H + th - 1) / th;
    int maxlen = 1;
    for (long long t = 0; t < gx * gy; ++t) {
        int len = (int)(ranges[2 * t + 1] - ranges[2 * t]);
        if (len > maxlen) maxlen = len;
    }
    contrib_t* cs = (contrib_t*)malloc(sizeof(contrib_t) * (size_t)maxlen);
    contrib_t* cs2 = (contrib_t*)malloc(sizeof(contrib_t) * (size_t)maxlen);
    double* gr = (double*)malloc(sizeof(double) * 9 * (size_t)maxlen);
    double* mg = (double*)malloc(sizeof(double) * 9 * (size_t)maxlen);
    double* gr2 = (double*)malloc(sizeof(double) * 9 * (size_t)maxlen);
    ambig_t* amb = (ambig_t*)malloc(sizeof(ambig_t) * 4 * (size_t)maxlen);
    if (!cs || !cs2 || !gr || !mg || !gr2 || !amb) {
        free(cs); free(cs2); free(gr); free(mg); free(gr2); free(amb);
        return -1;
    }
    if (grad2d) memset(grad2d, 0, sizeof(double) * 9 * (size_t)N);
    if (gscale) memset(gscale, 0, sizeof(double) * 9 * (size_t)N);
    if (glit) memset(glit, 0, sizeof(double) * 9 * (size_t)N);
    if (gallow) memset(gallow, 0, sizeof(double) * 9 * (size_t)N);
    const size_t HW = (size_t)W * H;
    for (long long ty = 0; ty < gy; ++ty)
        for (long long tx = 0; tx < gx; ++tx) {
            long long t = ty * gx + tx;
            if (tile_mask && !tile_mask[t]) continue;
            const uint32_t* list = point_list + ranges[2 * t];
            int n = (int)(ranges[2 * t + 1] - ranges[2 * t]);
            for (int yy = 0; yy < th; ++yy)
                for (int xx = 0; xx < tw; ++xx) {
                    long long px = tx * tw + xx, py = ty * th + yy;
                    if (px >= W || py >= H) continue;
                    size_t pix = (size_t)py * W + (size_t)px;
                    double out[3], Tf, eTf;
                    int last, namb;
                    int nc = walk_pixel(&S, (double)px, (double)py, list, n, -1, 0, cs, out, &Tf, &last,
                                        &eTf, amb, &namb);
                    if (image) for (int ch = 0; ch < 3; ++ch) image[ch * HW + pix] = out[ch];
                    if (final_T) final_T[pix] = Tf;
                    if (n_contrib) n_contrib[pix] = last;
                    if (pix_ambig) pix_ambig[pix] = namb;
                    if (n_active) n_active[pix] = nc;
                    if (nc_alt) nc_alt[pix] = -1;
                    if (iallow) for (int ch = 0; ch < 3; ++ch) iallow[ch * HW + pix] = 0;
                    if (tallow) tallow[pix] = 0;
                    double g[3] = {0, 0, 0};
                    if (dL_dimage) for (int ch = 0; ch < 3; ++ch) g[ch] = dL_dimage[ch * HW + pix];
                    double bpix = 2.0 * eTf + 32.0 * EPS32;
                    for (int j = 0; j < nc; ++j) {
                        double r = cs[j].alpha / (1.0 - cs[j].alpha);
                        double e = cs[j].e_a * (1.0 + r);
                        if (2.0 * eTf + e + 32.0 * EPS32 > bpix) bpix = 2.0 * eTf + e + 32.0 * EPS32;
                    }
                    double widen = AMBIG_SAFETY * bpix / 1e-5;
                    if (widen < 1.0) widen = 1.0;
                    if (pix_widen) pix_widen[pix] = widen;
                    if (terr) terr[pix] = eTf;
                    if (dL_dimage) {
                        pixel_grads(&S, cs, nc, Tf, g, gr, mg);
                        for (int j = 0; j < nc; ++j)
                            for (int p = 0; p < 9; ++p) {
                                size_t o = 9 * (size_t)cs[j].id + p;
                                if (grad2d) grad2d[o] += gr[9 * j + p];
                                if (gscale) gscale[o] += mg[9 * j + p] * widen;
                                if (glit) glit[o] += mg[9 * j + p];
                            }
                    }
                    /* decisions that FP32 may take the other way */
                    for (int a = 0; a < namb; ++a) {
                        double out2[3], Tf2;
                        int last2;
                        int nc2 = walk_pixel(&S, (double)px, (double)py, list, n, amb[a].pos, amb[a].kind,
                                             cs2, out2, &Tf2, &last2, NULL, NULL, NULL);
                        if (iallow) for (int ch = 0; ch < 3; ++ch) iallow[ch * HW + pix] += fabs(out2[ch] - out[ch]);
                        if (tallow) tallow[pix] += fabs(Tf2 - Tf);
                        if (nc_alt && last2 != last) nc_alt[pix] = last2;
                        if (dL_dimage && gallow) {
                            pixel_grads(&S, cs2, nc2, Tf2, g, gr2, NULL);
                            /* merge the two contributor lists by list position */
                            int i = 0, k = 0;
                            while (i < nc || k < nc2) {
                                int pi = i < nc ? cs[i].pos : 1 << 30, pk = k < nc2 ? cs2[k].pos : 1 << 30;
                                uint32_t id = pi <= pk ? cs[i].id : cs2[k].id;
                                for (int p = 0; p < 9; ++p) {
                                    double x1 = pi <= pk ? gr[9 * i + p] : 0.0;
                                    double x2 = pk <= pi ? gr2[9 * k + p] : 0.0;
                                    gallow[9 * (size_t)id + p] += fabs(x2 - x1);
                                }
                                if (pi <= pk) ++i;
                                if (pk <= pi) ++k;
                            }
                        }
                    }
                }
        }
    free(cs); free(cs2); free(gr); free(mg); free(gr2); free(amb);
    return 0;
}

/* ------------------------------------------------------------------ */
/* backward projection: 2D gradients -> 3D parameters                  */
/* ------------------------------------------------------------------ */
/*
 * Chain rule from grad2d [N,9] = dL/d(u, v, A, B, C, o, r, g, b) to
 * dL/dmean [N,3], dL/dscale [N,3], dL/dquat [N,4] (w.r.t. the unnormalised
 * quaternion), dL/dopacity [N], dL/dfeat (SH [N,K,3] or colours [N,3]).
 * Gaussians with radius <= 0 receive zero.  The *_mag outputs (may be NULL)
 * receive the chain evaluated on absolute values, with every division by the
 * 2D determinant weighted by its FP32 conditioning (|ac| + b^2)/det: the scale
 * against which FP32 results are compared.
 * Derivatives are the exact derivatives of the projection as defined: the
 * frustum clamp of x/z, y/z has zero derivative where it is active, the colour
 * clamp at zero likewise.  Depth receives no gradient (it only orders).
 */
static void backproject_one(const orc_camera* cam, int sh_deg, const gauss_t* G, const double* feat,
                            const double* scale, const double* quat_in, const double* g9, int absmode,
                            double* dmean, double* dscale, double* dquat, double* dopac, double* dfeat) {
    (void)quat_in;
    const double* V = cam->view;
    double gv[9];
    for (int i = 0; i < 9; ++i) gv[i] = absmode ? fabs(g9[i]) : g9[i];
    int K = sh_deg < 0 ? 1 : (sh_deg + 1) * (sh_deg + 1);
    double dm[3] = {0, 0, 0};

    /* colour */
    double dcol[3];
    for (int ch = 0; ch < 3; ++ch) dcol[ch] = (sh_deg >= 0 && G->raw[ch] < 0.0) ? 0.0 : gv[6 + ch];
    if (sh_deg < 0) {
        for (int ch = 0; ch < 3; ++ch) dfeat[ch] = dcol[ch];
    } else {
        double Y[16], dY[48];
        sh_eval(sh_deg, G->dir, Y, dY);
        double dd[3] = {0, 0, 0};
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) {
                double y = absmode ? fabs(Y[k]) : Y[k];
                dfeat[3 * k + ch] = y * dcol[ch];
                double f = absmode ? fabs(feat[3 * k + ch]) : feat[3 * k + ch];
                for (int a = 0; a < 3; ++a) dd[a] += f * dcol[ch] * (absmode ? fabs(dY[3 * k + a]) : dY[3 * k + a]);
            }
        /* d = v/|v|: dL/dv = (dL/dd - d (d . dL/dd)) / |v| */
        double dot = G->dir[0] * dd[0] + G->dir[1] * dd[1] + G->dir[2] * dd[2];
        for (int a = 0; a < 3; ++a) {
            if (absmode) {
                double s = fabs(G->dir[0]) * dd[0] + fabs(G->dir[1]) * dd[1] + fabs(G->dir[2]) * dd[2];
                dm[a] += (dd[a] + fabs(G->dir[a]) * s) / G->dist;
            } else {
                dm[a] += (dd[a] - G->dir[a] * dot) / G->dist;
            }
        }
    }
    *dopac = gv[5];

    /* conic (A,B,C) = inverse of [[a,b],[b,c]] */
    const double a = G->a, b = G->b, c = G->c, det = G->det;
    double id2 = 1.0 / (det * det);
    double kap = absmode ? (fabs(a * c) + b * b) / det : 1.0;
    double gA = gv[2], gB = gv[3], gC = gv[4];
    double da, db, dc;
    if (!absmode) {
        da = (-c * c * gA + b * c * gB - b * b * gC) * id2;
        db = (2.0 * b * c * gA - (a * c + b * b) * gB + 2.0 * a * b * gC) * id2;
        dc = (-b * b * gA + a * b * gB - a * a * gC) * id2;
    } else {
        da = (c * c * gA + fabs(b * c) * gB + b * b * gC) * id2 * kap;
        db = (fabs(2.0 * b * c) * gA + (fabs(a * c) + b * b) * gB + fabs(2.0 * a * b) * gC) * id2 * kap;
        dc = (b * b * gA + fabs(a * b) * gB + a * a * gC) * id2 * kap;
    }
    /* symmetric 2x2 gradient of Sigma2 (off-diagonal shared by two entries) */
    double G2[4] = {da, 0.5 * db, 0.5 * db, dc};

    /* Sigma2 = Tm S3 Tm^T: dL/dS3 = Tm^T G2 Tm, dL/dTm = 2 G2 Tm S3 */
    double Tm[6], S3[9];
    for (int i = 0; i < 6; ++i) Tm[i] = absmode ? fabs(G->Tm[i]) : G->Tm[i];
    for (int i = 0; i < 9; ++i) S3[i] = absmode ? fabs(G->S3[i]) : G->S3[i];
    double dS3[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int r = 0; r < 2; ++r)
                for (int q = 0; q < 2; ++q) s += Tm[3 * r + i] * G2[2 * r + q] * Tm[3 * q + j];
            dS3[3 * i + j] = s;
        }
    double dTm[6];
    for (int r = 0; r < 2; ++r)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int q = 0; q < 2; ++q)
                for (int k = 0; k < 3; ++k) s += G2[2 * r + q] * Tm[3 * q + k] * S3[3 * k + j];
            dTm[3 * r + j] = 2.0 * s;
        }
    /* S3 = M M^T, M = R diag(s): dL/dM = 2 dS3 M */
    double M[9], R[9];
    for (int i = 0; i < 9; ++i) { M[i] = absmode ? fabs(G->M[i]) : G->M[i]; R[i] = absmode ? fabs(G->R[i]) : G->R[i]; }
    double dM[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += dS3[3 * i + k] * M[3 * k + j];
            dM[3 * i + j] = 2.0 * s;
        }
    double dR[9];
    for (int j = 0; j < 3; ++j) {
        double s = 0;
        for (int i = 0; i < 3; ++i) {
            s += dM[3 * i + j] * R[3 * i + j];
            dR[3 * i + j] = dM[3 * i + j] * scale[j];
        }
        dscale[j] = s;
    }
    /* R(q) with q = (w,x,y,z) normalised */
    const double w = G->qn[0], x = G->qn[1], y = G->qn[2], z = G->qn[3];
    double dqn[4];
    if (!absmode) {
        dqn[0] = 2.0 * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
        dqn[1] = 2.0 * (y * dR[1] + z * dR[2] + y * dR[3] - 2 * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] - 2 * x * dR[8]);
        dqn[2] = 2.0 * (-2 * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] - 2 * y * dR[8]);
        dqn[3] = 2.0 * (-2 * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2 * z * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
    } else {
        const double W_ = fabs(w), X = fabs(x), Y_ = fabs(y), Z = fabs(z);
        dqn[0] = 2.0 * (Z * dR[1] + Y_ * dR[2] + Z * dR[3] + X * dR[5] + Y_ * dR[6] + X * dR[7]);
        dqn[1] = 2.0 * (Y_ * dR[1] + Z * dR[2] + Y_ * dR[3] + 2 * X * dR[4] + W_ * dR[5] + Z * dR[6] + W_ * dR[7] + 2 * X * dR[8]);
        dqn[2] = 2.0 * (2 * Y_ * dR[0] + X * dR[1] + W_ * dR[2] + X * dR[3] + Z * dR[5] + W_ * dR[6] + Z * dR[7] + 2 * Y_ * dR[8]);
        dqn[3] = 2.0 * (2 * Z * dR[0] + W_ * dR[1] + X * dR[2] + W_ * dR[3] + 2 * Z * dR[4] + Y_ * dR[5] + X * dR[6] + Y_ * dR[7]);
    }
    {
        double dot = G->qn[0] * dqn[0] + G->qn[1] * dqn[1] + G->qn[2] * dqn[2] + G->qn[3] * dqn[3];
        double dota = fabs(G->qn[0]) * dqn[0] + fabs(G->qn[1]) * dqn[1] + fabs(G->qn[2]) * dqn[2] + fabs(G->qn[3]) * dqn[3];
        for (int i = 0; i < 4; ++i)
            dquat[i] = absmode ? (dqn[i] + fabs(G->qn[i]) * dota) / G->qnorm
                               : (dqn[i] - G->qn[i] * dot) / G->qnorm;
    }
    /* Tm = J W: dL/dJ = dL/dTm W^T */
    double dJ[6];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) {
            double s = 0;
            for (int j = 0; j < 3; ++j) s += dTm[3 * r + j] * (absmode ? fabs(V[4 * k + j]) : V[4 * k + j]);
            dJ[3 * r + k] = s;
        }
    /* J(p) and (u,v)(p) */
    const double pz = G->p[2], px = G->p[0], py = G->p[1];
    const double fx = cam->fx, fy = cam->fy;
    double dp[3];
    double gu = gv[0], gvv = gv[1];
    if (!absmode) {
        double dJ02_dx = G->clx ? 0.0 : -fx / (pz * pz);
        double dJ02_dz = fx * G->tx / (pz * pz) * (G->clx ? 1.0 : 2.0);
        double dJ12_dy = G->cly ? 0.0 : -fy / (pz * pz);
        double dJ12_dz = fy * G->ty / (pz * pz) * (G->cly ? 1.0 : 2.0);
        dp[0] = gu * fx / pz + dJ[2] * dJ02_dx;
        dp[1] = gvv * fy / pz + dJ[5] * dJ12_dy;
        dp[2] = -gu * fx * px / (pz * pz) - gvv * fy * py / (pz * pz) - dJ[0] * fx / (pz * pz) -
                dJ[4] * fy / (pz * pz) + dJ[2] * dJ02_dz + dJ[5] * dJ12_dz;
    } else {
        double dJ02_dx = G->clx ? 0.0 : fx / (pz * pz);
        double dJ02_dz = fx * fabs(G->tx) / (pz * pz) * (G->clx ? 1.0 : 2.0);
        double dJ12_dy = G->cly ? 0.0 : fy / (pz * pz);
        double dJ12_dz = fy * fabs(G->ty) / (pz * pz) * (G->cly ? 1.0 : 2.0);
        dp[0] = gu * fx / pz + dJ[2] * dJ02_dx;
        dp[1] = gvv * fy / pz + dJ[5] * dJ12_dy;
        dp[2] = gu * fx * fabs(px) / (pz * pz) + gvv * fy * fabs(py) / (pz * pz) + dJ[0] * fx / (pz * pz) +
                dJ[4] * fy / (pz * pz) + dJ[2] * dJ02_dz + dJ[5] * dJ12_dz;
    }
    /* p = W mean + t */
    for (int i = 0; i < 3; ++i) {
        double s = 0;
        for (int k = 0; k < 3; ++k) s += (absmode ? fabs(V[4 * k + i]) : V[4 * k + i]) * dp[k];
        dmean[i] = dm[i] + s;
    }
}

int orc_backproject(int N, int sh_deg, const double* mean, const double* scale, const double* quat,
                    const double* opacity, const double* feat, const orc_camera* cam, int tw, int th,
                    const double* grad2d, double* dmean, double* dscale, double* dquat, double* dopac,
                    double* dfeat, double* dmean_mag, double* dscale_mag, double* dquat_mag,
                    double* dfeat_mag) {
    int K = sh_deg < 0 ? 1 : (sh_deg + 1) * (sh_deg + 1);
    (void)opacity;
    for (int i = 0; i < N; ++i) {
        gauss_t G;
        project_one(cam, sh_deg, mean + 3 * i, scale + 3 * i, quat + 4 * i, feat + 3 * K * i, tw, th, &G);
        double* fm = dfeat + 3 * (size_t)K * i;
        if (G.culled) {
            memset(dmean + 3 * i, 0, 3 * sizeof(double));
            memset(dscale + 3 * i, 0, 3 * sizeof(double));
            memset(dquat + 4 * i, 0, 4 * sizeof(double));
            dopac[i] = 0;
            memset(fm, 0, 3 * (size_t)K * sizeof(double));
            if (dmean_mag) memset(dmean_mag + 3 * i, 0, 3 * sizeof(double));
            if (dscale_mag) memset(dscale_mag + 3 * i, 0, 3 * sizeof(double));
            if (dquat_mag) memset(dquat_mag + 4 * i, 0, 4 * sizeof(double));
            if (dfeat_mag) memset(dfeat_mag + 3 * (size_t)K * i, 0, 3 * (size_t)K * sizeof(double));
            continue;
        }
        backproject_one(cam, sh_deg, &G, feat + 3 * K * i, scale + 3 * i, quat + 4 * i, grad2d + 9 * i, 0,
                        dmean + 3 * i, dscale + 3 * i, dquat + 4 * i, dopac + i, fm);
        if (dmean_mag && dscale_mag && dquat_mag && dfeat_mag) {
            double op;
            backproject_one(cam, sh_deg, &G, feat + 3 * K * i, scale + 3 * i, quat + 4 * i, grad2d + 9 * i, 1,
                            dmean_mag + 3 * i, dscale_mag + 3 * i, dquat_mag + 4 * i, &op,
                            dfeat_mag + 3 * (size_t)K * i);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Adam (Kingma & Ba 2015, Algorithm 1) on a flat parameter array        */
/* ------------------------------------------------------------------ */
void orc_adam(long long n, double* param, const double* grad, double* m, double* v, double lr,
              double beta1, double beta2, double eps, int step) {
    double bc1 = 1.0 - pow(beta1, step), bc2 = 1.0 - pow(beta2, step);
    for (long long i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        double mh = m[i] / bc1, vh = v[i] / bc2;
        param[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
