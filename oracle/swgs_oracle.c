/*
 * swgs_oracle.c -- plain, slow FP64 CPU oracle for the SwinGS frame-t
 * splatting hot path (arXiv 2409.07759).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
 * this file; only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark do. It shares no code, header or constant table with the CUDA
 * library: every formula below is written out here on its own.
 *
 * What it computes, and where the paper defines it:
 *   - active set of frame t: start <= t < expire (Sec. 4.2; Alg. 1 filter on
 *     gs and matured; Alg. 2 render_thread filter);
 *   - 3D Gaussian and covariance Sigma = R S S^T R^T (Eq. 1, Eq. 2);
 *   - projection to a 2D Gaussian and front-to-back compositing in z order
 *     (Sec. 2.1, Eq. 3); the projection formula itself is deferred by the paper
 *     to 3DGS [13]; the affine (EWA) form is used;
 *   - view-dependent colour from real spherical harmonics (Sec. 8.1);
 *   - the L1 photometric gradient and analytic backward (Alg. 1 loss and
 *     backward);
 *   - SGLD noise on active optimisable Gaussians and relocation of dead
 *     Gaussians (Alg. 1 noise and relocate steps; Sec. 3.2, Sec. 4.4, following
 *     3DGS-MCMC [14]);
 *   - slice replacement (Alg. 2) lives in the Python wrapper.
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   pinhole camera with pixel (i,j) sampled at (i+0.5, j+0.5); near plane
 *   culling; a 1.3x guard band on the projection Jacobian; +0.3 px^2 dilation;
 *   support limited to Mahalanobis^2 <= 9; alpha = min(0.99, o*G), skipped below
 *   1/255; blending stops before a Gaussian that would take T below 1e-4; depth
 *   ties broken by slot index.
 *
 * Two precisions:
 *   - "key mode" (functions prefixed km_): the discrete decisions -- culling,
 *     tile rectangle, tile count, depth key -- computed in FP32 with a written
 *     down sequence of correctly rounded +,-,*,/,sqrt, floor and a polynomial
 *     exp, so that they are integers both sides decide identically. This file
 *     must be compiled with -ffp-contract=off and without fast-math.
 *   - everything else (pixel values, gradients, SGLD, relocation values) in
 *     FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Structures passed from Python (ctypes).                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R[9]; /* world -> camera rotation, row major */
    float t[3];
    int32_t frame;
} or_view;

typedef struct {
    const float *means;          /* [N,3] */
    const float *log_scales;     /* [N,3] */
    const float *quats;          /* [N,4] (w,x,y,z), unnormalised */
    const float *logits;         /* [N]   opacity = sigmoid(logit) */
    const float *sh;             /* [N,K,3] */
    const int32_t *start;        /* [N] */
    const int32_t *expire;       /* [N] */
    const uint8_t *frozen;       /* [N] 1 = matured (no gradient) */
    int64_t n;
    int32_t sh_degree;
} or_scene;

/* Key-mode (FP32) record of one Gaussian seen from one view. */
typedef struct {
    float u, v, z;             /* projected centre (pixels), camera depth */
    float a, b, c;             /* dilated 2D covariance */
    float det, lambda1, radius;
    int32_t culled;            /* 1: behind near plane or det <= 0 */
    int32_t tx0, tx1, ty0, ty1;/* inclusive bounding tile rectangle (empty if tx1<tx0) */
    int32_t tiles;             /* tiles of the rectangle the 3-sigma ellipse covers */
    float A, B, C;             /* conic: m = A dx^2 + 2 B dx dy + C dy^2 */
} or_km;

/* A tile is kept when the ellipse {m <= OR_TILE_MAHAL} reaches the rectangle
 * spanned by its pixel centres (9 = the 3-sigma support, plus 0.1% so that
 * FP32 rounding can never drop a tile holding a pixel with m <= 9). */
#define OR_TILE_MAHAL 9.009f

/* Row rule (key mode). The ellipse E = {m <= OR_TILE_MAHAL} meets the band of
 * pixel-centre rows dy in [ya, yb] in a convex set, so the tiles of a tile row
 * that E reaches form one run; its x-extent [left, right] over the band comes
 * from the chord ends c(y) -+ w(y) at the band ends (c = -(B/A) y,
 * w = sqrt(A T - det_c y^2) / A) and from E's extreme points
 * (+-xm, -+(B/C) xm), xm = sqrt(C T / det_c), where the x-extent is attained.
 * km_row_extent returns 0 when the band misses E. */
typedef struct { float AT, detc, rBA, iA, rBC, xm, ym; } km_ell;

static km_ell km_ellipse(float A, float B, float C)
{
    km_ell e;
    e.AT = A * OR_TILE_MAHAL;
    float t1 = A * C;
    float t2 = B * B;
    e.detc = t1 - t2;
    e.rBA = B / A;
    e.iA = 1.0f / A;
    e.rBC = B / C;
    float q = C * OR_TILE_MAHAL;
    q = q / e.detc;
    e.xm = sqrtf(q);
    q = e.AT / e.detc;
    e.ym = sqrtf(q);
    return e;
}

/* The two ends c(y) -+ w(y) of the ellipse's chord at row offset y. */
static void km_chord(const km_ell *e, float y, float *l, float *r)
{
    float c = e->rBA * y;
    c = -c;
    float q = e->detc * y;
    q = q * y;
    q = e->AT - q;
    if (q < 0.0f) q = 0.0f;
    q = sqrtf(q);
    float w = q * e->iA;
    *l = c - w;
    *r = c + w;
}

static int km_row_extent(const km_ell *e, float ya, float yb, float *left, float *right)
{
    float lo = ya > -e->ym ? ya : -e->ym;
    float hi = yb < e->ym ? yb : e->ym;
    if (!(lo <= hi)) return 0;
    float t = e->rBC * e->xm;
    float dyr = -t;      /* row of the rightmost point */
    float dyl = t;       /* row of the leftmost point */
    float l0, r0, l1, r1;
    km_chord(e, lo, &l0, &r0);
    km_chord(e, hi, &l1, &r1);
    if (lo <= dyr && dyr <= hi) *right = e->xm;
    else *right = r0 > r1 ? r0 : r1;
    if (lo <= dyl && dyl <= hi) *left = -e->xm;
    else *left = l0 < l1 ? l0 : l1;
    return 1;
}

/* The run [*first, *last] of kept tiles of row ty inside [tx0, tx1]
 * (returns its length, 0 if none). A tile is kept when its pixel-centre
 * x-span [xa, xb] meets [left, right]: xb >= left and xa <= right. If det_c <= 0 (degenerate conic) the
 * whole row of the rectangle is kept. */
static int km_row_run(const km_ell *e, float u, float v, int tx0, int tx1, int ty, int tile_w,
                      int tile_h, int *first, int *last)
{
    if (!(e->detc > 0.0f)) { *first = tx0; *last = tx1; return tx1 - tx0 + 1; }
    float by = (float)(ty * tile_h);
    float ya = (by + 0.5f) - v;
    float yb = (by + ((float)tile_h - 0.5f)) - v;
    float left, right;
    if (!km_row_extent(e, ya, yb, &left, &right)) return 0;
    int a = tx0;
    while (a <= tx1) {
        float xb = ((float)(a * tile_w) + ((float)tile_w - 0.5f)) - u;
        if (xb >= left) break;
        ++a;
    }
    if (a > tx1) return 0;
    int b = tx1;
    while (b > a) {
        float xa = ((float)(b * tile_w) + 0.5f) - u;
        if (xa <= right) break;
        --b;
    }
    /* [left, right] may fall short of tile a's span (left of its first pixel
     * centre, or in the gap between two tiles' pixel centres): no tile then */
    {
        float xa = ((float)(a * tile_w) + 0.5f) - u;
        if (!(xa <= right)) return 0;
    }
    *first = a;
    *last = b;
    return b - a + 1;
}

/* Blend thresholds (readings of the unspecified renderer details). */
#define OR_ALPHA_MIN   (1.0 / 255.0)
#define OR_ALPHA_MAX   0.99
#define OR_T_STOP      1e-4
#define OR_MAHAL_MAX   9.0
#define OR_DILATION    0.3
#define OR_GUARD       1.3

/* Near-discontinuity bands (relative), set by the caller. */
typedef struct {
    double m, alpha, t_stop, clamp, guard, colour;
} or_bands;

static int sh_count(int degree) { return (degree + 1) * (degree + 1); }

/* ------------------------------------------------------------------------ */
/* Active set (Sec. 4.2: a Gaussian renders iff start <= frame < expire).    */
/* ------------------------------------------------------------------------ */

int64_t or_active_ids(const int32_t *start, const int32_t *expire, int64_t n,
                      int32_t frame, int32_t *out)
{
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i)
        if (start[i] <= frame && frame < expire[i]) out[k++] = (int32_t)i;
    return k;
}

/* ------------------------------------------------------------------------ */
/* Key mode: FP32, one rounding per written operation.                       */
/* ------------------------------------------------------------------------ */

/* exp(x) for the discrete path: Cody-Waite reduction x = k ln2 + r with ln2
 * split into a 16-bit head and a tail, then the degree-7 Taylor polynomial of
 * exp(r) by Horner's rule, then an exact scaling by 2^k. */
static float km_exp(float x)
{
    const float L2E = 0x1.715476p+0f;
    const float LN2_HI = 0x1.62e4p-1f;
    const float LN2_LO = 0x1.7f7d1cp-20f;
    if (x < -80.0f) x = -80.0f;
    if (x > 80.0f) x = 80.0f;
    float t = x * L2E;
    t = t + 0.5f;
    float k = floorf(t);
    float h = k * LN2_HI;
    float r = x - h;
    float l = k * LN2_LO;
    r = r - l;
    float p = 0x1.a01a02p-13f;           /* 1/7! */
    p = p * r; p = p + 0x1.6c16c2p-10f;   /* 1/6! */
    p = p * r; p = p + 0x1.111112p-7f;    /* 1/5! */
    p = p * r; p = p + 0x1.555556p-5f;    /* 1/4! */
    p = p * r; p = p + 0x1.555556p-3f;    /* 1/3! */
    p = p * r; p = p + 0.5f;
    p = p * r; p = p + 1.0f;
    p = p * r; p = p + 1.0f;
    int e = (int)k;
    union { uint32_t u; float f; } sc;
    sc.u = (uint32_t)(e + 127) << 23;
    return p * sc.f;
}

/* The discrete quantities of one (view, Gaussian) pair. */
void or_keymode(const or_scene *sc, const or_view *vw, int64_t slot,
                int32_t tile_w, int32_t tile_h, float near_plane, or_km *o)
{
    memset(o, 0, sizeof(*o));
    const float *mu = sc->means + 3 * slot;
    const float *R = vw->R;
    float p[3];
    for (int k = 0; k < 3; ++k) {
        float s0 = R[3 * k + 0] * mu[0];
        float s1 = R[3 * k + 1] * mu[1];
        float s2 = R[3 * k + 2] * mu[2];
        float s = s0 + s1;
        s = s + s2;
        p[k] = s + vw->t[k];
    }
    float z = p[2];
    o->z = z;
    if (!(z > near_plane)) { o->culled = 1; return; }

    /* guard band on the Jacobian */
    float tanx = (0.5f * (float)vw->width) / vw->fx;
    float tany = (0.5f * (float)vw->height) / vw->fy;
    float limx = 1.3f * tanx;
    float limy = 1.3f * tany;
    float xz = p[0] / z;
    float yz = p[1] / z;
    float xzc = xz < -limx ? -limx : (xz > limx ? limx : xz);
    float yzc = yz < -limy ? -limy : (yz > limy ? limy : yz);
    float tx = xzc * z;
    float ty = yzc * z;
    float zz = z * z;
    float J00 = vw->fx / z;
    float J11 = vw->fy / z;
    float J02 = -((vw->fx * tx) / zz);
    float J12 = -((vw->fy * ty) / zz);

    /* Sigma = M M^T with M = Rq S (Eq. 2) */
    const float *ls = sc->log_scales + 3 * slot;
    float s[3] = {km_exp(ls[0]), km_exp(ls[1]), km_exp(ls[2])};
    const float *q = sc->quats + 4 * slot;
    float nn = q[0] * q[0];
    nn = nn + q[1] * q[1];
    nn = nn + q[2] * q[2];
    nn = nn + q[3] * q[3];
    float n = sqrtf(nn);
    float w = q[0] / n, x = q[1] / n, y = q[2] / n, zq = q[3] / n;
    float xx = x * x, yy = y * y, qz2 = zq * zq;
    float xy = x * y, xzq = x * zq, yzq = y * zq;
    float wx = w * x, wy = w * y, wz = w * zq;
    float Rq[9];
    Rq[0] = 1.0f - 2.0f * (yy + qz2);
    Rq[1] = 2.0f * (xy - wz);
    Rq[2] = 2.0f * (xzq + wy);
    Rq[3] = 2.0f * (xy + wz);
    Rq[4] = 1.0f - 2.0f * (xx + qz2);
    Rq[5] = 2.0f * (yzq - wx);
    Rq[6] = 2.0f * (xzq - wy);
    Rq[7] = 2.0f * (yzq + wx);
    Rq[8] = 1.0f - 2.0f * (xx + yy);
    float M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[3 * i + j] = Rq[3 * i + j] * s[j];
    float Sg[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            float a0 = M[3 * i + 0] * M[3 * j + 0];
            float a1 = M[3 * i + 1] * M[3 * j + 1];
            float a2 = M[3 * i + 2] * M[3 * j + 2];
            float acc = a0 + a1;
            Sg[3 * i + j] = acc + a2;
        }
    /* T = J W, structural zeros of J skipped */
    float T0[3], T1[3];
    for (int j = 0; j < 3; ++j) {
        float a0 = J00 * R[0 + j];
        float a2 = J02 * R[6 + j];
        T0[j] = a0 + a2;
        float b1 = J11 * R[3 + j];
        float b2 = J12 * R[6 + j];
        T1[j] = b1 + b2;
    }
    /* U = T Sigma, cov = U T^T */
    float U0[3], U1[3];
    for (int j = 0; j < 3; ++j) {
        float a0 = T0[0] * Sg[0 + j];
        float a1 = T0[1] * Sg[3 + j];
        float a2 = T0[2] * Sg[6 + j];
        float acc = a0 + a1;
        U0[j] = acc + a2;
        float b0 = T1[0] * Sg[0 + j];
        float b1 = T1[1] * Sg[3 + j];
        float b2 = T1[2] * Sg[6 + j];
        acc = b0 + b1;
        U1[j] = acc + b2;
    }
    float c00, c01, c11;
    { float a0 = U0[0] * T0[0], a1 = U0[1] * T0[1], a2 = U0[2] * T0[2];
      float acc = a0 + a1; c00 = acc + a2; }
    { float a0 = U0[0] * T1[0], a1 = U0[1] * T1[1], a2 = U0[2] * T1[2];
      float acc = a0 + a1; c01 = acc + a2; }
    { float a0 = U1[0] * T1[0], a1 = U1[1] * T1[1], a2 = U1[2] * T1[2];
      float acc = a0 + a1; c11 = acc + a2; }
    float a = c00 + 0.3f;
    float b = c01;
    float c = c11 + 0.3f;
    o->a = a; o->b = b; o->c = c;
    float ac = a * c;
    float bb = b * b;
    float det = ac - bb;
    o->det = det;
    if (!(det > 0.0f)) { o->culled = 1; return; }
    float mid = 0.5f * (a + c);
    float disc = mid * mid;
    disc = disc - det;
    if (disc < 0.1f) disc = 0.1f;
    float l1 = mid + sqrtf(disc);
    o->lambda1 = l1;
    float rad = ceilf(3.0f * sqrtf(l1));
    o->radius = rad;
    float u = vw->fx * xz;
    u = u + vw->cx;
    float v = vw->fy * yz;
    v = v + vw->cy;
    o->u = u; o->v = v;

    int ntx = (vw->width + tile_w - 1) / tile_w;
    int nty = (vw->height + tile_h - 1) / tile_h;
    float fxlo = floorf((u - rad) / (float)tile_w);
    float fxhi = floorf((u + rad) / (float)tile_w);
    float fylo = floorf((v - rad) / (float)tile_h);
    float fyhi = floorf((v + rad) / (float)tile_h);
    int x0 = fxlo < 0.0f ? 0 : (fxlo > (float)ntx ? ntx : (int)fxlo);
    int x1 = fxhi > (float)(ntx - 1) ? ntx - 1 : (fxhi < -1.0f ? -1 : (int)fxhi);
    int y0 = fylo < 0.0f ? 0 : (fylo > (float)nty ? nty : (int)fylo);
    int y1 = fyhi > (float)(nty - 1) ? nty - 1 : (fyhi < -1.0f ? -1 : (int)fyhi);
    o->tx0 = x0; o->tx1 = x1; o->ty0 = y0; o->ty1 = y1;
    float A = c / det;
    float B = -(b / det);
    float C = a / det;
    o->A = A; o->B = B; o->C = C;
    km_ell e = km_ellipse(A, B, C);
    int covered = 0;
    if (x1 >= x0)
        for (int ty = y0; ty <= y1; ++ty) {
            int f, l;
            covered += km_row_run(&e, u, v, x0, x1, ty, tile_w, tile_h, &f, &l);
        }
    o->tiles = covered;
}

/* Tiles covered by one key-mode record, row-major within its rectangle;
 * returns their number (out: global-in-view tile ids, may be NULL). */
int32_t or_record_tiles(const or_km *k, int32_t ntx, int32_t tile_w, int32_t tile_h, int32_t *out)
{
    int32_t n = 0;
    if (k->culled || k->tx1 < k->tx0) return 0;
    km_ell e = km_ellipse(k->A, k->B, k->C);
    for (int ty = k->ty0; ty <= k->ty1; ++ty) {
        int f, l;
        if (!km_row_run(&e, k->u, k->v, k->tx0, k->tx1, ty, tile_w, tile_h, &f, &l)) continue;
        for (int tx = f; tx <= l; ++tx) {
            if (out) out[n] = ty * ntx + tx;
            ++n;
        }
    }
    return n;
}

/* Depth key: the bits of a positive FP32 depth order like the depth. */
static uint32_t depth_bits(float z)
{
    union { float f; uint32_t u; } c;
    c.f = z;
    return c.u;
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics, degrees 0..3 (Sec. 8.1).                        */
/* Y_lm = (-1)^m * (standard real SH); constants from the normalised forms.  */
/* ------------------------------------------------------------------------ */

static void sh_basis(double x, double y, double z, double Y[16], double dY[16][3])
{
    const double PI = 3.14159265358979323846;
    const double C0 = 0.5 * sqrt(1.0 / PI);
    const double C1 = sqrt(3.0 / (4.0 * PI));
    const double C2a = 0.5 * sqrt(15.0 / PI);
    const double C2b = 0.25 * sqrt(5.0 / PI);
    const double C2c = 0.25 * sqrt(15.0 / PI);
    const double C3a = 0.25 * sqrt(35.0 / (2.0 * PI));
    const double C3b = 0.5 * sqrt(105.0 / PI);
    const double C3c = 0.25 * sqrt(21.0 / (2.0 * PI));
    const double C3d = 0.25 * sqrt(7.0 / PI);
    const double C3e = 0.25 * sqrt(105.0 / PI);
    double xx = x * x, yy = y * y, zz = z * z;
    memset(dY, 0, sizeof(double) * 16 * 3);
    Y[0] = C0;
    /* l = 1: m = -1, 0, 1 */
    Y[1] = -C1 * y;  dY[1][1] = -C1;
    Y[2] = C1 * z;   dY[2][2] = C1;
    Y[3] = -C1 * x;  dY[3][0] = -C1;
    /* l = 2 */
    Y[4] = C2a * x * y;              dY[4][0] = C2a * y; dY[4][1] = C2a * x;
    Y[5] = -C2a * y * z;             dY[5][1] = -C2a * z; dY[5][2] = -C2a * y;
    Y[6] = C2b * (2 * zz - xx - yy); dY[6][0] = -2 * C2b * x; dY[6][1] = -2 * C2b * y;
                                     dY[6][2] = 4 * C2b * z;
    Y[7] = -C2a * x * z;             dY[7][0] = -C2a * z; dY[7][2] = -C2a * x;
    Y[8] = C2c * (xx - yy);          dY[8][0] = 2 * C2c * x; dY[8][1] = -2 * C2c * y;
    /* l = 3 */
    Y[9] = -C3a * y * (3 * xx - yy);
    dY[9][0] = -C3a * 6 * x * y; dY[9][1] = -C3a * (3 * xx - 3 * yy);
    Y[10] = C3b * x * y * z;
    dY[10][0] = C3b * y * z; dY[10][1] = C3b * x * z; dY[10][2] = C3b * x * y;
    Y[11] = -C3c * y * (4 * zz - xx - yy);
    dY[11][0] = C3c * 2 * x * y; dY[11][1] = -C3c * (4 * zz - xx - 3 * yy);
    dY[11][2] = -C3c * 8 * y * z;
    Y[12] = C3d * z * (2 * zz - 3 * xx - 3 * yy);
    dY[12][0] = -C3d * 6 * x * z; dY[12][1] = -C3d * 6 * y * z;
    dY[12][2] = C3d * (6 * zz - 3 * xx - 3 * yy);
    Y[13] = -C3c * x * (4 * zz - xx - yy);
    dY[13][0] = -C3c * (4 * zz - 3 * xx - yy); dY[13][1] = C3c * 2 * x * y;
    dY[13][2] = -C3c * 8 * x * z;
    Y[14] = C3e * z * (xx - yy);
    dY[14][0] = C3e * 2 * x * z; dY[14][1] = -C3e * 2 * y * z; dY[14][2] = C3e * (xx - yy);
    Y[15] = -C3a * x * (xx - 3 * yy);
    dY[15][0] = -C3a * (3 * xx - 3 * yy); dY[15][1] = C3a * 6 * x * y;
}

/* Exposed for the quadrature / library pins. */
void or_sh_basis(double x, double y, double z, double *Y16)
{
    double dY[16][3];
    sh_basis(x, y, z, Y16, dY);
}

/* ------------------------------------------------------------------------ */
/* FP64 projection of one Gaussian into one view.                            */
/* ------------------------------------------------------------------------ */

typedef struct {
    /* outputs used by the blend */
    double u, v, A, B, C, o, rgb[3];
    /* intermediates kept for the backward pass */
    double p[3], z, xz, yz, clampx, clampy, limx, limy, tx, ty;
    double J00, J02, J11, J12, Tm[2][3], Sg[3][3], M[3][3], Rq[3][3], s[3];
    double qn[4], qnorm, cov[3], covd[3], det;
    double dir[3], dist, raw[3];
    double Y[16], dY[16][3];
    double logit;
} or_proj;

static void mat3_mul(const double A[3][3], const double B[3][3], double C[3][3])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[i][k] * B[k][j];
            C[i][j] = s;
        }
}

static void project64(const or_scene *sc, const or_view *vw, int64_t slot, or_proj *P)
{
    double W[3][3], t[3], mu[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) W[i][j] = vw->R[3 * i + j];
        t[i] = vw->t[i];
        mu[i] = sc->means[3 * slot + i];
    }
    for (int i = 0; i < 3; ++i)
        P->p[i] = W[i][0] * mu[0] + W[i][1] * mu[1] + W[i][2] * mu[2] + t[i];
    double z = P->p[2];
    P->z = z;
    double fx = vw->fx, fy = vw->fy;
    P->limx = OR_GUARD * (0.5 * vw->width / fx);
    P->limy = OR_GUARD * (0.5 * vw->height / fy);
    P->xz = P->p[0] / z;
    P->yz = P->p[1] / z;
    P->clampx = P->xz < -P->limx ? -1.0 : (P->xz > P->limx ? 1.0 : 0.0);
    P->clampy = P->yz < -P->limy ? -1.0 : (P->yz > P->limy ? 1.0 : 0.0);
    double xzc = P->clampx != 0.0 ? P->clampx * P->limx : P->xz;
    double yzc = P->clampy != 0.0 ? P->clampy * P->limy : P->yz;
    P->tx = xzc * z;
    P->ty = yzc * z;
    P->J00 = fx / z;
    P->J11 = fy / z;
    P->J02 = -fx * P->tx / (z * z);
    P->J12 = -fy * P->ty / (z * z);
    double J[2][3] = {{P->J00, 0.0, P->J02}, {0.0, P->J11, P->J12}};
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += J[i][k] * W[k][j];
            P->Tm[i][j] = s;
        }
    /* Eq. 2 */
    for (int j = 0; j < 3; ++j) P->s[j] = exp((double)sc->log_scales[3 * slot + j]);
    const float *q = sc->quats + 4 * slot;
    double qq[4] = {q[0], q[1], q[2], q[3]};
    P->qnorm = sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
    for (int k = 0; k < 4; ++k) P->qn[k] = qq[k] / P->qnorm;
    double w = P->qn[0], x = P->qn[1], y = P->qn[2], zq = P->qn[3];
    double Rq[3][3] = {
        {1 - 2 * (y * y + zq * zq), 2 * (x * y - w * zq), 2 * (x * zq + w * y)},
        {2 * (x * y + w * zq), 1 - 2 * (x * x + zq * zq), 2 * (y * zq - w * x)},
        {2 * (x * zq - w * y), 2 * (y * zq + w * x), 1 - 2 * (x * x + y * y)}};
    memcpy(P->Rq, Rq, sizeof(Rq));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P->M[i][j] = Rq[i][j] * P->s[j];
    double Mt[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Mt[i][j] = P->M[j][i];
    mat3_mul(P->M, Mt, P->Sg);
    /* cov = T Sigma T^T */
    double U[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += P->Tm[i][k] * P->Sg[k][j];
            U[i][j] = s;
        }
    double c00 = 0, c01 = 0, c11 = 0;
    for (int k = 0; k < 3; ++k) {
        c00 += U[0][k] * P->Tm[0][k];
        c01 += U[0][k] * P->Tm[1][k];
        c11 += U[1][k] * P->Tm[1][k];
    }
    P->cov[0] = c00; P->cov[1] = c01; P->cov[2] = c11;
    P->covd[0] = c00 + OR_DILATION; P->covd[1] = c01; P->covd[2] = c11 + OR_DILATION;
    P->det = P->covd[0] * P->covd[2] - P->covd[1] * P->covd[1];
    P->A = P->covd[2] / P->det;
    P->B = -P->covd[1] / P->det;
    P->C = P->covd[0] / P->det;
    P->u = fx * P->p[0] / z + vw->cx;
    P->v = fy * P->p[1] / z + vw->cy;
    P->logit = sc->logits[slot];
    P->o = 1.0 / (1.0 + exp(-P->logit));
    /* colour: direction from the camera centre -R^T t to the mean */
    double cc[3];
    for (int j = 0; j < 3; ++j) cc[j] = -(W[0][j] * t[0] + W[1][j] * t[1] + W[2][j] * t[2]);
    double d[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
    P->dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    for (int j = 0; j < 3; ++j) P->dir[j] = d[j] / P->dist;
    sh_basis(P->dir[0], P->dir[1], P->dir[2], P->Y, P->dY);
    int K = sh_count(sc->sh_degree);
    const float *sh = sc->sh + (int64_t)slot * K * 3;
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += P->Y[k] * sh[3 * k + ch];
        P->raw[ch] = acc + 0.5;
        P->rgb[ch] = P->raw[ch] > 0.0 ? P->raw[ch] : 0.0;
    }
}

/* Public per-record FP64 values: u, v, A, B, C, opacity, r, g, b, depth. */
void or_project(const or_scene *sc, const or_view *vw, int64_t slot, double *out10)
{
    or_proj P;
    project64(sc, vw, slot, &P);
    out10[0] = P.u; out10[1] = P.v; out10[2] = P.A; out10[3] = P.B; out10[4] = P.C;
    out10[5] = P.o; out10[6] = P.rgb[0]; out10[7] = P.rgb[1]; out10[8] = P.rgb[2];
    out10[9] = P.z;
}

/* ------------------------------------------------------------------------ */
/* Per-view render set: active, not culled (key mode), depth-ordered.        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n;          /* records (active Gaussians of this view's frame) */
    int32_t *slot;      /* [n] ascending slot ids */
    or_km *km;          /* [n] */
    or_proj *pj;        /* [n] (only filled where !culled) */
    int32_t *order;     /* records in (depth bits, slot) order, culled dropped */
    int64_t n_order;
    int32_t ntx, nty;
    int64_t *tile_off;  /* [ntx*nty+1] CSR over (tile -> sorted records) */
    int32_t *tile_rec;
} or_vset;

typedef struct { uint64_t key; int64_t idx; } kv_pair;

static int cmp_kv(const void *a, const void *b)
{
    const kv_pair *x = (const kv_pair *)a, *y = (const kv_pair *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

static void vset_free(or_vset *S)
{
    free(S->slot); free(S->km); free(S->pj); free(S->order);
    free(S->tile_off); free(S->tile_rec);
    memset(S, 0, sizeof(*S));
}

static int vset_build(const or_scene *sc, const or_view *vw, int32_t tile_w, int32_t tile_h,
                      float near_plane, int with_tiles, or_vset *S)
{
    memset(S, 0, sizeof(*S));
    S->slot = (int32_t *)malloc(sizeof(int32_t) * (sc->n > 0 ? sc->n : 1));
    S->n = or_active_ids(sc->start, sc->expire, sc->n, vw->frame, S->slot);
    S->km = (or_km *)calloc(S->n > 0 ? S->n : 1, sizeof(or_km));
    S->pj = (or_proj *)calloc(S->n > 0 ? S->n : 1, sizeof(or_proj));
    S->order = (int32_t *)malloc(sizeof(int32_t) * (S->n > 0 ? S->n : 1));
    if (!S->slot || !S->km || !S->pj || !S->order) return -1;
    kv_pair *kv = (kv_pair *)malloc(sizeof(kv_pair) * (S->n > 0 ? S->n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < S->n; ++i) {
        or_keymode(sc, vw, S->slot[i], tile_w, tile_h, near_plane, &S->km[i]);
        if (S->km[i].culled) continue;
        project64(sc, vw, S->slot[i], &S->pj[i]);
        kv[m].key = depth_bits(S->km[i].z);
        kv[m].idx = i;
        ++m;
    }
    qsort(kv, (size_t)m, sizeof(kv_pair), cmp_kv);
    for (int64_t j = 0; j < m; ++j) S->order[j] = (int32_t)kv[j].idx;
    S->n_order = m;
    free(kv);
    S->ntx = (vw->width + tile_w - 1) / tile_w;
    S->nty = (vw->height + tile_h - 1) / tile_h;
    if (!with_tiles) return 0;
    /* Emit (tile << 32 | depth bits) keys in record order and sort them
     * stably: the per-tile lists of Eq. 3's depth ordering. */
    int64_t nkeys = 0;
    for (int64_t i = 0; i < S->n; ++i) if (!S->km[i].culled) nkeys += S->km[i].tiles;
    kv_pair *keys = (kv_pair *)malloc(sizeof(kv_pair) * (nkeys > 0 ? nkeys : 1));
    int64_t e = 0;
    for (int64_t i = 0; i < S->n; ++i) {
        const or_km *k = &S->km[i];
        if (k->culled || k->tiles == 0) continue;
        km_ell el = km_ellipse(k->A, k->B, k->C);
        for (int ty = k->ty0; ty <= k->ty1; ++ty) {
            int f, l;
            if (!km_row_run(&el, k->u, k->v, k->tx0, k->tx1, ty, tile_w, tile_h, &f, &l))
                continue;
            for (int tx = f; tx <= l; ++tx) {
                uint64_t tile = (uint64_t)(ty * S->ntx + tx);
                keys[e].key = (tile << 32) | depth_bits(k->z);
                keys[e].idx = i;  /* record order == ascending slot */
                ++e;
            }
        }
    }
    {
        /* ties on the full key keep emission (record) order: sort on
         * (key, emission position) */
        kv_pair *kp = (kv_pair *)malloc(sizeof(kv_pair) * (e > 0 ? e : 1));
        int32_t *rec = (int32_t *)malloc(sizeof(int32_t) * (e > 0 ? e : 1));
        for (int64_t j = 0; j < e; ++j) { kp[j].key = keys[j].key; kp[j].idx = j; rec[j] = (int32_t)keys[j].idx; }
        qsort(kp, (size_t)e, sizeof(kv_pair), cmp_kv);
        int64_t nt = (int64_t)S->ntx * S->nty;
        S->tile_off = (int64_t *)calloc((size_t)nt + 1, sizeof(int64_t));
        S->tile_rec = (int32_t *)malloc(sizeof(int32_t) * (e > 0 ? e : 1));
        for (int64_t j = 0; j < e; ++j) {
            S->tile_rec[j] = rec[kp[j].idx];
            S->tile_off[(kp[j].key >> 32) + 1] += 1;
        }
        for (int64_t tI = 0; tI < nt; ++tI) S->tile_off[tI + 1] += S->tile_off[tI];
        free(kp); free(rec);
    }
    free(keys);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Eq. 3 for one pixel over an ordered candidate list.                       */
/* ------------------------------------------------------------------------ */

static void flag_or(uint8_t *p, uint8_t v)
{
#pragma omp atomic update
    *p |= v;
}

typedef struct {
    int32_t rec;     /* record index */
    double alpha, aU, G, T;  /* alpha used, unclamped o*G, G, T before */
    int clamped;
} or_hit;

/* Returns number of hits; *pos_last = 1 + list position of last included. */
static int blend_pixel(const or_vset *S, const int32_t *list, int64_t len, double px, double py,
                       const double bg[3], const or_bands *bd, double out[4],
                       int32_t *pos_last, int32_t *slot_last, uint8_t *flag,
                       or_hit *hits, uint8_t *rec_flag)
{
    double T = 1.0, C[3] = {0, 0, 0};
    int nh = 0;
    *pos_last = 0; *slot_last = -1; *flag = 0;
    for (int64_t j = 0; j < len; ++j) {
        int32_t r = list[j];
        const or_proj *P = &S->pj[r];
        double dx = px - P->u, dy = py - P->v;
        double m = P->A * dx * dx + 2.0 * P->B * dx * dy + P->C * dy * dy;
        if (bd && fabs(m - OR_MAHAL_MAX) <= bd->m * OR_MAHAL_MAX) {
            *flag |= 1; if (rec_flag) flag_or(&rec_flag[r], 1);
        }
        if (m > OR_MAHAL_MAX) continue;
        double G = exp(-0.5 * m);
        double aU = P->o * G;
        int clamped = aU > OR_ALPHA_MAX;
        double alpha = clamped ? OR_ALPHA_MAX : aU;
        if (bd && fabs(aU - OR_ALPHA_MAX) <= bd->clamp * OR_ALPHA_MAX) {
            *flag |= 2; if (rec_flag) flag_or(&rec_flag[r], 2);
        }
        if (bd && fabs(alpha - OR_ALPHA_MIN) <= bd->alpha * OR_ALPHA_MIN) {
            *flag |= 1; if (rec_flag) flag_or(&rec_flag[r], 1);
        }
        if (alpha < OR_ALPHA_MIN) continue;
        double tT = T * (1.0 - alpha);
        if (bd && fabs(tT - OR_T_STOP) <= bd->t_stop * OR_T_STOP) {
            *flag |= 1; if (rec_flag) flag_or(&rec_flag[r], 1);
        }
        if (tT < OR_T_STOP) break;
        if (hits) {
            hits[nh].rec = r; hits[nh].alpha = alpha; hits[nh].aU = aU;
            hits[nh].G = G; hits[nh].T = T; hits[nh].clamped = clamped;
        }
        ++nh;
        for (int ch = 0; ch < 3; ++ch) C[ch] += P->rgb[ch] * alpha * T;
        T = tT;
        *pos_last = (int32_t)(j + 1);
        *slot_last = S->slot[r];
    }
    for (int ch = 0; ch < 3; ++ch) out[ch] = C[ch] + T * bg[ch];
    out[3] = T;
    return nh;
}

/*
 * Render one view in FP64.
 *   mode 0: brute force -- every pixel walks the whole depth-ordered active
 *           set, no tiles;
 *   mode 1: tiled -- every pixel walks its tile's list.
 * rgb: [3,H,W] planar; T: [H,W]; last_slot: slot of the last included
 * Gaussian (-1: none); last_pos: 1 + tile-list position (mode 1 only);
 * flags: per-pixel near-discontinuity bits (1: value, 2: gradient only).
 * Returns 0 on success.
 */
int or_render(const or_scene *sc, const or_view *vw, const double bg[3], int32_t tile_w,
              int32_t tile_h, float near_plane, int32_t mode, const or_bands *bd,
              double *rgb, double *T, int32_t *last_slot, int32_t *last_pos, uint8_t *flags)
{
    or_vset S;
    if (vset_build(sc, vw, tile_w, tile_h, near_plane, mode == 1, &S)) { vset_free(&S); return -1; }
    const int W = vw->width, H = vw->height;
    const int64_t HW = (int64_t)W * H;
    if (mode == 0) {
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t pix = 0; pix < HW; ++pix) {
            int i = (int)(pix % W), j = (int)(pix / W);
            double out[4];
            int32_t pl, sl;
            uint8_t fl;
            blend_pixel(&S, S.order, S.n_order, i + 0.5, j + 0.5, bg, bd, out, &pl, &sl, &fl,
                        NULL, NULL);
            for (int ch = 0; ch < 3; ++ch) rgb[ch * HW + pix] = out[ch];
            T[pix] = out[3];
            last_slot[pix] = sl;
            if (last_pos) last_pos[pix] = -1;
            if (flags) flags[pix] = fl;
        }
    } else {
        const int64_t nt = (int64_t)S.ntx * S.nty;
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t tI = 0; tI < nt; ++tI) {
            int tx = (int)(tI % S.ntx), ty = (int)(tI / S.ntx);
            const int32_t *list = S.tile_rec + S.tile_off[tI];
            int64_t len = S.tile_off[tI + 1] - S.tile_off[tI];
            for (int j = ty * tile_h; j < (ty + 1) * tile_h && j < H; ++j)
                for (int i = tx * tile_w; i < (tx + 1) * tile_w && i < W; ++i) {
                    int64_t pix = (int64_t)j * W + i;
                    double out[4];
                    int32_t pl, sl;
                    uint8_t fl;
                    blend_pixel(&S, list, len, i + 0.5, j + 0.5, bg, bd, out, &pl, &sl, &fl,
                                NULL, NULL);
                    for (int ch = 0; ch < 3; ++ch) rgb[ch * HW + pix] = out[ch];
                    T[pix] = out[3];
                    last_slot[pix] = sl;
                    if (last_pos) last_pos[pix] = pl;
                    if (flags) flags[pix] = fl;
                }
        }
    }
    vset_free(&S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Every valid result of one pixel when the per-pair tests of Eq. 3 are      */
/* decided in a lower precision.                                              */
/* ------------------------------------------------------------------------ */

/* Near a threshold, an FP32 renderer can take the other side of a test that
 * FP64 decides one way: m <= 9 (the 3-sigma support), alpha >= 1/255, and the
 * stop rule T (1 - alpha) < 1e-4. Both outcomes are then valid renders of the
 * same rule. The walk below is the one of blend_pixel, but at every pair whose
 * FP64 test value lies within the band of its threshold it follows both
 * outcomes (depth first), each with its own running T, so later tests are
 * judged on that branch's own values. Every leaf is one valid (rgb, T, last).
 * The 0.99 clamp is continuous in value and is not branched. */
typedef struct {
    const or_vset *S;
    const int32_t *list;
    int64_t len;
    double px, py;
    const double *bg;
    const or_bands *bd;
    int32_t max_out, n_out, overflow;
    double *out;      /* [max_out, 4]: rgb, T */
    int32_t *last;    /* [max_out] */
} var_walk;

static void var_leaf(var_walk *w, const double C[3], double T, int32_t last)
{
    if (w->n_out >= w->max_out) { w->overflow = 1; return; }
    double *o = w->out + 4 * (int64_t)w->n_out;
    for (int ch = 0; ch < 3; ++ch) o[ch] = C[ch] + T * w->bg[ch];
    o[3] = T;
    w->last[w->n_out] = last;
    w->n_out += 1;
}

static void var_step(var_walk *w, int64_t j, double T, const double Cin[3], int32_t last)
{
    double C[3] = {Cin[0], Cin[1], Cin[2]};
    for (; j < w->len; ++j) {
        if (w->overflow) return;
        const or_proj *P = &w->S->pj[w->list[j]];
        double dx = w->px - P->u, dy = w->py - P->v;
        double m = P->A * dx * dx + 2.0 * P->B * dx * dy + P->C * dy * dy;
        int pass = m <= OR_MAHAL_MAX;
        if (fabs(m - OR_MAHAL_MAX) <= w->bd->m * OR_MAHAL_MAX) {
            /* both outcomes of the support test: skipped (recursion), inside (below) */
            var_step(w, j + 1, T, C, last);
            pass = 1;
        }
        if (!pass) continue;
        double aU = P->o * exp(-0.5 * m);
        double alpha = aU > OR_ALPHA_MAX ? OR_ALPHA_MAX : aU;
        int big = alpha >= OR_ALPHA_MIN;
        if (fabs(alpha - OR_ALPHA_MIN) <= w->bd->alpha * OR_ALPHA_MIN) {
            /* both outcomes of the alpha test */
            var_step(w, j + 1, T, C, last);
            big = 1;
        }
        if (!big) continue;
        double tT = T * (1.0 - alpha);
        int stop = tT < OR_T_STOP;
        if (fabs(tT - OR_T_STOP) <= w->bd->t_stop * OR_T_STOP) {
            /* both: stop here, and include it and go on */
            var_leaf(w, C, T, last);
            stop = 0;
        }
        if (stop) { var_leaf(w, C, T, last); return; }
        for (int ch = 0; ch < 3; ++ch) C[ch] += P->rgb[ch] * alpha * T;
        T = tT;
        last = (int32_t)(j + 1);
    }
    var_leaf(w, C, T, last);
}

/* For n pixels (px, py) of one view in tiled mode: up to max_per valid
 * results each (out[k, i] = rgb[3], T; last[k, i] = 1 + tile-list position of
 * the last included Gaussian), count[k] = the number written, or -1 when the
 * pixel has more than max_per. Returns 0 on success. */
int or_render_variants(const or_scene *sc, const or_view *vw, const double bg[3],
                       int32_t tile_w, int32_t tile_h, float near_plane, const or_bands *bd,
                       int64_t n, const int32_t *px, const int32_t *py, int32_t max_per,
                       double *out, int32_t *last, int32_t *count)
{
    or_vset S;
    if (vset_build(sc, vw, tile_w, tile_h, near_plane, 1, &S)) { vset_free(&S); return -1; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < n; ++k) {
        const int64_t tI = (int64_t)(py[k] / tile_h) * S.ntx + px[k] / tile_w;
        var_walk w;
        w.S = &S;
        w.list = S.tile_rec + S.tile_off[tI];
        w.len = S.tile_off[tI + 1] - S.tile_off[tI];
        w.px = px[k] + 0.5;
        w.py = py[k] + 0.5;
        w.bg = bg;
        w.bd = bd;
        w.max_out = max_per;
        w.n_out = 0;
        w.overflow = 0;
        w.out = out + 4 * k * (int64_t)max_per;
        w.last = last + k * (int64_t)max_per;
        const double C0[3] = {0.0, 0.0, 0.0};
        var_step(&w, 0, 1.0, C0, 0);
        count[k] = w.overflow ? -1 : w.n_out;
    }
    vset_free(&S);
    return 0;
}

/* Render selected pixels only (brute force), for sampled checks at full size.
 * px, py: pixel indices; out: [n,3] rgb, T[n], last_slot[n], flags[n]. */
int or_render_pixels(const or_scene *sc, const or_view *vw, const double bg[3], float near_plane,
                     const or_bands *bd, int64_t n, const int32_t *px, const int32_t *py,
                     double *rgb, double *T, int32_t *last_slot, uint8_t *flags)
{
    or_vset S;
    if (vset_build(sc, vw, 16, 16, near_plane, 0, &S)) { vset_free(&S); return -1; }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t k = 0; k < n; ++k) {
        double out[4];
        int32_t pl, sl;
        uint8_t fl;
        blend_pixel(&S, S.order, S.n_order, px[k] + 0.5, py[k] + 0.5, bg, bd, out, &pl, &sl, &fl,
                    NULL, NULL);
        for (int ch = 0; ch < 3; ++ch) rgb[3 * k + ch] = out[ch];
        T[k] = out[3];
        last_slot[k] = sl;
        if (flags) flags[k] = fl;
    }
    vset_free(&S);
    return 0;
}

/* Key-mode records and per-tile sorted lists of one view, for the
 * bit-exact checks. ids: [n_active]; km: [n_active]; returns n_active.
 * tile_off: [ntx*nty+1] and tile_slot: [n_keys] if non-NULL (caller sizes them
 * from a first call with tile_off == NULL; *n_keys receives the key count). */
int64_t or_view_lists(const or_scene *sc, const or_view *vw, int32_t tile_w, int32_t tile_h,
                      float near_plane, int32_t *ids, or_km *km, int64_t *n_keys,
                      int64_t *tile_off, int32_t *tile_slot)
{
    or_vset S;
    if (vset_build(sc, vw, tile_w, tile_h, near_plane, tile_off != NULL, &S)) {
        vset_free(&S); return -1;
    }
    int64_t keys = 0;
    for (int64_t i = 0; i < S.n; ++i) {
        if (ids) ids[i] = S.slot[i];
        if (km) km[i] = S.km[i];
        if (!S.km[i].culled) keys += S.km[i].tiles;
    }
    if (n_keys) *n_keys = keys;
    if (tile_off) {
        int64_t nt = (int64_t)S.ntx * S.nty;
        for (int64_t t = 0; t <= nt; ++t) tile_off[t] = S.tile_off[t];
        for (int64_t j = 0; j < keys; ++j) tile_slot[j] = S.slot[S.tile_rec[j]];
    }
    int64_t n = S.n;
    vset_free(&S);
    return n;
}

/* ------------------------------------------------------------------------ */
/* Backward (Alg. 1 loss.backward): analytic adjoint of the tiled forward.    */
/* ------------------------------------------------------------------------ */

typedef struct {
    double *means, *log_scales, *quats, *logits, *sh;   /* [N,...] FP64 grads */
} or_grads;

static void atomic_add(double *p, double v)
{
#pragma omp atomic
    *p += v;
}

/* Chain rule from the 2D quantities of one record to the Gaussian's
 * parameters (projection backward). g2: du, dv, dA, dB, dC, do, dr, dg, db. */
static void project_backward(const or_scene *sc, const or_view *vw, int64_t slot,
                             const or_proj *P, const double g2[9], or_grads *G)
{
    int K = sh_count(sc->sh_degree);
    double W[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) W[i][j] = vw->R[3 * i + j];
    double fx = vw->fx, fy = vw->fy, z = P->z;
    double gmu[3] = {0, 0, 0};
    /* opacity */
    atomic_add(&G->logits[slot], g2[5] * P->o * (1.0 - P->o));
    /* colour -> SH coefficients and view direction */
    double gdir[3] = {0, 0, 0};
    const float *sh = sc->sh + (int64_t)slot * K * 3;
    for (int ch = 0; ch < 3; ++ch) {
        if (!(P->raw[ch] > 0.0)) continue;
        double gc = g2[6 + ch];
        for (int k = 0; k < K; ++k) {
            atomic_add(&G->sh[((int64_t)slot * K + k) * 3 + ch], P->Y[k] * gc);
            for (int a = 0; a < 3; ++a) gdir[a] += gc * sh[3 * k + ch] * P->dY[k][a];
        }
    }
    {
        double dd = P->dir[0] * gdir[0] + P->dir[1] * gdir[1] + P->dir[2] * gdir[2];
        for (int a = 0; a < 3; ++a) gmu[a] += (gdir[a] - P->dir[a] * dd) / P->dist;
    }
    /* conic (A,B,C) -> dilated covariance: d(S^-1) = -S^-1 dS S^-1 */
    double Ci[2][2] = {{P->A, P->B}, {P->B, P->C}};
    double Gc[2][2] = {{g2[2], 0.5 * g2[3]}, {0.5 * g2[3], g2[4]}};
    double tmp[2][2], Gcov[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) tmp[i][j] = Ci[i][0] * Gc[0][j] + Ci[i][1] * Gc[1][j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) Gcov[i][j] = -(tmp[i][0] * Ci[0][j] + tmp[i][1] * Ci[1][j]);
    /* cov = T Sigma T^T: dSigma = T^T Gcov T, dT = 2 Gcov T Sigma */
    double GS[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) s += P->Tm[a][i] * Gcov[a][b] * P->Tm[b][j];
            GS[i][j] = s;
        }
    double GT[2][3];
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int b = 0; b < 2; ++b)
                for (int k = 0; k < 3; ++k) s += Gcov[a][b] * P->Tm[b][k] * P->Sg[k][j];
            GT[a][j] = 2.0 * s;
        }
    /* T = J W: dJ = dT W^T */
    double GJ[2][3];
    for (int a = 0; a < 2; ++a)
        for (int k = 0; k < 3; ++k) {
            double s = 0.0;
            for (int j = 0; j < 3; ++j) s += GT[a][j] * W[k][j];
            GJ[a][k] = s;
        }
    /* J(p) with the guard band */
    double gp[3] = {0, 0, 0};
    double z2 = z * z, z3 = z2 * z;
    gp[2] += GJ[0][0] * (-fx / z2) + GJ[1][1] * (-fy / z2)
           + GJ[0][2] * (2.0 * fx * P->tx / z3) + GJ[1][2] * (2.0 * fy * P->ty / z3);
    double gtx = GJ[0][2] * (-fx / z2);
    double gty = GJ[1][2] * (-fy / z2);
    if (P->clampx == 0.0) gp[0] += gtx; else gp[2] += gtx * P->clampx * P->limx;
    if (P->clampy == 0.0) gp[1] += gty; else gp[2] += gty * P->clampy * P->limy;
    /* projected centre */
    gp[0] += g2[0] * fx / z;
    gp[2] += g2[0] * (-fx * P->p[0] / z2);
    gp[1] += g2[1] * fy / z;
    gp[2] += g2[1] * (-fy * P->p[1] / z2);
    /* p = W mu + t */
    for (int j = 0; j < 3; ++j) gmu[j] += W[0][j] * gp[0] + W[1][j] * gp[1] + W[2][j] * gp[2];
    for (int j = 0; j < 3; ++j) atomic_add(&G->means[3 * slot + j], gmu[j]);
    /* Sigma = M M^T: dM = 2 dSigma M (dSigma symmetric) */
    double GM[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += (GS[i][k] + GS[k][i]) * P->M[k][j];
            GM[i][j] = s;
        }
    /* M = Rq diag(s) */
    double GR[3][3];
    for (int j = 0; j < 3; ++j) {
        double gs = 0.0;
        for (int i = 0; i < 3; ++i) { gs += P->Rq[i][j] * GM[i][j]; GR[i][j] = P->s[j] * GM[i][j]; }
        atomic_add(&G->log_scales[3 * slot + j], gs * P->s[j]);
    }
    /* Rq(q/|q|) */
    double w = P->qn[0], x = P->qn[1], y = P->qn[2], zq = P->qn[3];
    double gq[4];
    gq[0] = 2 * (-zq * GR[0][1] + y * GR[0][2] + zq * GR[1][0] - x * GR[1][2] - y * GR[2][0] + x * GR[2][1]);
    gq[1] = 2 * (y * GR[0][1] + zq * GR[0][2] + y * GR[1][0] - 2 * x * GR[1][1] - w * GR[1][2]
                 + zq * GR[2][0] + w * GR[2][1] - 2 * x * GR[2][2]);
    gq[2] = 2 * (-2 * y * GR[0][0] + x * GR[0][1] + w * GR[0][2] + x * GR[1][0] + zq * GR[1][2]
                 - w * GR[2][0] + zq * GR[2][1] - 2 * y * GR[2][2]);
    gq[3] = 2 * (-2 * zq * GR[0][0] - w * GR[0][1] + x * GR[0][2] + w * GR[1][0] - 2 * zq * GR[1][1]
                 + y * GR[1][2] + x * GR[2][0] + y * GR[2][1]);
    double dq = w * gq[0] + x * gq[1] + y * gq[2] + zq * gq[3];
    for (int k = 0; k < 4; ++k) atomic_add(&G->quats[4 * slot + k], (gq[k] - P->qn[k] * dq) / P->qnorm);
}

/*
 * Backward of one view's tiled FP64 render for dL/dC given as FP64 planar
 * [3,H,W]. Accumulates into the FP64 parameter grads for non-frozen slots.
 * grad2d (optional): [n_active, 9] per-record 2D grads in active-id order.
 * rec_flags (optional): [n_active] bits: 1 value-discontinuity, 2 clamp,
 *   4 guard band, 8 colour clamp (near the discontinuities of the derivative).
 */
int or_render_bwd(const or_scene *sc, const or_view *vw, const double bg[3], int32_t tile_w,
                  int32_t tile_h, float near_plane, const double *dLdC, const or_bands *bd,
                  or_grads *G, double *grad2d, uint8_t *rec_flags)
{
    or_vset S;
    if (vset_build(sc, vw, tile_w, tile_h, near_plane, 1, &S)) { vset_free(&S); return -1; }
    const int Wd = vw->width, H = vw->height;
    const int64_t HW = (int64_t)Wd * H;
    double *g2 = (double *)calloc((size_t)(S.n > 0 ? S.n : 1) * 9, sizeof(double));
    uint8_t *rf = (uint8_t *)calloc((size_t)(S.n > 0 ? S.n : 1), 1);
    int64_t maxlen = 0;
    const int64_t nt = (int64_t)S.ntx * S.nty;
    for (int64_t t = 0; t < nt; ++t)
        if (S.tile_off[t + 1] - S.tile_off[t] > maxlen) maxlen = S.tile_off[t + 1] - S.tile_off[t];
#pragma omp parallel
    {
        or_hit *hits = (or_hit *)malloc(sizeof(or_hit) * (maxlen > 0 ? maxlen : 1));
#pragma omp for schedule(dynamic, 1)
        for (int64_t tI = 0; tI < nt; ++tI) {
            int tx = (int)(tI % S.ntx), ty = (int)(tI / S.ntx);
            const int32_t *list = S.tile_rec + S.tile_off[tI];
            int64_t len = S.tile_off[tI + 1] - S.tile_off[tI];
            for (int j = ty * tile_h; j < (ty + 1) * tile_h && j < H; ++j)
                for (int i = tx * tile_w; i < (tx + 1) * tile_w && i < Wd; ++i) {
                    int64_t pix = (int64_t)j * Wd + i;
                    double out[4];
                    int32_t pl, sl;
                    uint8_t fl;
                    double px = i + 0.5, py = j + 0.5;
                    int nh = blend_pixel(&S, list, len, px, py, bg, bd, out, &pl, &sl, &fl, hits, rf);
                    double gC[3] = {dLdC[pix], dLdC[HW + pix], dLdC[2 * HW + pix]};
                    /* colour behind each hit: B_last = bg, B_{i-1} = a_i c_i + (1-a_i) B_i */
                    double Bk[3] = {bg[0], bg[1], bg[2]};
                    for (int h = nh - 1; h >= 0; --h) {
                        const or_hit *hh = &hits[h];
                        const or_proj *P = &S.pj[hh->rec];
                        double gl[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                        double ga = 0.0;
                        for (int ch = 0; ch < 3; ++ch) {
                            gl[6 + ch] = hh->alpha * hh->T * gC[ch];
                            ga += gC[ch] * (P->rgb[ch] - Bk[ch]) * hh->T;
                        }
                        if (!hh->clamped) {
                            double dx = px - P->u, dy = py - P->v;
                            gl[5] = hh->G * ga;                 /* d alpha / d o = G */
                            double gm = -0.5 * hh->aU * ga;     /* d alpha / d m */
                            gl[2] = gm * dx * dx;
                            gl[3] = gm * 2.0 * dx * dy;
                            gl[4] = gm * dy * dy;
                            gl[0] = gm * (-2.0) * (P->A * dx + P->B * dy);
                            gl[1] = gm * (-2.0) * (P->B * dx + P->C * dy);
                        }
                        for (int k = 0; k < 9; ++k) atomic_add(&g2[9 * hh->rec + k], gl[k]);
                        for (int ch = 0; ch < 3; ++ch)
                            Bk[ch] = hh->alpha * P->rgb[ch] + (1.0 - hh->alpha) * Bk[ch];
                    }
                }
        }
        free(hits);
    }
    for (int64_t r = 0; r < S.n; ++r) {
        if (S.km[r].culled) continue;
        const or_proj *P = &S.pj[r];
        if (bd) {
            if (fabs(fabs(P->xz) - P->limx) <= bd->guard * P->limx) rf[r] |= 4;
            if (fabs(fabs(P->yz) - P->limy) <= bd->guard * P->limy) rf[r] |= 4;
            for (int ch = 0; ch < 3; ++ch)
                if (fabs(P->raw[ch]) <= bd->colour) rf[r] |= 8;
        }
        if (grad2d) for (int k = 0; k < 9; ++k) grad2d[9 * r + k] = g2[9 * r + k];
        if (rec_flags) rec_flags[r] = rf[r];
        if (sc->frozen && sc->frozen[S.slot[r]]) continue;
        project_backward(sc, vw, S.slot[r], P, &g2[9 * r], G);
    }
    if (rec_flags) for (int64_t r = 0; r < S.n; ++r) if (S.km[r].culled) rec_flags[r] = 0;
    free(g2); free(rf);
    vset_free(&S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Counter-based RNG: Philox4x64-10 (Salmon et al., SC'11).                  */
/* ------------------------------------------------------------------------ */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void or_philox4x64(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c[0], &hi0, &lo0);
        mulhilo64(M1, c[2], &hi1, &lo1);
        uint64_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

/* Stream tags: one key word per purpose so the streams never overlap. */
#define OR_TAG_NOISE 0x53474c44ULL   /* "SGLD" */
#define OR_TAG_RELOC 0x52454c4fULL   /* "RELO" */

/* Three N(0,1) draws for (seed, step, slot) by Box-Muller on the top 24 bits
 * of each 64-bit word, u in (0, 1]. */
void or_normal3(uint64_t seed, uint64_t step, int64_t slot, double out[3])
{
    uint64_t ctr[4] = {(uint64_t)slot, step, 0, 0}, key[2] = {seed, OR_TAG_NOISE}, r[4];
    or_philox4x64(ctr, key, r);
    double u[4];
    for (int i = 0; i < 4; ++i) u[i] = ((double)(r[i] >> 40) + 1.0) * (1.0 / 16777216.0);
    const double TWO_PI = 6.28318530717958647692;
    double r0 = sqrt(-2.0 * log(u[0])), r1 = sqrt(-2.0 * log(u[2]));
    out[0] = r0 * cos(TWO_PI * u[1]);
    out[1] = r0 * sin(TWO_PI * u[1]);
    out[2] = r1 * cos(TWO_PI * u[3]);
}

/* ------------------------------------------------------------------------ */
/* Optimiser step, SGLD noise and relocation (Alg. 1 steps after backward).  */
/* ------------------------------------------------------------------------ */

typedef struct {
    float lr_means, lr_log_scales, lr_quats, lr_logits, lr_sh_dc, lr_sh_rest;
    float beta1, beta2, eps;
    float noise_lr;          /* Sec. 8.1: 5e4 */
    float noise_k, noise_t;  /* sigmoid sharpness and opacity threshold of the noise gate */
    int32_t adam;            /* 1: Adam step before the noise */
    int32_t relocate;        /* 1: relocate dead Gaussians after the noise */
    int32_t max_n;           /* cap on N in the relocation formulas */
} or_sgld_params;

typedef struct {
    float *means, *log_scales, *quats, *logits, *sh;       /* updated in place */
    const int32_t *start, *expire;
    const uint8_t *frozen;
    int64_t n;
    int32_t sh_degree;
} or_state;

typedef struct {
    float *m_means, *v_means, *m_log_scales, *v_log_scales, *m_quats, *v_quats,
          *m_logits, *v_logits, *m_sh, *v_sh;
} or_adam;

typedef struct {
    const float *means, *log_scales, *quats, *logits, *sh;
} or_fgrads;

static int eligible(const or_state *st, int64_t i, const int32_t *frames, int32_t nf)
{
    if (st->frozen && st->frozen[i]) return 0;
    for (int32_t f = 0; f < nf; ++f)
        if (st->start[i] <= frames[f] && frames[f] < st->expire[i]) return 1;
    return 0;
}

static void adam_one(float *p, float *m, float *v, float g, double lr, const or_sgld_params *pr,
                     double bc1, double bc2)
{
    double mm = pr->beta1 * (double)*m + (1.0 - pr->beta1) * g;
    double vv = pr->beta2 * (double)*v + (1.0 - pr->beta2) * (double)g * g;
    double mh = mm / bc1, vh = vv / bc2;
    *p = (float)((double)*p - lr * mh / (sqrt(vh) + pr->eps));
    *m = (float)mm;
    *v = (float)vv;
}

/* Same exp construction as km_exp but in FP64 (degree 13); used only where an
 * integer is derived from a float (relocation weights). */
static double kd_exp(double x)
{
    const double L2E = 0x1.71547652b82fep+0;
    const double LN2_HI = 0x1.62e42feep-1;
    const double LN2_LO = 0x1.a39ef35793c76p-33;
    static const double P[14] = {
        0x1p+0, 0x1p+0, 0x1p-1, 0x1.5555555555555p-3, 0x1.5555555555555p-5,
        0x1.1111111111111p-7, 0x1.6c16c16c16c17p-10, 0x1.a01a01a01a01ap-13,
        0x1.a01a01a01a01ap-16, 0x1.71de3a556c734p-19, 0x1.27e4fb7789f5cp-22,
        0x1.ae64567f544e4p-26, 0x1.1eed8eff8d898p-29, 0x1.6124613a86d09p-33};
    if (x < -700.0) x = -700.0;
    if (x > 700.0) x = 700.0;
    double t = x * L2E;
    t = t + 0.5;
    double k = floor(t);
    double h = k * LN2_HI;
    double r = x - h;
    double l = k * LN2_LO;
    r = r - l;
    double p = P[13];
    for (int i = 12; i >= 0; --i) { p = p * r; p = p + P[i]; }
    return ldexp(p, (int)k);
}

/* Relocation weight of an alive Gaussian: floor(sigmoid(logit) * 2^32). */
uint64_t or_reloc_weight(float logit)
{
    double e = kd_exp(-(double)logit);
    double den = 1.0 + e;
    double o = 1.0 / den;
    double w = floor(o * 4294967296.0);
    if (w > 4294967295.0) w = 4294967295.0;
    return (uint64_t)w;
}

/* Dead: sigmoid(logit) <= 0.005, decided on the FP32 logit against the largest
 * float not above ln(0.005/0.995). */
#define OR_LOGIT_DEAD (-0x1.52c582p+2f)

static double binom(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

/* 3DGS-MCMC relocation of N copies: o' = 1 - (1-o)^(1/N) and
 * s' = s * o / sum_{i=1..N} sum_{k=0..i-1} C(i-1,k) (-1)^k o'^(k+1) / sqrt(k+1). */
void or_reloc_values(double o, int n, double *o_new, double *scale_ratio)
{
    double on = 1.0 - pow(1.0 - o, 1.0 / n);
    double den = 0.0;
    for (int i = 1; i <= n; ++i)
        for (int k = 0; k <= i - 1; ++k)
            den += binom(i - 1, k) * ((k & 1) ? -1.0 : 1.0) * pow(on, k + 1) / sqrt(k + 1.0);
    *o_new = on;
    *scale_ratio = o / den;
}

/*
 * One optimiser + SGLD (+ relocation) step on the Gaussians eligible at the
 * frames of this step (active at any of them and not frozen).
 *  1. optional Adam step from grads (bias-corrected, step count = step + 1);
 *  2. noise mu += lr_means * noise_lr * sigmoid(-k (o - t)) * Sigma eta;
 *  3. optional relocation of dead (o <= 0.005) onto alive Gaussians sampled in
 *     proportion to opacity (integer CDF), with Adam moments of all touched
 *     slots reset.
 * Returns the number of relocated (dead) slots; targets[i] receives the
 * target slot of dead slot i (-1 otherwise) when non-NULL.
 */
int64_t or_sgld_step(or_state *st, const or_fgrads *g, or_adam *ad, const int32_t *frames,
                     int32_t nf, const or_sgld_params *pr, uint64_t seed, uint64_t step,
                     int32_t *targets)
{
    const int64_t N = st->n;
    const int K = sh_count(st->sh_degree);
    uint8_t *el = (uint8_t *)malloc((size_t)(N > 0 ? N : 1));
    for (int64_t i = 0; i < N; ++i) el[i] = (uint8_t)eligible(st, i, frames, nf);
    if (pr->adam) {
        double bc1 = 1.0 - pow(pr->beta1, (double)(step + 1));
        double bc2 = 1.0 - pow(pr->beta2, (double)(step + 1));
        for (int64_t i = 0; i < N; ++i) {
            if (!el[i]) continue;
            for (int j = 0; j < 3; ++j) {
                adam_one(&st->means[3 * i + j], &ad->m_means[3 * i + j], &ad->v_means[3 * i + j],
                         g->means[3 * i + j], pr->lr_means, pr, bc1, bc2);
                adam_one(&st->log_scales[3 * i + j], &ad->m_log_scales[3 * i + j],
                         &ad->v_log_scales[3 * i + j], g->log_scales[3 * i + j], pr->lr_log_scales,
                         pr, bc1, bc2);
            }
            for (int j = 0; j < 4; ++j)
                adam_one(&st->quats[4 * i + j], &ad->m_quats[4 * i + j], &ad->v_quats[4 * i + j],
                         g->quats[4 * i + j], pr->lr_quats, pr, bc1, bc2);
            adam_one(&st->logits[i], &ad->m_logits[i], &ad->v_logits[i], g->logits[i],
                     pr->lr_logits, pr, bc1, bc2);
            for (int k = 0; k < K; ++k)
                for (int ch = 0; ch < 3; ++ch) {
                    int64_t e = ((int64_t)i * K + k) * 3 + ch;
                    adam_one(&st->sh[e], &ad->m_sh[e], &ad->v_sh[e], g->sh[e],
                             k == 0 ? pr->lr_sh_dc : pr->lr_sh_rest, pr, bc1, bc2);
                }
        }
    }
    /* noise, from the (possibly updated) opacity and covariance */
    for (int64_t i = 0; i < N; ++i) {
        if (!el[i]) continue;
        double o = 1.0 / (1.0 + exp(-(double)st->logits[i]));
        double gate = 1.0 / (1.0 + exp(pr->noise_k * (o - pr->noise_t)));
        double s[3];
        for (int j = 0; j < 3; ++j) s[j] = exp((double)st->log_scales[3 * i + j]);
        double q[4] = {st->quats[4 * i], st->quats[4 * i + 1], st->quats[4 * i + 2], st->quats[4 * i + 3]};
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
        double Rq[3][3] = {
            {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
            {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
            {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
        double Sg[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += Rq[a][k] * s[k] * s[k] * Rq[b][k];
                Sg[a][b] = acc;
            }
        double eta[3];
        or_normal3(seed, step, i, eta);
        double scale = (double)pr->lr_means * pr->noise_lr * gate;
        for (int a = 0; a < 3; ++a) {
            double d = Sg[a][0] * eta[0] + Sg[a][1] * eta[1] + Sg[a][2] * eta[2];
            st->means[3 * i + a] = (float)((double)st->means[3 * i + a] + scale * d);
        }
    }
    int64_t n_dead = 0;
    if (targets) for (int64_t i = 0; i < N; ++i) targets[i] = -1;
    if (pr->relocate) {
        /* integer CDF over alive eligible Gaussians, in slot order */
        uint64_t *cdf = (uint64_t *)malloc(sizeof(uint64_t) * (N > 0 ? N : 1));
        uint64_t acc = 0;
        for (int64_t i = 0; i < N; ++i) {
            uint64_t w = 0;
            if (el[i] && !(st->logits[i] <= OR_LOGIT_DEAD)) w = or_reloc_weight(st->logits[i]);
            acc += w;
            cdf[i] = acc;
        }
        int32_t *tgt = (int32_t *)malloc(sizeof(int32_t) * (N > 0 ? N : 1));
        int32_t *cnt = (int32_t *)calloc((size_t)(N > 0 ? N : 1), sizeof(int32_t));
        for (int64_t i = 0; i < N; ++i) {
            tgt[i] = -1;
            if (!el[i] || !(st->logits[i] <= OR_LOGIT_DEAD) || acc == 0) continue;
            uint64_t ctr[4] = {(uint64_t)i, step, 0, 0}, key[2] = {seed, OR_TAG_RELOC}, r[4];
            or_philox4x64(ctr, key, r);
            uint64_t xh, xl;
            mulhilo64(r[0], acc, &xh, &xl);   /* floor(r * total / 2^64) in [0, total) */
            /* first j with cdf[j] > xh */
            int64_t lo = 0, hi = N - 1;
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (cdf[mid] > xh) hi = mid; else lo = mid + 1;
            }
            tgt[i] = (int32_t)lo;
            cnt[lo] += 1;
            ++n_dead;
        }
        /* new values from the targets' current state */
        float *new_logit = (float *)malloc(sizeof(float) * (N > 0 ? N : 1));
        float *new_ls = (float *)malloc(sizeof(float) * 3 * (N > 0 ? N : 1));
        for (int64_t j = 0; j < N; ++j) {
            if (cnt[j] == 0) continue;
            int nn = cnt[j] + 1;
            if (nn > pr->max_n) nn = pr->max_n;
            double o = 1.0 / (1.0 + exp(-(double)st->logits[j]));
            double on, ratio;
            or_reloc_values(o, nn, &on, &ratio);
            new_logit[j] = (float)log(on / (1.0 - on));
            for (int a = 0; a < 3; ++a)
                new_ls[3 * j + a] = (float)((double)st->log_scales[3 * j + a] + log(ratio));
        }
        /* dead copies the target (with its new opacity and scale) */
        for (int64_t i = 0; i < N; ++i) {
            int32_t j = tgt[i];
            if (j < 0) continue;
            for (int a = 0; a < 3; ++a) {
                st->means[3 * i + a] = st->means[3 * j + a];
                st->log_scales[3 * i + a] = new_ls[3 * j + a];
            }
            for (int a = 0; a < 4; ++a) st->quats[4 * i + a] = st->quats[4 * j + a];
            st->logits[i] = new_logit[j];
            for (int e = 0; e < 3 * K; ++e) st->sh[(int64_t)i * 3 * K + e] = st->sh[(int64_t)j * 3 * K + e];
            if (targets) targets[i] = j;
        }
        for (int64_t j = 0; j < N; ++j) {
            if (cnt[j] == 0) continue;
            st->logits[j] = new_logit[j];
            for (int a = 0; a < 3; ++a) st->log_scales[3 * j + a] = new_ls[3 * j + a];
        }
        /* reset optimiser moments of every touched slot */
        if (ad) {
            for (int64_t i = 0; i < N; ++i) {
                if (tgt[i] < 0 && cnt[i] == 0) continue;
                for (int a = 0; a < 3; ++a) {
                    ad->m_means[3 * i + a] = ad->v_means[3 * i + a] = 0.0f;
                    ad->m_log_scales[3 * i + a] = ad->v_log_scales[3 * i + a] = 0.0f;
                }
                for (int a = 0; a < 4; ++a) ad->m_quats[4 * i + a] = ad->v_quats[4 * i + a] = 0.0f;
                ad->m_logits[i] = ad->v_logits[i] = 0.0f;
                for (int e = 0; e < 3 * K; ++e)
                    ad->m_sh[(int64_t)i * 3 * K + e] = ad->v_sh[(int64_t)i * 3 * K + e] = 0.0f;
            }
        }
        free(cdf); free(tgt); free(cnt); free(new_logit); free(new_ls);
    }
    free(el);
    return n_dead;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops from now on (n >= 1); used to time the
 * oracle single-threaded beside its all-core run. */
void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}


/*
 * Table 6 opacity code (uint8): k = rint(255 sigmoid(logit)), the sigmoid
 * computed in FP32 through the key-mode exp above so that the integer does not
 * depend on a library's exp. Round half to even (rintf, default mode).
 */
void or_opacity_u8(const float *logits, int64_t n, uint8_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        float e = km_exp(-logits[i]);
        float den = 1.0f + e;
        float o = 1.0f / den;
        float t = o * 255.0f;
        float k = rintf(t);
        if (k < 0.0f) k = 0.0f;
        if (k > 255.0f) k = 255.0f;
        out[i] = (uint8_t)k;
    }
}
