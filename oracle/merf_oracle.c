/* merf_oracle.c -- plain FP64 CPU oracle of the MERF real-time renderer.
 *
 * TEST INFRASTRUCTURE ONLY: only tests, the smoke check and the benchmark's oracle leg and
 * reference arm may build, load or call this file.  The product (the CUDA library) never does.
 *
 * It computes, per pixel ray and with no empty-space hierarchy and no other acceleration,
 * exactly what the paper defines:
 *   ray  x(t) = o + t d                                             (Sec. 2, Eq. 1)
 *   contraction contract_pi, seven regions                          (Sec. 3.2)
 *   the contracted ray as straight segments, a uniform lattice of samples in contracted
 *   arc length, a sample evaluated iff its finest occupancy cell is set (Sec. 4.3, Sec. 5)
 *   field t~ = V + P_x + P_y + P_z, trilinear / bilinear            (Sec. 3.1, Eq. 3)
 *   (grid-only scenes, R = 0: t~ = V, the SNeRG++-style baseline of Sec. 6)
 *   dequantisation 2 m k / 255 - m, m = 14 density, 7 otherwise     (Sec. 4.2)
 *   tau = exp(t~_0), c_d = sigmoid(t~_1..3), f = sigmoid(t~_4..7)   (Sec. 3.1, Eq. 4)
 *   front-to-back quadrature of C_d and F, T < 2e-4 termination      (Eq. 1, Eq. 2, Sec. 5)
 *   C = C_d + h(C_d, F, d), h a 3-layer MLP with 16 hidden units   (Sec. 2, App. B)
 * Readings where the paper is silent (lattice phase, step length in world units, tie
 * rule of the contraction, texel centres, missing blocks, posenc layout) follow the
 * library's documented conventions; each is restated at the function that takes it.
 *
 * Every floating-point value is double, except in the orc32_* functions: those restate,
 * in float, the decisions the kernel takes in float (which lattice samples exist and which
 * occupancy cell each falls in), so that an integer outcome decided in FP32 can be
 * compared exactly.  They are the only FP32 code here and are used only when a caller
 * asks for FP32 decisions.
 *
 * Pins: tests/test_oracle_*.py check every function against closed forms, hand-derived
 * values of the contraction equation, brute-force dense sampling and textbook routines.
 */
#include "merf_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* contraction, Sec. 3.2                                                                 */

/* Region of a world point: 0 inside the unit cube (|x|_inf <= 1), else 1 + 2 j + (x_j < 0)
 * with j the coordinate of largest magnitude.  Reading of the paper's garbled conditions:
 * "x_j = |x|_inf" means |x_j| = |x|_inf; on ties |x_j| = |x_k| the lowest axis index wins. */
int orc_region(const double x[3])
{
    int j = 0;
    double ax = fabs(x[0]);
    for (int a = 1; a < 3; ++a)
        if (fabs(x[a]) > ax) { ax = fabs(x[a]); j = a; }
    if (ax <= 1.0) return 0;
    return 1 + 2 * j + (x[j] < 0.0 ? 1 : 0);
}

/* The projective map of one region applied to x (x need not lie in that region). */
void orc_contract_in_region(int region, const double x[3], double p[3])
{
    if (region == 0) { p[0] = x[0]; p[1] = x[1]; p[2] = x[2]; return; }
    int j = (region - 1) / 2;
    double s = ((region - 1) & 1) ? -1.0 : 1.0;
    double ax = fabs(x[j]);
    for (int k = 0; k < 3; ++k) p[k] = x[k] / ax;          /* x_k / |x|_inf */
    p[j] = (2.0 - 1.0 / ax) * s;                            /* (2 - 1/|x_j|) x_j/|x_j| */
}

void orc_contract(const double x[3], double p[3])
{
    orc_contract_in_region(orc_region(x), x, p);
}

/* Inverse of one region's map: |x_j| = 1 / (2 - |p_j|), x_k = p_k |x_j|. */
void orc_uncontract(int region, const double p[3], double x[3])
{
    if (region == 0) { x[0] = p[0]; x[1] = p[1]; x[2] = p[2]; return; }
    int j = (region - 1) / 2;
    double s = ((region - 1) & 1) ? -1.0 : 1.0;
    double ax = 1.0 / (2.0 - s * p[j]);
    for (int k = 0; k < 3; ++k) x[k] = p[k] * ax;
    x[j] = s * ax;
}

/* ------------------------------------------------------------------------------------ */
/* rays                                                                                  */

/* OpenCV pinhole through the centre (i + 1/2, j + 1/2) of pixel column i, row j; the
 * camera-to-world matrix is row-major 3x4 [R | o]; d is normalised so t is world length. */
void orc_ray(const float *cam, int i, int j, double o[3], double d[3])
{
    double xc = ((double)i + 0.5 - (double)cam[14]) / (double)cam[12];
    double yc = ((double)j + 0.5 - (double)cam[15]) / (double)cam[13];
    double n = 0.0;
    for (int r = 0; r < 3; ++r) {
        d[r] = (double)cam[4 * r + 0] * xc + (double)cam[4 * r + 1] * yc + (double)cam[4 * r + 2];
        o[r] = (double)cam[4 * r + 3];
        n += d[r] * d[r];
    }
    n = sqrt(n);
    for (int r = 0; r < 3; ++r) d[r] /= n;
}

/* ------------------------------------------------------------------------------------ */
/* the contracted ray as segments (Sec. 3.2: straight within a region, a new direction   */
/* only at region boundaries)                                                            */

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Region boundaries along the ray: where |x|_inf crosses 1 (|x_a| = 1) and where the
 * axis of largest magnitude can change (|x_a| = |x_b|).  Between consecutive candidates
 * the region is constant; it is read at the interval's midpoint.  Adjacent intervals of
 * one region are merged.  Each segment's contracted ends come from its own region's map;
 * the last segment ends at the contracted image of t = infinity. */
int orc_segments(const double o[3], const double d[3], orc_seg *segs)
{
    double cand[16];
    int nc = 0;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) continue;
        double t1 = (1.0 - o[a]) / d[a], t2 = (-1.0 - o[a]) / d[a];
        if (t1 > 0.0) cand[nc++] = t1;
        if (t2 > 0.0) cand[nc++] = t2;
    }
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            for (int sg = -1; sg <= 1; sg += 2) {
                /* x_a = sg x_b  <=>  t (d_a - sg d_b) = sg o_b - o_a */
                double den = d[a] - sg * d[b];
                if (den == 0.0) continue;
                double t = (sg * o[b] - o[a]) / den;
                if (t > 0.0 && isfinite(t)) cand[nc++] = t;
            }
    qsort(cand, nc, sizeof(double), cmp_double);

    double bounds[18];
    int nb = 0;
    bounds[nb++] = 0.0;
    for (int i = 0; i < nc; ++i)
        if (cand[i] > bounds[nb - 1]) bounds[nb++] = cand[i];
    bounds[nb++] = INFINITY;

    int n = 0;
    for (int m = 0; m + 1 < nb; ++m) {
        double ta = bounds[m], tb = bounds[m + 1];
        double tm = isinf(tb) ? 2.0 * ta + 1.0 : 0.5 * (ta + tb);
        double x[3] = {o[0] + tm * d[0], o[1] + tm * d[1], o[2] + tm * d[2]};
        int r = orc_region(x);
        if (n > 0 && segs[n - 1].region == r) { segs[n - 1].t1 = tb; continue; }
        segs[n].region = r;
        segs[n].t0 = ta;
        segs[n].t1 = tb;
        ++n;
    }
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        orc_seg *g = &segs[i];
        double xa[3] = {o[0] + g->t0 * d[0], o[1] + g->t0 * d[1], o[2] + g->t0 * d[2]};
        orc_contract_in_region(g->region, xa, g->a);
        if (isinf(g->t1)) {
            /* limit of the region's map as t -> infinity: p_j -> 2 s, p_k -> d_k / |d_j| */
            int j = (g->region - 1) / 2;
            double sgn = ((g->region - 1) & 1) ? -1.0 : 1.0;
            for (int k = 0; k < 3; ++k) g->b[k] = d[k] / fabs(d[j]);
            g->b[j] = 2.0 * sgn;
        } else {
            double xb[3] = {o[0] + g->t1 * d[0], o[1] + g->t1 * d[1], o[2] + g->t1 * d[2]};
            orc_contract_in_region(g->region, xb, g->b);
        }
        double l2 = 0.0;
        for (int k = 0; k < 3; ++k) l2 += (g->b[k] - g->a[k]) * (g->b[k] - g->a[k]);
        g->len = sqrt(l2);
        g->s0 = s;
        s += g->len;
    }
    return n;
}

static int seg_of(const orc_seg *segs, int n, double s)
{
    for (int i = 0; i < n; ++i)
        if (s <= segs[i].s0 + segs[i].len && segs[i].len > 0.0) return i;
    return -1;
}

/* contracted point at cumulative contracted arc length s (jumps between regions carry no
 * arc length) */
void orc_point_at(const orc_seg *segs, int n, double s, double p[3])
{
    int i = seg_of(segs, n, s);
    if (i < 0) i = n - 1;
    const orc_seg *g = &segs[i];
    double u = (s - g->s0) / g->len;
    if (u > 1.0) u = 1.0;
    for (int k = 0; k < 3; ++k) p[k] = g->a[k] + u * (g->b[k] - g->a[k]);
}

/* world ray parameter t at cumulative contracted arc length s: the region's inverse map
 * gives the world point, then t = (x - o) . d.  +inf at or beyond the end of the ray. */
double orc_t_of_s(const orc_seg *segs, int n, const double o[3], const double d[3], double s)
{
    if (s <= 0.0) return 0.0;
    double total = segs[n - 1].s0 + segs[n - 1].len;
    if (s >= total) return INFINITY;
    int i = seg_of(segs, n, s);
    double p[3], x[3];
    orc_point_at(segs, n, s, p);
    orc_uncontract(segs[i].region, p, x);
    return (x[0] - o[0]) * d[0] + (x[1] - o[1]) * d[1] + (x[2] - o[2]) * d[2];
}

/* ------------------------------------------------------------------------------------ */
/* the feature field, Sec. 3.1 and Sec. 4.2                                              */

static double dequant(int ch, int byte)
{
    double m = (ch == 0) ? 14.0 : 7.0;
    return 2.0 * m * (double)byte / 255.0 - m;
}

/* value of channel ch of logical 3D-grid voxel (ix, iy, iz); returns 0 if its block is not
 * stored (a missing voxel contributes nothing to the interpolation) */
static int voxel(const orc_scene *sc, int ix, int iy, int iz, double v[8])
{
    int C = sc->C;
    if (sc->storage == 1) {
        const float *q = sc->grid_f32 + (((size_t)iz * sc->L + iy) * sc->L + ix) * C;
        for (int c = 0; c < C; ++c) v[c] = q[c];
        return 1;
    }
    int B = sc->B, nb = sc->L / B;
    int32_t b = sc->index_grid[((size_t)(iz / B) * nb + iy / B) * nb + ix / B];
    if (b < 0) return 0;
    const uint8_t *q = sc->atlas + ((((size_t)b * B + iz % B) * B + iy % B) * B + ix % B) * C;
    for (int c = 0; c < C; ++c) v[c] = dequant(c, q[c]);
    return 1;
}

static void texel(const orc_scene *sc, int plane, int row, int col, double v[8])
{
    int C = sc->C, R = sc->R;
    size_t off = (((size_t)plane * R + row) * R + col) * C;
    if (sc->storage == 1) {
        for (int c = 0; c < C; ++c) v[c] = sc->planes_f32[off + c];
    } else {
        for (int c = 0; c < C; ++c) v[c] = dequant(c, sc->planes[off + c]);
    }
}

/* Texel centres: sample i of a resolution-N axis sits at p = (i + 1/2) 4/N - 2, so the
 * continuous index of p is u = (p + 2) N / 4 - 1/2.  Out-of-range neighbours are clamped
 * to the edge (the reading of linear texture filtering with clamp-to-edge). */
static void lin(double p, int N, int *i0, int *i1, double *w1)
{
    double u = (p + 2.0) * (double)N / 4.0 - 0.5;
    double f = floor(u);
    *w1 = u - f;
    int a = (int)f, b = a + 1;
    *i0 = a < 0 ? 0 : (a > N - 1 ? N - 1 : a);
    *i1 = b < 0 ? 0 : (b > N - 1 ? N - 1 : b);
}

/* t~(p) = V(x,y,z) + P_x(y,z) + P_y(x,z) + P_z(x,y), each source dequantised per texel and
 * interpolated (the affine dequantisation commutes with interpolation). */
void orc_field(const orc_scene *sc, const double p[3], double out[8], int *missing)
{
    int C = sc->C;
    for (int c = 0; c < C; ++c) out[c] = 0.0;
    int ix[2], iy[2], iz[2];
    double wx, wy, wz;
    lin(p[0], sc->L, &ix[0], &ix[1], &wx);
    lin(p[1], sc->L, &iy[0], &iy[1], &wy);
    lin(p[2], sc->L, &iz[0], &iz[1], &wz);
    int miss = 0;
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double w = (cx ? wx : 1.0 - wx) * (cy ? wy : 1.0 - wy) * (cz ? wz : 1.0 - wz);
                double v[8];
                if (!voxel(sc, ix[cx], iy[cy], iz[cz], v)) { ++miss; continue; }
                for (int c = 0; c < C; ++c) out[c] += w * v[c];
            }
    if (missing) *missing = miss;
    /* planes: (axis of columns, axis of rows) = P_x: (y, z), P_y: (x, z), P_z: (x, y).  A scene
     * with R = 0 has none: the grid-only (SNeRG++-style) baseline of Sec. 6, t~ = V. */
    static const int col_axis[3] = {1, 0, 0}, row_axis[3] = {2, 2, 1};
    for (int q = 0; q < (sc->R > 0 ? 3 : 0); ++q) {
        int u[2], v[2];
        double wu, wv;
        lin(p[col_axis[q]], sc->R, &u[0], &u[1], &wu);
        lin(p[row_axis[q]], sc->R, &v[0], &v[1], &wv);
        for (int cv = 0; cv < 2; ++cv)
            for (int cu = 0; cu < 2; ++cu) {
                double w = (cu ? wu : 1.0 - wu) * (cv ? wv : 1.0 - wv);
                double t[8];
                texel(sc, q, v[cv], u[cu], t);
                for (int c = 0; c < C; ++c) out[c] += w * t[c];
            }
    }
}

/* ------------------------------------------------------------------------------------ */
/* deferred view-dependence MLP h (Sec. 2 Eq. 3, App. B): input [C_d, F, gamma(d)],       */
/* gamma(d) = [d, sin d, cos d, sin 2d, cos 2d, sin 4d, cos 4d, sin 8d, cos 8d] (27),     */
/* 34 -> 16 ReLU -> 16 ReLU -> 3 linear.                                                 */

void orc_mlp(const float *w, const double cd[3], const double f[4], const double d[3], double out[3])
{
    double x[34];
    int n = 0;
    for (int k = 0; k < 3; ++k) x[n++] = cd[k];
    for (int k = 0; k < 4; ++k) x[n++] = f[k];
    for (int k = 0; k < 3; ++k) x[n++] = d[k];
    for (int l = 0; l < 4; ++l) {
        double fr = (double)(1 << l);
        for (int k = 0; k < 3; ++k) x[n++] = sin(fr * d[k]);
        for (int k = 0; k < 3; ++k) x[n++] = cos(fr * d[k]);
    }
    const float *W0 = w, *b0 = W0 + 34 * 16, *W1 = b0 + 16, *b1 = W1 + 16 * 16, *W2 = b1 + 16,
                *b2 = W2 + 16 * 3;
    double h1[16], h2[16];
    for (int o = 0; o < 16; ++o) {
        double a = b0[o];
        for (int i = 0; i < 34; ++i) a += x[i] * (double)W0[i * 16 + o];
        h1[o] = a > 0.0 ? a : 0.0;
    }
    for (int o = 0; o < 16; ++o) {
        double a = b1[o];
        for (int i = 0; i < 16; ++i) a += h1[i] * (double)W1[i * 16 + o];
        h2[o] = a > 0.0 ? a : 0.0;
    }
    for (int o = 0; o < 3; ++o) {
        double a = b2[o];
        for (int i = 0; i < 16; ++i) a += h2[i] * (double)W2[i * 3 + o];
        out[o] = a;
    }
}

/* ------------------------------------------------------------------------------------ */
/* FP32 decision replica.  The kernel decides in float which lattice samples exist and    */
/* which occupancy cell each lands in; these functions restate that float arithmetic,     */
/* operation by operation with every result rounded to float (no fused multiply-add), so  */
/* an integer decision can be compared bit for bit.  Values (features, weights, colour)   */
/* are never taken from here.                                                            */

void orc32_ray(const float *cam, int i, int j, float o[3], float d[3])
{
    float u = (float)i + 0.5f, v = (float)j + 0.5f;
    float xc = (u - cam[14]) / cam[12];
    float yc = (v - cam[15]) / cam[13];
    float w[3];
    for (int r = 0; r < 3; ++r) {
        float t0 = cam[4 * r + 0] * xc;
        float t1 = cam[4 * r + 1] * yc;
        float t2 = t0 + t1;
        w[r] = t2 + cam[4 * r + 2];
        o[r] = cam[4 * r + 3];
    }
    float n2 = w[0] * w[0];
    n2 = n2 + w[1] * w[1];
    n2 = n2 + w[2] * w[2];
    float n = sqrtf(n2);
    for (int r = 0; r < 3; ++r) d[r] = w[r] / n;
}

static int region32(const float x[3])
{
    int j = 0;
    float ax = fabsf(x[0]);
    for (int a = 1; a < 3; ++a)
        if (fabsf(x[a]) > ax) { ax = fabsf(x[a]); j = a; }
    if (ax <= 1.0f) return 0;
    return 1 + 2 * j + (x[j] < 0.0f ? 1 : 0);
}

static void contract32(int region, const float x[3], float p[3])
{
    if (region == 0) { p[0] = x[0]; p[1] = x[1]; p[2] = x[2]; return; }
    int j = (region - 1) / 2;
    float ax = fabsf(x[j]);
    for (int k = 0; k < 3; ++k) p[k] = x[k] / ax;
    float q = 2.0f - 1.0f / ax;
    p[j] = ((region - 1) & 1) ? -q : q;
}

void orc32_segments(const float o[3], const float d[3], orc32_segs *sg)
{
    float cand[12];
    int nc = 0;
    for (int a = 0; a < 3; ++a) {
        float t1 = (1.0f - o[a]) / d[a];
        float t2 = (-1.0f - o[a]) / d[a];
        if (t1 > 0.0f && t1 < INFINITY) cand[nc++] = t1;
        if (t2 > 0.0f && t2 < INFINITY) cand[nc++] = t2;
    }
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            for (int s = 0; s < 2; ++s) {
                float num = (s == 0 ? o[b] : -o[b]) - o[a];
                float den = d[a] - (s == 0 ? d[b] : -d[b]);
                float t = num / den;
                if (t > 0.0f && t < INFINITY) cand[nc++] = t;
            }
    for (int i = 1; i < nc; ++i) {          /* insertion sort, ascending */
        float v = cand[i];
        int k = i - 1;
        while (k >= 0 && cand[k] > v) { cand[k + 1] = cand[k]; --k; }
        cand[k + 1] = v;
    }
    float bounds[14];
    int nb = 0;
    bounds[nb++] = 0.0f;
    for (int i = 0; i < nc; ++i)
        if (cand[i] > bounds[nb - 1]) bounds[nb++] = cand[i];
    bounds[nb++] = INFINITY;

    float ta[ORC_MAX_SEGS], tb[ORC_MAX_SEGS];
    int n = 0;
    for (int m = 0; m + 1 < nb; ++m) {
        float t0 = bounds[m], t1 = bounds[m + 1];
        float tm = (t1 < INFINITY) ? (t0 + t1) * 0.5f : t0 * 2.0f + 1.0f;
        float x[3];
        for (int k = 0; k < 3; ++k) x[k] = o[k] + tm * d[k];
        int r = region32(x);
        if (n > 0 && sg->region[n - 1] == r) { tb[n - 1] = t1; continue; }
        sg->region[n] = r;
        ta[n] = t0;
        tb[n] = t1;
        ++n;
    }
    sg->n = n;
    sg->s0[0] = 0.0f;
    for (int i = 0; i < n; ++i) {
        int r = sg->region[i];
        float xa[3], pa[3], pb[3];
        for (int k = 0; k < 3; ++k) xa[k] = o[k] + ta[i] * d[k];
        contract32(r, xa, pa);
        if (tb[i] < INFINITY) {
            float xb[3];
            for (int k = 0; k < 3; ++k) xb[k] = o[k] + tb[i] * d[k];
            contract32(r, xb, pb);
        } else if (r == 0) {
            for (int k = 0; k < 3; ++k) pb[k] = pa[k];     /* degenerate direction only */
        } else {
            int j = (r - 1) / 2;
            float adj = fabsf(d[j]);
            for (int k = 0; k < 3; ++k) pb[k] = d[k] / adj;
            pb[j] = ((r - 1) & 1) ? -2.0f : 2.0f;
        }
        float e[3];
        for (int k = 0; k < 3; ++k) e[k] = pb[k] - pa[k];
        float l2 = e[0] * e[0];
        l2 = l2 + e[1] * e[1];
        l2 = l2 + e[2] * e[2];
        float len = sqrtf(l2);
        if (!(len < INFINITY)) len = 0.0f;
        for (int k = 0; k < 3; ++k) {
            sg->a[i][k] = pa[k];
            sg->e[i][k] = len > 0.0f ? e[k] / len : 0.0f;
        }
        sg->s0[i + 1] = sg->s0[i] + len;
    }
}

/* lattice sample k (centre ((float)k + 0.5) step) exists iff ((float)k + 1) step < total */
int orc32_lattice_count(const orc32_segs *sg, float step)
{
    float total = sg->s0[sg->n];
    int k = 0;
    while (((float)k + 1.0f) * step < total) ++k;
    return k;
}

/* Finest cell of lattice sample k: the segment i with s0[i] <= s < s0[i+1], the point
 * p = a_i + (s - s0[i]) e_i, the cell floor(p N/4) + N/2 clamped to [0, N-1]. */
int orc32_sample_cell(const orc32_segs *sg, float step, int k, int N, int cell[3])
{
    float s = ((float)k + 0.5f) * step;
    int i = -1;
    for (int m = 0; m < sg->n; ++m)
        if (sg->s0[m] <= s && s < sg->s0[m + 1]) { i = m; break; }
    if (i < 0) return 0;
    float u = s - sg->s0[i];
    float sc = (float)N * 0.25f;
    for (int a = 0; a < 3; ++a) {
        float p = sg->a[i][a] + u * sg->e[i][a];
        int c = (int)floorf(p * sc) + N / 2;
        cell[a] = c < 0 ? 0 : (c > N - 1 ? N - 1 : c);
    }
    return 1;
}

/* ------------------------------------------------------------------------------------ */
/* ablation: the spherical contraction (Eq. contract360) and its dense march               */

void orc_contract_sph(const double x[3], double p[3])
{
    double r = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    if (r <= 1.0) {
        for (int a = 0; a < 3; ++a) p[a] = x[a];
        return;
    }
    for (int a = 0; a < 3; ++a) p[a] = (2.0 - 1.0 / r) * x[a] / r;
}

/* Reading: the paper names no sampling for this contraction beyond "no AABB skipping"; samples
 * are spaced uniformly in s, with mip-NeRF 360's inverse spacing t(s) = s (s <= 1), 1/(2 - s)
 * (s > 1), so that s = 2 is the point at infinity. */
double orc_sph_t_of_s(double s) { return s <= 1.0 ? s : 1.0 / (2.0 - s); }

int orc_sph_count(double step)
{
    int k = 0;
    while (((double)k + 1.0) * step < 2.0) ++k;
    return k;
}

int orc32_sph_count(float step)
{
    int k = 0;
    while (((float)k + 1.0f) * step < 2.0f) ++k;
    return k;
}

/* FP32 replica of the kernel's sample position, each operation rounded once, in this order */
void orc32_sph_point(const float o[3], const float d[3], float step, int k, float p[3])
{
    float s = ((float)k + 0.5f) * step;
    float t = s <= 1.0f ? s : 1.0f / (2.0f - s);
    float x[3];
    for (int a = 0; a < 3; ++a) {
        float td = t * d[a];
        x[a] = o[a] + td;
    }
    float x0 = x[0] * x[0], x1 = x[1] * x[1], x2 = x[2] * x[2];
    float r = sqrtf((x0 + x1) + x2);
    if (r <= 1.0f) {
        for (int a = 0; a < 3; ++a) p[a] = x[a];
        return;
    }
    float w = (2.0f - 1.0f / r) / r;
    for (int a = 0; a < 3; ++a) p[a] = x[a] * w;
}

static void cell32(const float p[3], int N, int cell[3])
{
    float sc = (float)N * 0.25f;
    for (int a = 0; a < 3; ++a) {
        float q = p[a] * sc;
        int c = (int)floorf(q) + N / 2;
        cell[a] = c < 0 ? 0 : (c > N - 1 ? N - 1 : c);
    }
}

/* ------------------------------------------------------------------------------------ */
/* one ray                                                                               */

static int occ_at(const orc_scene *sc, const int cell[3])
{
    int N = sc->occ_res[0];
    return sc->occ[0][((size_t)cell[2] * N + cell[1]) * N + cell[0]] != 0;
}

static void cell64(const double p[3], int N, int cell[3], double *face_dist)
{
    double md = 1e30;
    for (int a = 0; a < 3; ++a) {
        double u = (p[a] + 2.0) * (double)N / 4.0;
        double f = floor(u);
        int c = (int)f;
        cell[a] = c < 0 ? 0 : (c > N - 1 ? N - 1 : c);
        double dd = fmin(u - f, f + 1.0 - u) * 4.0 / (double)N;
        if (dd < md) md = dd;
    }
    if (face_dist) *face_dist = md;
}

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* bit sets of the data read (orc_footprint) */
typedef struct {
    uint64_t *grid, *planes, *index;
} orc_marks;

static void set_bit(uint64_t *w, size_t i) { __atomic_fetch_or(w + (i >> 6), 1ull << (i & 63), __ATOMIC_RELAXED); }

static void mark_sample(const orc_scene *sc, const double p[3], orc_marks *mk)
{
    int ix[2], iy[2], iz[2];
    double w;
    lin(p[0], sc->L, &ix[0], &ix[1], &w);
    lin(p[1], sc->L, &iy[0], &iy[1], &w);
    lin(p[2], sc->L, &iz[0], &iz[1], &w);
    int B = sc->B, nb = sc->L / B;
    set_bit(mk->index, ((size_t)(iz[0] / B) * nb + iy[0] / B) * nb + ix[0] / B);
    for (int c = 0; c < 8; ++c) {
        int x = ix[c & 1], y = iy[(c >> 1) & 1], z = iz[c >> 2];
        if (sc->index_grid[((size_t)(z / B) * nb + y / B) * nb + x / B] >= 0)
            set_bit(mk->grid, ((size_t)z * sc->L + y) * sc->L + x);
    }
    static const int col_axis[3] = {1, 0, 0}, row_axis[3] = {2, 2, 1};
    for (int q = 0; q < (sc->R > 0 ? 3 : 0); ++q) {
        int u[2], v[2];
        lin(p[col_axis[q]], sc->R, &u[0], &u[1], &w);
        lin(p[row_axis[q]], sc->R, &v[0], &v[1], &w);
        for (int c = 0; c < 4; ++c)
            set_bit(mk->planes, ((size_t)q * sc->R + v[c >> 1]) * sc->R + u[c & 1]);
    }
}

/* The same quadrature with the spherical contraction, every sample visited (no skipping). */
static void render_ray_sph(const orc_scene *sc, const orc_opts *op, const float *cam, int i, int j,
                           double *rec)
{
    double o[3], d[3];
    orc_ray(cam, i, j, o, d);
    float o32[3], d32[3];
    orc32_ray(cam, i, j, o32, d32);
    double step = op->step;
    int nlat = op->decide_f32 ? orc32_sph_count((float)step) : orc_sph_count(step);
    double T = 1.0, cd[3] = {0, 0, 0}, F[4] = {0, 0, 0, 0};
    int neval = 0, napp = 0, term = 0;
    int N = sc->occ_res[0];
    for (int k = 0; k < nlat; ++k) {
        double s = ((double)k + 0.5) * step, t = orc_sph_t_of_s(s);
        double x[3], p[3];
        for (int a = 0; a < 3; ++a) x[a] = o[a] + t * d[a];
        orc_contract_sph(x, p);
        int cell[3];
        if (op->decide_f32) {
            float p32[3];
            orc32_sph_point(o32, d32, (float)step, k, p32);
            cell32(p32, N, cell);
        } else {
            cell64(p, N, cell, NULL);
        }
        if (!occ_at(sc, cell)) continue;
        double tt[8];
        orc_field(sc, p, tt, NULL);
        double tau = exp(tt[0]);
        double dt = orc_sph_t_of_s(((double)k + 1.0) * step) - orc_sph_t_of_s((double)k * step);
        double alpha = 1.0 - exp(-tau * dt);
        ++neval;
        if (alpha > 0.0) ++napp;
        double w = alpha * T;
        for (int c = 0; c < 3; ++c) cd[c] += w * sigmoid(tt[1 + c]);
        for (int c = 0; c < 4; ++c) F[c] += w * sigmoid(tt[4 + c]);
        T *= (1.0 - alpha);
        if (op->early_term && T < op->t_term) { term = 1; break; }
    }
    double h[3] = {0, 0, 0};
    if (!op->no_mlp) orc_mlp(sc->mlp, cd, F, d, h);
    for (int c = 0; c < 3; ++c) { rec[ORC_RGB + c] = cd[c] + h[c]; rec[ORC_CD + c] = cd[c]; }
    for (int c = 0; c < 4; ++c) rec[ORC_F + c] = F[c];
    rec[ORC_T] = T;
    rec[ORC_NLAT] = nlat;
    rec[ORC_NEVAL] = neval;
    rec[ORC_NAPP] = napp;
    rec[ORC_TERM] = term;
    rec[ORC_SEGS] = 0;
}

static void render_ray(const orc_scene *sc, const orc_opts *op, const float *cam, int i, int j,
                       double *rec, orc_marks *mk)
{
    if (op->contraction == 1) {
        render_ray_sph(sc, op, cam, i, j, rec);
        return;
    }
    double o[3], d[3];
    orc_seg segs[ORC_MAX_SEGS];
    orc_ray(cam, i, j, o, d);
    int ns = orc_segments(o, d, segs);
    double total = segs[ns - 1].s0 + segs[ns - 1].len;
    double step = op->step;

    orc32_segs sg;
    int nlat;
    if (op->decide_f32) {
        float o32[3], d32[3];
        orc32_ray(cam, i, j, o32, d32);
        orc32_segments(o32, d32, &sg);
        nlat = orc32_lattice_count(&sg, (float)step);
    } else {
        nlat = 0;
        while (((double)nlat + 1.0) * step < total) ++nlat;
    }

    double T = 1.0, cd[3] = {0, 0, 0}, F[4] = {0, 0, 0, 0};
    int neval = 0, napp = 0, term = 0;
    int N = sc->occ_res[0];
    for (int k = 0; k < nlat; ++k) {
        double s = ((double)k + 0.5) * step;
        double p[3];
        orc_point_at(segs, ns, s, p);
        int cell[3];
        if (op->decide_f32) {
            if (!orc32_sample_cell(&sg, (float)step, k, N, cell)) continue;
        } else {
            cell64(p, N, cell, NULL);
        }
        if (!occ_at(sc, cell)) continue;

        double tt[8];
        orc_field(sc, p, tt, NULL);
        if (mk) mark_sample(sc, p, mk);
        double tau = exp(tt[0]);
        double dt = orc_t_of_s(segs, ns, o, d, ((double)k + 1.0) * step) -
                    orc_t_of_s(segs, ns, o, d, (double)k * step);
        double alpha = isinf(dt) ? (tau > 0.0 ? 1.0 : 0.0) : 1.0 - exp(-tau * dt);
        ++neval;
        if (alpha > 0.0) ++napp;
        double w = alpha * T;
        for (int c = 0; c < 3; ++c) cd[c] += w * sigmoid(tt[1 + c]);
        for (int c = 0; c < 4; ++c) F[c] += w * sigmoid(tt[4 + c]);
        T *= (1.0 - alpha);
        if (op->early_term && T < op->t_term) { term = 1; break; }
    }
    double h[3] = {0, 0, 0};
    if (!op->no_mlp) orc_mlp(sc->mlp, cd, F, d, h);
    for (int c = 0; c < 3; ++c) { rec[ORC_RGB + c] = cd[c] + h[c]; rec[ORC_CD + c] = cd[c]; }
    for (int c = 0; c < 4; ++c) rec[ORC_F + c] = F[c];
    rec[ORC_T] = T;
    rec[ORC_NLAT] = nlat;
    rec[ORC_NEVAL] = neval;
    rec[ORC_NAPP] = napp;
    rec[ORC_TERM] = term;
    rec[ORC_SEGS] = ns;
}

/* ------------------------------------------------------------------------------------ */
/* adjoint (dense float storage): the gradient of Eq. 1 / Eq. 2 compositing, the activations,  */
/* the interpolation of Eq. 3 and the deferred MLP, by the chain rule, sample by sample.       */

/* add g (8 channels) times the interpolation weights of p into the grid and plane gradients */
static void scatter_field(const orc_scene *sc, const double p[3], const double g[8], double *g_grid,
                          double *g_planes)
{
    int C = sc->C, L = sc->L, R = sc->R;
    int ix[2], iy[2], iz[2];
    double wx, wy, wz;
    lin(p[0], L, &ix[0], &ix[1], &wx);
    lin(p[1], L, &iy[0], &iy[1], &wy);
    lin(p[2], L, &iz[0], &iz[1], &wz);
    for (int cz = 0; cz < 2; ++cz)
        for (int cy = 0; cy < 2; ++cy)
            for (int cx = 0; cx < 2; ++cx) {
                double w = (cx ? wx : 1.0 - wx) * (cy ? wy : 1.0 - wy) * (cz ? wz : 1.0 - wz);
                double *q = g_grid + (((size_t)iz[cz] * L + iy[cy]) * L + ix[cx]) * C;
                for (int c = 0; c < C; ++c) q[c] += w * g[c];
            }
    static const int col_axis[3] = {1, 0, 0}, row_axis[3] = {2, 2, 1};
    for (int q = 0; q < 3; ++q) {
        int u[2], v[2];
        double wu, wv;
        lin(p[col_axis[q]], R, &u[0], &u[1], &wu);
        lin(p[row_axis[q]], R, &v[0], &v[1], &wv);
        for (int cv = 0; cv < 2; ++cv)
            for (int cu = 0; cu < 2; ++cu) {
                double w = (cu ? wu : 1.0 - wu) * (cv ? wv : 1.0 - wv);
                double *t = g_planes + (((size_t)q * R + v[cv]) * R + u[cu]) * C;
                for (int c = 0; c < C; ++c) t[c] += w * g[c];
            }
    }
}

/* MLP forward with intermediates and backward: returns dL/dx[0..6] (C_d, F) for dL/dh = gh */
static void mlp_backward(const float *w, const double cd[3], const double f[4], const double d[3],
                         const double gh[3], double gx7[7], double *g_mlp)
{
    double x[34];
    int n = 0;
    for (int k = 0; k < 3; ++k) x[n++] = cd[k];
    for (int k = 0; k < 4; ++k) x[n++] = f[k];
    for (int k = 0; k < 3; ++k) x[n++] = d[k];
    for (int l = 0; l < 4; ++l) {
        double fr = (double)(1 << l);
        for (int k = 0; k < 3; ++k) x[n++] = sin(fr * d[k]);
        for (int k = 0; k < 3; ++k) x[n++] = cos(fr * d[k]);
    }
    const float *W0 = w, *b0 = W0 + 34 * 16, *W1 = b0 + 16, *b1 = W1 + 16 * 16, *W2 = b1 + 16;
    double z1[16], a1[16], z2[16], a2[16];
    for (int o = 0; o < 16; ++o) {
        double a = b0[o];
        for (int i = 0; i < 34; ++i) a += x[i] * (double)W0[i * 16 + o];
        z1[o] = a;
        a1[o] = a > 0.0 ? a : 0.0;
    }
    for (int o = 0; o < 16; ++o) {
        double a = b1[o];
        for (int i = 0; i < 16; ++i) a += a1[i] * (double)W1[i * 16 + o];
        z2[o] = a;
        a2[o] = a > 0.0 ? a : 0.0;
    }
    double *gW0 = g_mlp, *gb0 = gW0 + 34 * 16, *gW1 = gb0 + 16, *gb1 = gW1 + 16 * 16, *gW2 = gb1 + 16,
           *gb2 = gW2 + 16 * 3;
    double da2[16], dz2[16], da1[16], dz1[16];
    for (int o = 0; o < 3; ++o) gb2[o] += gh[o];
    for (int i = 0; i < 16; ++i) {
        double a = 0.0;
        for (int o = 0; o < 3; ++o) {
            gW2[i * 3 + o] += a2[i] * gh[o];
            a += (double)W2[i * 3 + o] * gh[o];
        }
        da2[i] = a;
        dz2[i] = z2[i] > 0.0 ? a : 0.0;
    }
    for (int o = 0; o < 16; ++o) gb1[o] += dz2[o];
    for (int i = 0; i < 16; ++i) {
        double a = 0.0;
        for (int o = 0; o < 16; ++o) {
            gW1[i * 16 + o] += a1[i] * dz2[o];
            a += (double)W1[i * 16 + o] * dz2[o];
        }
        da1[i] = a;
        dz1[i] = z1[i] > 0.0 ? a : 0.0;
    }
    for (int o = 0; o < 16; ++o) gb0[o] += dz1[o];
    for (int i = 0; i < 34; ++i) {
        double a = 0.0;
        for (int o = 0; o < 16; ++o) {
            gW0[i * 16 + o] += x[i] * dz1[o];
            a += (double)W0[i * 16 + o] * dz1[o];
        }
        if (i < 7) gx7[i] = a;
    }
}

typedef struct {
    double p[3], tau, delta, alpha, T, c[3], f[4];
} orc_sample;

static void grad_ray(const orc_scene *sc, const orc_opts *op, const float *cam, int i, int j,
                     const double gC[3], double *g_grid, double *g_planes, double *g_mlp)
{
    double o[3], d[3];
    orc_seg segs[ORC_MAX_SEGS];
    orc_ray(cam, i, j, o, d);
    int ns = orc_segments(o, d, segs);
    double step = op->step;
    orc32_segs sg;
    int nlat;
    if (op->decide_f32) {
        float o32[3], d32[3];
        orc32_ray(cam, i, j, o32, d32);
        orc32_segments(o32, d32, &sg);
        nlat = orc32_lattice_count(&sg, (float)step);
    } else {
        double total = segs[ns - 1].s0 + segs[ns - 1].len;
        nlat = 0;
        while (((double)nlat + 1.0) * step < total) ++nlat;
    }
    /* forward, keeping every evaluated sample */
    orc_sample *smp = (orc_sample *)malloc(sizeof(orc_sample) * (size_t)(nlat > 0 ? nlat : 1));
    int n = 0, N = sc->occ_res[0];
    double T = 1.0, cd[3] = {0, 0, 0}, F[4] = {0, 0, 0, 0};
    for (int k = 0; k < nlat; ++k) {
        double p[3];
        orc_point_at(segs, ns, ((double)k + 0.5) * step, p);
        int cell[3];
        if (op->decide_f32) {
            if (!orc32_sample_cell(&sg, (float)step, k, N, cell)) continue;
        } else {
            cell64(p, N, cell, NULL);
        }
        if (!occ_at(sc, cell)) continue;
        double tt[8];
        orc_field(sc, p, tt, NULL);
        orc_sample *s = &smp[n++];
        for (int a = 0; a < 3; ++a) s->p[a] = p[a];
        s->tau = exp(tt[0]);
        s->delta = orc_t_of_s(segs, ns, o, d, ((double)k + 1.0) * step) - orc_t_of_s(segs, ns, o, d, (double)k * step);
        s->alpha = 1.0 - exp(-s->tau * s->delta);
        s->T = T;
        for (int c = 0; c < 3; ++c) s->c[c] = sigmoid(tt[1 + c]);
        for (int c = 0; c < 4; ++c) s->f[c] = sigmoid(tt[4 + c]);
        double w = s->alpha * T;
        for (int c = 0; c < 3; ++c) cd[c] += w * s->c[c];
        for (int c = 0; c < 4; ++c) F[c] += w * s->f[c];
        T *= (1.0 - s->alpha);
        if (op->early_term && T < op->t_term) break;
    }
    /* C = C_d + h(C_d, F, d): dL/dC_d = gC + dh/dC_d^T gC, dL/dF = dh/dF^T gC */
    double gx7[7];
    mlp_backward(sc->mlp, cd, F, d, gC, gx7, g_mlp);
    double Gc[3] = {gC[0] + gx7[0], gC[1] + gx7[1], gC[2] + gx7[2]};
    double Gf[4] = {gx7[3], gx7[4], gx7[5], gx7[6]};
    /* back to front: U_i = sum_{j>i} prod_{i<k<j} (1 - alpha_k) alpha_j G.v_j, so that
     * dL/dalpha_i = T_i (G.v_i - U_i) */
    double U = 0.0;
    for (int m = n - 1; m >= 0; --m) {
        const orc_sample *s = &smp[m];
        double Gv = 0.0;
        for (int c = 0; c < 3; ++c) Gv += Gc[c] * s->c[c];
        for (int c = 0; c < 4; ++c) Gv += Gf[c] * s->f[c];
        double dalpha = s->T * (Gv - U);
        U = s->alpha * Gv + (1.0 - s->alpha) * U;
        double w = s->alpha * s->T;
        double g[8];
        /* alpha = 1 - exp(-tau delta): dalpha/dtau = delta (1 - alpha); tau = exp(t0) */
        g[0] = dalpha * s->delta * (1.0 - s->alpha) * s->tau;
        for (int c = 0; c < 3; ++c) g[1 + c] = w * Gc[c] * s->c[c] * (1.0 - s->c[c]);
        for (int c = 0; c < 4; ++c) g[4 + c] = w * Gf[c] * s->f[c] * (1.0 - s->f[c]);
        scatter_field(sc, s->p, g, g_grid, g_planes);
    }
    free(smp);
}

int orc_render_grad(const orc_scene *sc, const float *cams, int n_cams, int W, int H,
                    const int32_t *pix, int n_pix, const orc_opts *opts, const double *dl_drgb,
                    double *g_grid, double *g_planes, double *g_mlp)
{
    if (sc->storage != 1) return -1;
    for (int r = 0; r < n_pix; ++r) {
        int c = pix[3 * r + 0], i = pix[3 * r + 1], j = pix[3 * r + 2];
        if (c < 0 || c >= n_cams || i < 0 || i >= W || j < 0 || j >= H) return -2;
        grad_ray(sc, opts, cams + 16 * c, i, j, dl_drgb + 3 * r, g_grid, g_planes, g_mlp);
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* threaded drivers                                                                      */

typedef struct {
    const orc_scene *sc;
    const orc_opts *op;
    const float *cams;
    int n_cams, W, H;
    const int32_t *pix;
    int n_pix;
    double *out;
    int tid, nth;
    /* trace */
    double step, eps;
    int decide_f32, words, contraction;
    int decisive;          /* trace flags: 0 near any cell face, 1 only where a decision can change */
    uint32_t *mask, *flags;
    int32_t *nlat;
    orc_marks *marks;      /* footprint: NULL when only rendering */
} job;

static void pixel_of(const job *jb, long r, int *cam, int *i, int *j)
{
    if (jb->pix) {
        *cam = jb->pix[3 * r + 0]; *i = jb->pix[3 * r + 1]; *j = jb->pix[3 * r + 2];
    } else {
        long per = (long)jb->W * jb->H;
        *cam = (int)(r / per);
        long q = r % per;
        *j = (int)(q / jb->W);
        *i = (int)(q % jb->W);
    }
}

static void *render_worker(void *arg)
{
    job *jb = (job *)arg;
    long n = jb->pix ? jb->n_pix : (long)jb->n_cams * jb->W * jb->H;
    for (long r = jb->tid; r < n; r += jb->nth) {
        int c, i, j;
        pixel_of(jb, r, &c, &i, &j);
        render_ray(jb->sc, jb->op, jb->cams + 16 * c, i, j, jb->out + ORC_OUT * r, jb->marks);
    }
    return NULL;
}

static void run_jobs(job *proto, void *(*fn)(void *), int n_threads)
{
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    job jobs[256];
    for (int t = 0; t < n_threads; ++t) {
        jobs[t] = *proto;
        jobs[t].tid = t;
        jobs[t].nth = n_threads;
        if (t > 0) pthread_create(&th[t], NULL, fn, &jobs[t]);
    }
    fn(&jobs[0]);
    for (int t = 1; t < n_threads; ++t) pthread_join(th[t], NULL);
}

int orc_render(const orc_scene *sc, const float *cams, int n_cams, int W, int H,
               const int32_t *pix, int n_pix, const orc_opts *opts, double *out, int n_threads)
{
    job jb;
    memset(&jb, 0, sizeof jb);
    jb.sc = sc; jb.op = opts; jb.cams = cams; jb.n_cams = n_cams; jb.W = W; jb.H = H;
    jb.pix = pix; jb.n_pix = n_pix; jb.out = out;
    run_jobs(&jb, render_worker, n_threads);
    return 0;
}

int orc_footprint(const orc_scene *sc, const float *cams, int n_cams, int W, int H,
                  const int32_t *pix, int n_pix, const orc_opts *opts, uint64_t counts[3], int n_threads)
{
    if (sc->storage != 0) return -1;
    size_t nv = (size_t)sc->L * sc->L * sc->L, np = (size_t)3 * sc->R * sc->R, nb = (size_t)sc->L / sc->B;
    nb = nb * nb * nb;
    orc_marks mk;
    mk.grid = (uint64_t *)calloc(nv / 64 + 1, 8);
    mk.planes = (uint64_t *)calloc(np / 64 + 1, 8);
    mk.index = (uint64_t *)calloc(nb / 64 + 1, 8);
    if (!mk.grid || !mk.planes || !mk.index) {
        free(mk.grid); free(mk.planes); free(mk.index);
        return -2;
    }
    long n = pix ? n_pix : (long)n_cams * W * H;
    double *out = (double *)malloc(sizeof(double) * ORC_OUT * (size_t)(n > 0 ? n : 1));
    job jb;
    memset(&jb, 0, sizeof jb);
    jb.sc = sc; jb.op = opts; jb.cams = cams; jb.n_cams = n_cams; jb.W = W; jb.H = H;
    jb.pix = pix; jb.n_pix = n_pix; jb.out = out; jb.marks = &mk;
    run_jobs(&jb, render_worker, n_threads);
    free(out);
    uint64_t *sets[3] = {mk.grid, mk.planes, mk.index};
    size_t words[3] = {nv / 64 + 1, np / 64 + 1, nb / 64 + 1};
    for (int k = 0; k < 3; ++k) {
        uint64_t c = 0;
        for (size_t w = 0; w < words[k]; ++w) c += (uint64_t)__builtin_popcountll(sets[k][w]);
        counts[k] = c;
    }
    free(mk.grid); free(mk.planes); free(mk.index);
    return 0;
}

/* Reading 14 of the FP32-vs-FP64 comparison: an integer outcome of a lattice sample can differ
 * between two precisions only where a rounding-sized move of its position or arc length changes
 * it.  Position: some finest cell within eps of p (across a face, an edge or a corner, inside the
 * grid) holds an occupancy value other than p's own cell's.  Arc length: s lies within eps of an
 * interior segment boundary (the contracted ray may jump there, Sec. 3.2) or (k + 1) step lies
 * within eps of the total arc length (whether sample k exists at all). */
static int occ_decision_ambiguous(const orc_scene *sc, const double p[3], const int cell[3], double eps)
{
    int N = sc->occ_res[0], lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
        double u = (p[a] + 2.0) * (double)N / 4.0, f = floor(u);
        double d_lo = (u - f) * 4.0 / (double)N, d_hi = (f + 1.0 - u) * 4.0 / (double)N;
        lo[a] = (d_lo < eps && cell[a] > 0) ? cell[a] - 1 : cell[a];
        hi[a] = (d_hi < eps && cell[a] < N - 1) ? cell[a] + 1 : cell[a];
    }
    int own = occ_at(sc, cell);
    for (int z = lo[2]; z <= hi[2]; ++z)
        for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) {
                int c[3] = {x, y, z};
                if (occ_at(sc, c) != own) return 1;
            }
    return 0;
}

static int arc_decision_ambiguous(const orc_seg *segs, int ns, double step, int k, double eps)
{
    double s = ((double)k + 0.5) * step, total = segs[ns - 1].s0 + segs[ns - 1].len;
    for (int m = 1; m < ns; ++m)
        if (fabs(s - segs[m].s0) < eps) return 1;
    return fabs(((double)k + 1.0) * step - total) < eps;
}

static void *trace_worker(void *arg)
{
    job *jb = (job *)arg;
    long n = jb->pix ? jb->n_pix : (long)jb->n_cams * jb->W * jb->H;
    const orc_scene *sc = jb->sc;
    int N = sc->occ_res[0];
    for (long r = jb->tid; r < n; r += jb->nth) {
        int c, i, j;
        pixel_of(jb, r, &c, &i, &j);
        const float *cam = jb->cams + 16 * c;
        uint32_t *m = jb->mask + (size_t)r * jb->words;
        uint32_t *fl = jb->flags ? jb->flags + (size_t)r * jb->words : NULL;
        memset(m, 0, sizeof(uint32_t) * jb->words);
        if (fl) memset(fl, 0, sizeof(uint32_t) * jb->words);
        if (jb->contraction == 1) {       /* spherical contraction: every sample visited */
            double o[3], d[3];
            float o32[3], d32[3];
            orc_ray(cam, i, j, o, d);
            orc32_ray(cam, i, j, o32, d32);
            int nl = jb->decide_f32 ? orc32_sph_count((float)jb->step) : orc_sph_count(jb->step);
            jb->nlat[r] = nl;
            for (int k = 0; k < nl && k < 32 * jb->words; ++k) {
                double x[3], p[3], fd;
                double t = orc_sph_t_of_s(((double)k + 0.5) * jb->step);
                for (int a = 0; a < 3; ++a) x[a] = o[a] + t * d[a];
                orc_contract_sph(x, p);
                int cell[3];
                cell64(p, N, cell, &fd);
                int amb = jb->decisive ? occ_decision_ambiguous(sc, p, cell, jb->eps) : fd < jb->eps;
                if (fl && amb) fl[k >> 5] |= 1u << (k & 31);
                if (jb->decide_f32) {
                    float p32[3];
                    orc32_sph_point(o32, d32, (float)jb->step, k, p32);
                    cell32(p32, N, cell);
                }
                if (occ_at(sc, cell)) m[k >> 5] |= 1u << (k & 31);
            }
            continue;
        }
        double o[3], d[3];
        orc_seg segs[ORC_MAX_SEGS];
        orc_ray(cam, i, j, o, d);
        int ns = orc_segments(o, d, segs);
        double total = segs[ns - 1].s0 + segs[ns - 1].len;
        orc32_segs sg;
        int nlat;
        if (jb->decide_f32) {
            float o32[3], d32[3];
            orc32_ray(cam, i, j, o32, d32);
            orc32_segments(o32, d32, &sg);
            nlat = orc32_lattice_count(&sg, (float)jb->step);
        } else {
            nlat = 0;
            while (((double)nlat + 1.0) * jb->step < total) ++nlat;
        }
        jb->nlat[r] = nlat;
        for (int k = 0; k < nlat && k < 32 * jb->words; ++k) {
            double p[3], fd;
            int cell[3];
            orc_point_at(segs, ns, ((double)k + 0.5) * jb->step, p);
            cell64(p, N, cell, &fd);
            int amb = fd < jb->eps;
            if (jb->decisive)      /* from the FP64 position, before any FP32 decision replaces cell */
                amb = occ_decision_ambiguous(sc, p, cell, jb->eps) ||
                      arc_decision_ambiguous(segs, ns, jb->step, k, jb->eps);
            if (fl && amb) fl[k >> 5] |= 1u << (k & 31);
            if (jb->decide_f32 && !orc32_sample_cell(&sg, (float)jb->step, k, N, cell)) continue;
            if (occ_at(sc, cell)) m[k >> 5] |= 1u << (k & 31);
        }
        /* the first lattice index past the end may exist in another precision */
        if (fl && jb->decisive && nlat < 32 * jb->words &&
            arc_decision_ambiguous(segs, ns, jb->step, nlat, jb->eps))
            fl[nlat >> 5] |= 1u << (nlat & 31);
    }
    return NULL;
}

int orc_trace(const orc_scene *sc, const float *cams, int n_cams, int W, int H,
              const int32_t *pix, int n_pix, double step, int decide_f32, double eps,
              uint32_t *mask, uint32_t *flags, int words, int32_t *n_lattice, int n_threads,
              int contraction)
{
    return orc_trace_flagged(sc, cams, n_cams, W, H, pix, n_pix, step, decide_f32, eps, mask, flags, words,
                             n_lattice, n_threads, contraction, 0);
}

int orc_trace_flagged(const orc_scene *sc, const float *cams, int n_cams, int W, int H,
                      const int32_t *pix, int n_pix, double step, int decide_f32, double eps,
                      uint32_t *mask, uint32_t *flags, int words, int32_t *n_lattice, int n_threads,
                      int contraction, int decisive)
{
    job jb;
    memset(&jb, 0, sizeof jb);
    jb.contraction = contraction;
    jb.decisive = decisive;
    jb.sc = sc; jb.cams = cams; jb.n_cams = n_cams; jb.W = W; jb.H = H;
    jb.pix = pix; jb.n_pix = n_pix; jb.step = step; jb.decide_f32 = decide_f32; jb.eps = eps;
    jb.mask = mask; jb.flags = flags; jb.words = words; jb.nlat = n_lattice;
    run_jobs(&jb, trace_worker, n_threads);
    return 0;
}
