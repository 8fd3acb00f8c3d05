// traverse.cuh -- per-ray traversal of contracted space for sm_103a.
//
// A pixel ray x(t) = o + t d (Eq. 1) is mapped by the piecewise-projective contraction
// (Sec. 3.2) into [-2, 2]^3, where it becomes at most seven straight segments, one per region
// it crosses.  Samples sit on a uniform lattice s_k = (k + 1/2) delta_s of cumulative contracted
// arc length (the renderer's "small uniform step size", Sec. 4.3); sample k is evaluated iff
// its finest occupancy cell is set.  Each candidate sample reads its own finest cell (one
// cached byte: the test is the definition itself, and every lane of a warp does the same
// work).  A sample in an empty finest cell starts a skip through the max-pooled occupancy
// hierarchy (Sec. 5): the coarsest level that reports its cell empty gives the largest empty
// box around it, a slab test against that box on the current straight segment gives the exit,
// and the walk jumps past the last lattice sample before it.
//
// Exactness.  Every float operation that decides an integer (which lattice samples exist,
// which segment and which occupancy cell a sample falls in) is an IEEE round-to-nearest
// intrinsic (__fadd_rn, __fmul_rn, __fdiv_rn, __fsqrt_rn: never contracted into an FMA), in a
// fixed order.  The position of sample k within a segment is a composition of monotone
// rounded operations, so each of its coordinates -- and hence each cell index -- is monotone
// in k.  A skip therefore lands at lattice index m only after checking, from m's own computed
// position, that m - 1 still lies in the empty cell: every skipped sample lies in that cell,
// and the evaluated set equals dense sampling of the finest level, bit for bit.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "debug.cuh"

namespace merf {

// A ray has at most 12 region-boundary crossings (two faces of |x_a| = 1 per axis, two diagonal
// planes per axis pair), hence at most 13 intervals and 13 merged segments.
constexpr int kMaxSegs = 13;
constexpr int kMaxLevels = 8;

#define F_ADD __fadd_rn
#define F_SUB __fsub_rn
#define F_MUL __fmul_rn
#define F_DIV __fdiv_rn
#define F_SQRT __fsqrt_rn

struct OccView {
    const uint8_t *level[kMaxLevels];   // [N][N][N] bytes, finest first
    int res[kMaxLevels];
    int shift[kMaxLevels];              // log2(res[0] / res[l])
    int n;
};

// Pinhole ray through the centre of pixel (i, j); cam = c2w[12], fx, fy, cx, cy.
__device__ __forceinline__ void ray_f32(const float *cam, int i, int j, float o[3], float d[3])
{
    float u = F_ADD((float)i, 0.5f), v = F_ADD((float)j, 0.5f);
    float xc = F_DIV(F_SUB(u, cam[14]), cam[12]);
    float yc = F_DIV(F_SUB(v, cam[15]), cam[13]);
    float w[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        w[r] = F_ADD(F_ADD(F_MUL(cam[4 * r + 0], xc), F_MUL(cam[4 * r + 1], yc)), cam[4 * r + 2]);
        o[r] = cam[4 * r + 3];
    }
    float n2 = F_ADD(F_ADD(F_MUL(w[0], w[0]), F_MUL(w[1], w[1])), F_MUL(w[2], w[2]));
    float n = F_SQRT(n2);
#pragma unroll
    for (int r = 0; r < 3; ++r) d[r] = F_DIV(w[r], n);
}

// Component j (0, 1 or 2, not a compile-time constant) of a 3-vector, by selection: small arrays
// are never indexed dynamically, so they stay in registers.
__device__ __forceinline__ float comp3(const float v[3], int j)
{
    return j == 0 ? v[0] : (j == 1 ? v[1] : v[2]);
}

// Region of a point: 0 inside |x|_inf <= 1, else 1 + 2 j + (x_j < 0), j the first axis of
// largest magnitude.
__device__ __forceinline__ int region_f32(const float x[3])
{
    int j = 0;
    float ax = fabsf(x[0]), xj = x[0];
    if (fabsf(x[1]) > ax) { ax = fabsf(x[1]); xj = x[1]; j = 1; }
    if (fabsf(x[2]) > ax) { ax = fabsf(x[2]); xj = x[2]; j = 2; }
    if (ax <= 1.0f) return 0;
    return 1 + 2 * j + (xj < 0.0f ? 1 : 0);
}

// One region's projective map (Sec. 3.2): x_k / |x_j| and (2 - 1/|x_j|) sign(x_j).
__device__ __forceinline__ void contract_f32(int region, const float x[3], float p[3])
{
    if (region == 0) { p[0] = x[0]; p[1] = x[1]; p[2] = x[2]; return; }
    const int j = (region - 1) >> 1;
    const float ax = fabsf(comp3(x, j));
    const float q = F_SUB(2.0f, F_DIV(1.0f, ax));
    const float qs = ((region - 1) & 1) ? -q : q;
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k] = (k == j) ? qs : F_DIV(x[k], ax);
}

__device__ __forceinline__ float lattice_s(int k, float step)
{
    return F_MUL(F_ADD((float)k, 0.5f), step);
}

__device__ __forceinline__ bool lattice_exists(int k, float step, float total)
{
    return F_MUL(F_ADD((float)k, 1.0f), step) < total;
}

// smallest k >= 0 with lattice_s(k) >= S
__device__ __forceinline__ int first_k_at(float S, float step)
{
    float est = fmaxf(0.0f, fminf(ceilf(S / step - 0.5f), 16777216.0f));
    int k = (int)est;
    while (k > 0 && lattice_s(k - 1, step) >= S) --k;
    while (k < (1 << 24) && lattice_s(k, step) < S) ++k;
    return k;
}

// number of lattice samples: k exists iff ((float)k + 1) step < total
__device__ __forceinline__ int lattice_count(float total, float step)
{
    float est = fmaxf(0.0f, fminf(floorf(total / step), 16777216.0f));
    int n = (int)est;
    while (n > 0 && !lattice_exists(n - 1, step, total)) --n;
    while (n < (1 << 24) && lattice_exists(n, step, total)) ++n;
    return n;
}

// Segment table of one ray: start point A, unit direction e, cumulative arc length S, and
// the constants of the arc-length -> world-length map: the world length of arcs [u1, u2]
// (relative to the segment start) is c (u2 - u1) / ((1 - g u1)(1 - g u2)).
struct Segs {
    float A[kMaxSegs][3];
    float e[kMaxSegs][3];
    float c[kMaxSegs];
    float g[kMaxSegs];
    float S[kMaxSegs + 1];
    int n;
};

__device__ __forceinline__ void sort2(float &a, float &b)
{
    const float lo = fminf(a, b), hi = fmaxf(a, b);
    a = lo;
    b = hi;
}

// The segment table of a ray, built without scratch arrays (every index below is a compile-time
// constant except the table's own, so the candidates stay in registers): the 12 breakpoint
// candidates, rejected ones as +inf, sorted by an odd-even transposition network; the intervals
// between strictly increasing breakpoints classified by their midpoints and merged while the
// region repeats, each merged segment's [t_a, t_b] and region recorded as it closes; then each
// segment's contracted end points, direction, arc length and world-length constants.  The same
// values, in the same order of operations, as sorting the candidates, dropping duplicates,
// classifying every interval and then merging.
__device__ __forceinline__ void build_segments(const float o[3], const float d[3], Segs &sg)
{
    // region-boundary candidates: |x_a| = 1 and x_a = +-x_b
    float c[12];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float t1 = F_DIV(F_SUB(1.0f, o[a]), d[a]);
        const float t2 = F_DIV(F_SUB(-1.0f, o[a]), d[a]);
        c[2 * a] = (t1 > 0.0f && t1 < CUDART_INF_F) ? t1 : CUDART_INF_F;
        c[2 * a + 1] = (t2 > 0.0f && t2 < CUDART_INF_F) ? t2 : CUDART_INF_F;
    }
#pragma unroll
    for (int pr = 0; pr < 3; ++pr) {
        const int a = pr == 2 ? 1 : 0, b = pr == 0 ? 1 : 2;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const float num = F_SUB(s == 0 ? o[b] : -o[b], o[a]);
            const float den = F_SUB(d[a], s == 0 ? d[b] : -d[b]);
            const float t = F_DIV(num, den);
            c[6 + 2 * pr + s] = (t > 0.0f && t < CUDART_INF_F) ? t : CUDART_INF_F;
        }
    }
#pragma unroll
    for (int round = 0; round < 12; ++round)
#pragma unroll
        for (int i = round & 1; i + 1 < 12; i += 2) sort2(c[i], c[i + 1]);

    // merged segments: t_a in sg.c, t_b in sg.g (until the second pass), regions 3 bits each
    unsigned long long regions = 0ull;
    int n = 0, cur = -1;
    float t0 = 0.0f;
#pragma unroll
    for (int m = 0; m <= 12; ++m) {
        const float t1 = m < 12 ? c[m] : CUDART_INF_F;
        if (m < 12 && !(t1 > t0 && t1 < CUDART_INF_F)) continue;    // duplicate or no crossing
        const float tm = (t1 < CUDART_INF_F) ? F_MUL(F_ADD(t0, t1), 0.5f) : F_ADD(F_MUL(t0, 2.0f), 1.0f);
        float x[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) x[k] = F_ADD(o[k], F_MUL(tm, d[k]));
        const int r = region_f32(x);
        if (r != cur) {
            if (cur >= 0) ++n;
            sg.c[n] = t0;
            regions |= (unsigned long long)r << (3 * n);
            cur = r;
        }
        sg.g[n] = t1;
        t0 = t1;
    }
    ++n;

    sg.n = n;
    sg.S[0] = 0.0f;
    for (int i = 0; i < n; ++i) {
        const int r = (int)((regions >> (3 * i)) & 7ull);
        const float ta = sg.c[i], tb = sg.g[i];
        float xa[3], pa[3], pb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) xa[k] = F_ADD(o[k], F_MUL(ta, d[k]));
        contract_f32(r, xa, pa);
        const int j = (r - 1) >> 1;
        if (tb < CUDART_INF_F) {
            float xb[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) xb[k] = F_ADD(o[k], F_MUL(tb, d[k]));
            contract_f32(r, xb, pb);
        } else if (r == 0) {
            // only reachable for a degenerate direction: an empty segment
            pb[0] = pa[0]; pb[1] = pa[1]; pb[2] = pa[2];
        } else {
            // image of t -> infinity in region (j, s): p_j = 2 s, p_k = d_k / |d_j|
            const float adj = fabsf(comp3(d, j));
            const float lim = ((r - 1) & 1) ? -2.0f : 2.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) pb[k] = (k == j) ? lim : F_DIV(d[k], adj);
        }
        float ev[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) ev[k] = F_SUB(pb[k], pa[k]);
        float l2 = F_ADD(F_ADD(F_MUL(ev[0], ev[0]), F_MUL(ev[1], ev[1])), F_MUL(ev[2], ev[2]));
        float len = F_SQRT(l2);
        if (!(len < CUDART_INF_F)) len = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sg.A[i][k] = pa[k];
            sg.e[i][k] = len > 0.0f ? F_DIV(ev[k], len) : 0.0f;
        }
        sg.S[i + 1] = F_ADD(sg.S[i], len);
        // world-length constants (values, not decisions: ordinary float arithmetic)
        if (r == 0) {
            sg.c[i] = 1.0f;
            sg.g[i] = 0.0f;
        } else {
            const float sgn = ((r - 1) & 1) ? -1.0f : 1.0f;
            const float dj = comp3(d, j);
            const float xj = comp3(o, j) + ta * dj;
            const float w = 1.0f / fabsf(xj);           // 1 / |x_j| at the segment start
            float v2 = 0.0f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                // contracted velocity per unit t: w^2 d_j along j, w (d_k - s d_j p_k) otherwise
                const float vk = (k == j) ? dj * w * w : w * (d[k] - sgn * dj * pa[k]);
                v2 += vk * vk;
            }
            const float ej = len > 0.0f ? F_DIV(comp3(ev, j), len) : 0.0f;
            sg.c[i] = 1.0f / sqrtf(v2);
            sg.g[i] = sgn * ej / w;
        }
    }
}

// cell of a contracted coordinate at resolution N (N even): floor(p N/4) + N/2, clamped
__device__ __forceinline__ int cell_of(float p, float scale, int half, int N)
{
    int c = __float2int_rd(F_MUL(p, scale)) + half;
    return min(max(c, 0), N - 1);
}

// ---------------------------------------------------------------------------------------------
// Ablation (Sec. 3.2, Table 2 (c)): the spherical contraction of mip-NeRF 360,
// contract(x) = x for |x|_2 <= 1 and (2 - 1/|x|_2) x / |x|_2 beyond.  It bends straight rays, so
// there is no segment lattice and no AABB exit: the ray is marched densely, sample k at
// s_k = (k + 1/2) delta_s for (k + 1) delta_s < 2, at ray parameter t(s) = s for s <= 1 and
// 1 / (2 - s) beyond (mip-NeRF 360's inverse spacing, s = 2 being the point at infinity), each
// sample evaluated iff its finest occupancy cell is set.  Positions are decisions (they pick the
// cell), so they use the same IEEE-rounded operations, in a fixed order, as the FP32 restatement
// the tests compare against.

// number of samples: k with (k + 1) delta_s < 2
__device__ __forceinline__ int sph_count(float step)
{
    int n = (int)F_DIV(2.0f, step);
    while (n > 0 && !(F_MUL(F_ADD((float)(n - 1), 1.0f), step) < 2.0f)) --n;
    while (F_MUL(F_ADD((float)n, 1.0f), step) < 2.0f) ++n;
    return n;
}

__device__ __forceinline__ float sph_t(float s) { return s <= 1.0f ? s : F_DIV(1.0f, F_SUB(2.0f, s)); }

__device__ __forceinline__ void sph_point(const float o[3], const float d[3], float step, int k, float p[3])
{
    const float t = sph_t(F_MUL(F_ADD((float)k, 0.5f), step));
    const float x0 = F_ADD(o[0], F_MUL(t, d[0])), x1 = F_ADD(o[1], F_MUL(t, d[1])),
                x2 = F_ADD(o[2], F_MUL(t, d[2]));
    const float r = F_SQRT(F_ADD(F_ADD(F_MUL(x0, x0), F_MUL(x1, x1)), F_MUL(x2, x2)));
    const float w = r <= 1.0f ? 1.0f : F_DIV(F_SUB(2.0f, F_DIV(1.0f, r)), r);
    p[0] = r <= 1.0f ? x0 : F_MUL(x0, w);
    p[1] = r <= 1.0f ? x1 : F_MUL(x1, w);
    p[2] = r <= 1.0f ? x2 : F_MUL(x2, w);
}

// Walk state of one ray.
struct Walker {
    Segs sg;
    float A0, A1, A2, e0, e1, e2, S0, S1;  // current segment
    float ie0, ie1, ie2;                   // approximate 1/e (slab-exit candidates only)
    int seg, kend, k, nlat;
    float step, inv_step, total;

    __device__ __forceinline__ void load_seg(int i)
    {
        seg = i;
        A0 = sg.A[i][0]; A1 = sg.A[i][1]; A2 = sg.A[i][2];
        e0 = sg.e[i][0]; e1 = sg.e[i][1]; e2 = sg.e[i][2];
        ie0 = __frcp_rn(e0); ie1 = __frcp_rn(e1); ie2 = __frcp_rn(e2);
        S0 = sg.S[i];
        S1 = sg.S[i + 1];
        kend = (i == sg.n - 1) ? 0x7fffffff : first_k_at(S1, step);
    }

    __device__ __forceinline__ void init(const float o[3], const float d[3], float step_)
    {
        step = step_;
        inv_step = 1.0f / step_;
        build_segments(o, d, sg);
        total = sg.S[sg.n];
        nlat = lattice_count(total, step);
        k = 0;
        load_seg(0);
    }

    __device__ __forceinline__ void position(int kk, float &p0, float &p1, float &p2) const
    {
        const float u = F_SUB(lattice_s(kk, step), S0);
        p0 = F_ADD(A0, F_MUL(u, e0));
        p1 = F_ADD(A1, F_MUL(u, e1));
        p2 = F_ADD(A2, F_MUL(u, e2));
    }

    // One past the last lattice index whose sample still lies in the cell (x, y, z) of the
    // level of resolution N0 >> sh; k + 1 if that cannot be shown.  The candidate comes from a
    // slab test against the cell's box on the current segment; it is accepted only if the
    // candidate sample's own position (the same rounded arithmetic as every sample) lands in
    // the same cell.  By per-axis monotonicity of positions along a segment, every sample in
    // between lands there too.
    __device__ __forceinline__ int cell_exit(float p0, float p1, float p2, int x, int y, int z, int sh,
                                             int N0, float sc0, int h0) const
    {
        const int Nl = N0 >> sh;
        const float inv = 4.0f / (float)Nl;
        const int hl = Nl >> 1;
        const float lo0 = (float)(x - hl) * inv, lo1 = (float)(y - hl) * inv, lo2 = (float)(z - hl) * inv;
        float umin = CUDART_INF_F;
        if (e0 != 0.0f) umin = fminf(umin, ((e0 > 0.0f ? lo0 + inv : lo0) - p0) * ie0);
        if (e1 != 0.0f) umin = fminf(umin, ((e1 > 0.0f ? lo1 + inv : lo1) - p1) * ie1);
        if (e2 != 0.0f) umin = fminf(umin, ((e2 > 0.0f ? lo2 + inv : lo2) - p2) * ie2);
        const int last = min(kend, nlat) - 1;
        int m = last;
        const float s_exit = lattice_s(k, step) + umin;
        if (s_exit < CUDART_INF_F) {
            const float mf = ceilf(s_exit * inv_step - 0.5f) - 1.0f;
            m = (mf < (float)last) ? (int)fmaxf(mf, -1.0f) : last;
        }
        if (m > k) {
            float q0, q1, q2;
            position(m, q0, q1, q2);
            if ((cell_of(q0, sc0, h0, N0) >> sh) == x && (cell_of(q1, sc0, h0, N0) >> sh) == y &&
                (cell_of(q2, sc0, h0, N0) >> sh) == z)
                return m + 1;
            if (m - 1 > k) {
                position(m - 1, q0, q1, q2);
                if ((cell_of(q0, sc0, h0, N0) >> sh) == x && (cell_of(q1, sc0, h0, N0) >> sh) == y &&
                    (cell_of(q2, sc0, h0, N0) >> sh) == z)
                    return m;
            }
        }
        return k + 1;
    }

    // Advance k to the next lattice sample whose own finest occupancy cell is set and return
    // its position.  A sample in an empty finest cell starts a skip out of the largest empty
    // cell that contains it (coarse-to-fine: the first empty level from the coarsest), through
    // cell_exit's verified jump.  False when the ray has no further occupied sample.  Idx: the
    // offset type of the occupancy indices (32 bits only when the finest level fits).
    template <typename Idx = size_t>
    __device__ __forceinline__ bool next_sample(const OccView &occ, float &p0, float &p1, float &p2)
    {
        const int N0 = occ.res[0];
        const float sc0 = (float)N0 * 0.25f;
        const int h0 = N0 >> 1;
        while (k < nlat) {
            while (k >= kend) load_seg(seg + 1);
            position(k, p0, p1, p2);
            const int c0 = cell_of(p0, sc0, h0, N0), c1 = cell_of(p1, sc0, h0, N0),
                      c2 = cell_of(p2, sc0, h0, N0);
            const Idx oi = ((Idx)c2 * N0 + c1) * N0 + c0;
            if (MERF_IN_RANGE(oi, (long long)N0 * N0 * N0, kBadOcc) && __ldg(occ.level[0] + oi) != 0) return true;
            int sh = 0;
            for (int l = occ.n - 1; l > 0; --l) {
                const int s = occ.shift[l], Nl = occ.res[l];
                const Idx li = ((Idx)(c2 >> s) * Nl + (c1 >> s)) * Nl + (c0 >> s);
                if (!MERF_IN_RANGE(li, (long long)Nl * Nl * Nl, kBadOcc) || __ldg(occ.level[l] + li) == 0) {
                    sh = s;
                    break;
                }
            }
            k = cell_exit(p0, p1, p2, c0 >> sh, c1 >> sh, c2 >> sh, sh, N0, sc0, h0);
        }
        return false;
    }

    // World length of the lattice interval [k step, (k + 1) step] of sample k (Eq. 1's delta),
    // summed over the segments it overlaps.
    __device__ __forceinline__ float delta_world(int kk) const
    {
        const float lo = (float)kk * step, hi = ((float)kk + 1.0f) * step;
        if (lo >= S0 && hi <= S1) {
            const float c = sg.c[seg], g = sg.g[seg];
            const float u1 = lo - S0, u2 = hi - S0;
            return __fdividef(c * (hi - lo), (1.0f - g * u1) * (1.0f - g * u2));
        }
        int m = seg;
        while (m > 0 && lo < sg.S[m]) --m;
        float dw = 0.0f;
        for (;;) {
            const float a = fmaxf(lo, sg.S[m]), b = fminf(hi, sg.S[m + 1]);
            if (b > a) {
                const float c = sg.c[m], g = sg.g[m];
                const float u1 = a - sg.S[m], u2 = b - sg.S[m];
                dw += c * (b - a) / ((1.0f - g * u1) * (1.0f - g * u2));
            }
            if (hi <= sg.S[m + 1] || m >= sg.n - 1) break;
            ++m;
        }
        return dw;
    }
};

}  // namespace merf
