/* merf_oracle.h -- plain FP64 CPU oracle of the MERF real-time renderer.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call this
 * code: it exists so that tests, the smoke check and the benchmark's oracle leg (CPU
 * baseline, precision-form reference values, footprint) and reference arm can check and
 * time the CUDA renderer against a slow, obviously correct restatement of the paper.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * Sections cited are those of "MERF: Memory-Efficient Radiance Fields for Real-time View
 * Synthesis in Unbounded Scenes" (Reiser et al., SIGGRAPH 2023).
 */
#ifndef MERF_ORACLE_H
#define MERF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_SEGS 16
#define ORC_OUT 16   /* doubles per pixel in orc_render's output record */

/* Output record layout (per pixel, doubles). */
enum {
    ORC_RGB = 0,        /* [3] final colour C = C_d + h(C_d, F, d)                  */
    ORC_CD = 3,         /* [3] accumulated diffuse colour C_d (Eq. 2)               */
    ORC_F = 6,          /* [4] accumulated feature F (Eq. 2)                        */
    ORC_T = 10,         /* transmittance after the last composited sample          */
    ORC_NLAT = 11,      /* number of lattice samples on the ray                    */
    ORC_NEVAL = 12,     /* samples evaluated (occupied and not terminated)         */
    ORC_NAPP = 13,      /* evaluated samples whose opacity is non-zero             */
    ORC_TERM = 14,      /* 1 if the ray stopped by early termination               */
    ORC_SEGS = 15       /* number of contracted segments of the ray                */
};

typedef struct {
    int L, B, R, C;                 /* grid res, block edge (0 = dense f32), plane res, channels */
    int n_occ;                      /* occupancy levels (only the finest, index 0, is used) */
    int occ_res[8];
    const uint8_t *occ[8];          /* [N][N][N] bytes, z-major */
    int storage;                    /* 0: uint8 block-sparse, 1: float32 dense */
    const int32_t *index_grid;      /* [L/B]^3 block ids or -1 */
    const uint8_t *atlas;           /* [n_blocks][B][B][B][C] */
    int n_blocks;
    const uint8_t *planes;          /* [3][R][R][C] */
    const float *grid_f32;          /* [L][L][L][C] */
    const float *planes_f32;        /* [3][R][R][C] */
    const float *mlp;               /* 883 floats: W0[34][16] b0 W1[16][16] b1 W2[16][3] b2 */
} orc_scene;

typedef struct {
    double step;        /* lattice step delta_s in contracted arc length */
    double t_term;      /* early-termination threshold on transmittance (Sec. 5: 2e-4) */
    int early_term;     /* 1: stop after the sample at which T drops below t_term */
    int decide_f32;     /* 1: lattice / occupancy decisions taken in FP32 (the kernel's precision) */
    int no_mlp;         /* 1: output C_d only (RGB = C_d) */
    int contraction;    /* 0: contract_pi with its segment lattice (Sec. 3.2); 1: the spherical
                           contraction of mip-NeRF 360 (Eq. contract360) marched densely */
} orc_opts;

typedef struct {
    int region;             /* 0 inner, 1 + 2*j + (s < 0) for the outer region of axis j, sign s */
    double t0, t1;          /* world ray parameters of the ends (t1 = +inf for the last) */
    double a[3], b[3];      /* contracted end points */
    double len;             /* |b - a| */
    double s0;              /* cumulative contracted arc length at a */
} orc_seg;

/* Eq. (contract_pi), Sec. 3.2 */
int  orc_region(const double x[3]);
void orc_contract(const double x[3], double p[3]);
void orc_contract_in_region(int region, const double x[3], double p[3]);
void orc_uncontract(int region, const double p[3], double x[3]);

/* pinhole ray of pixel (i, j) of camera rec (16 floats: c2w[12], fx, fy, cx, cy) */
void orc_ray(const float *cam, int i, int j, double o[3], double d[3]);
int  orc_segments(const double o[3], const double d[3], orc_seg *segs);
double orc_t_of_s(const orc_seg *segs, int n, const double o[3], const double d[3], double s);
void orc_point_at(const orc_seg *segs, int n, double s, double p[3]);

/* summed, dequantised pre-activation feature t~(p) (Sec. 3.1, Sec. 4.2) */
void orc_field(const orc_scene *sc, const double p[3], double out[8], int *missing);
void orc_mlp(const float *w, const double cd[3], const double f[4], const double d[3], double out[3]);

int orc_render(const orc_scene *sc, const float *cams, int n_cams, int W, int H,
               const int32_t *pix, int n_pix, const orc_opts *opts, double *out, int n_threads);

/* Gradient of L = sum over the listed pixels of dl_drgb . C with respect to the dense float
 * grid, the planes and the MLP weights (dense float storage only; lattice, occupancy and
 * termination decisions frozen at their forward values).  g_grid [L^3][8], g_planes [3][R][R][8]
 * and g_mlp [883] are accumulated (caller zeroes them).  Single-threaded. */
int orc_render_grad(const orc_scene *sc, const float *cams, int n_cams, int W, int H,
                    const int32_t *pix, int n_pix, const orc_opts *opts, const double *dl_drgb,
                    double *g_grid, double *g_planes, double *g_mlp);

/* evaluated-lattice-sample sets (early termination off): bit k of row r is set iff
 * lattice sample k of ray r lies in an occupied finest cell; flag bit k is set where the
 * FP64 position lies within `eps` of a cell face. */
int orc_trace(const orc_scene *sc, const float *cams, int n_cams, int W, int H,
              const int32_t *pix, int n_pix, double step, int decide_f32, double eps,
              uint32_t *mask, uint32_t *flags, int words, int32_t *n_lattice, int n_threads,
              int contraction);

/* orc_trace with a choice of flags: decisive 0 flags every sample within eps of a cell face (as
 * orc_trace); decisive 1 flags, from the FP64 position and arc length, only the samples whose
 * outcome a move of eps can change: a finest cell of other occupancy within eps, an interior
 * segment boundary within eps (the contracted ray may jump there), or (k + 1) step within eps
 * of the total arc length.  Rows also flag lattice index n_lattice when that sample is within eps
 * of existing. */
int orc_trace_flagged(const orc_scene *sc, const float *cams, int n_cams, int W, int H,
                      const int32_t *pix, int n_pix, double step, int decide_f32, double eps,
                      uint32_t *mask, uint32_t *flags, int words, int32_t *n_lattice, int n_threads,
                      int contraction, int decisive);

/* Distinct data a set of rays reads (the reuse beside the bandwidth roofline): the render's own
 * evaluated samples (opts as in orc_render) each mark the eight grid voxels of their trilinear
 * interpolation that lie in stored blocks, the index-grid entry of their lowest corner's block,
 * and the four texels of each plane (clamped indices, as read).  counts[0..2] = distinct grid
 * voxels, plane texels, index entries.  uint8 block-sparse scenes only. */
int orc_footprint(const orc_scene *sc, const float *cams, int n_cams, int W, int H,
                  const int32_t *pix, int n_pix, const orc_opts *opts, uint64_t counts[3], int n_threads);

/* Ablation (Sec. 3.2, Table 2 (c)): the spherical contraction of mip-NeRF 360 and its dense
 * march.  orc_contract_sph maps |x|_2 <= 1 to itself and beyond to (2 - 1/|x|) x/|x|.  Sample k
 * of a ray sits at s_k = (k + 1/2) step for (k + 1) step < 2, at ray parameter t(s) = s for
 * s <= 1 and 1/(2 - s) beyond; its world step is t((k+1) step) - t(k step). */
void   orc_contract_sph(const double x[3], double p[3]);
double orc_sph_t_of_s(double s);
int    orc_sph_count(double step);
int    orc32_sph_count(float step);
void   orc32_sph_point(const float o[3], const float d[3], float step, int k, float p[3]);

/* FP32 decision replica (the kernel's traversal arithmetic, Sec. 3.2 + Sec. 5) */
typedef struct {
    int n;
    int region[ORC_MAX_SEGS];
    float a[ORC_MAX_SEGS][3], e[ORC_MAX_SEGS][3];
    float s0[ORC_MAX_SEGS + 1];
} orc32_segs;
void orc32_ray(const float *cam, int i, int j, float o[3], float d[3]);
void orc32_segments(const float o[3], const float d[3], orc32_segs *sg);
int  orc32_lattice_count(const orc32_segs *sg, float step);
int  orc32_sample_cell(const orc32_segs *sg, float step, int k, int N, int cell[3]);

#ifdef __cplusplus
}
#endif
#endif
