/*
 * FP64 brute-force CPU oracle for walk on stars (Sawhney, Miller, Gkioulekas,
 * Crane, "Walk on Stars", ACM TOG 42(4), 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this library: it exists so that tests, the smoke check and the CPU
 * baseline of the benchmark can check the CUDA path against a plain, slow,
 * obviously correct restatement of the method.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * Every geometric query is brute force over all primitives (Sec. 5, queries
 * Q.1-Q.3), the Neumann point sampler follows Algs. 5-6 on the oracle's own
 * plain median-split tree (Sec. 5.2), and the walk follows Alg. 1 in the
 * paper's order with the readings listed in wost_oracle.c.
 *
 * Conventions: dim is 2 (segments) or 3 (triangles); vertices are double
 * [nv*dim]; prims are int32 [np*dim]; flags are uint8 [np] (0 Dirichlet,
 * 1 Neumann).  Boundary data kinds:
 *   ORC_DATA_NONE       field absent (f only: zero source)
 *   ORC_DATA_PER_VERTEX values[nv], linearly interpolated on a primitive
 *   ORC_DATA_PER_CORNER values[np*dim], one value per primitive corner
 *   ORC_DATA_ANALYTIC   exact solution id (see ORC_FN_*); g = u, h = du/dn,
 *                       f = -Laplacian(u)
 *   ORC_DATA_GRID       f only: node-centred grid, (bi/tri)linear, clamped
 */
#ifndef WOST_ORACLE_H
#define WOST_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_DATA_NONE = 0, ORC_DATA_PER_VERTEX = 1, ORC_DATA_PER_CORNER = 2,
       ORC_DATA_ANALYTIC = 3, ORC_DATA_GRID = 4 };

/* Exact solutions used as analytic boundary data (u, grad u, -Lap u). */
enum { ORC_FN_ZERO = 0,        /* u = 0                                   */
       ORC_FN_EXP_COS = 1,     /* u = e^x cos y                           */
       ORC_FN_SIN2X_COS3Y = 2, /* u = sin 2x cos 3y, -Lap u = 13 u (2D)   */
       ORC_FN_QUAD3 = 3,       /* u = x^2 - y^2 + z/2                     */
       ORC_FN_BUMP = 4,        /* u = (1 - |x|^2) / (2 dim), -Lap u = 1   */
       ORC_FN_LINEAR = 5,      /* u = p0 + p1 x + p2 y + p3 z             */
       ORC_FN_LOG_RADIAL = 6,  /* 2D: p0 + p1 log|x-c|, 3D: p0 + p1/|x-c|,
                                  c = (p2, p3, p4)                        */
       ORC_FN_EXP_PLANE = 7    /* u = p0 exp(p1 x + p2 y + p3 z): solves the
                                  screened equation -Lap u + sigma u = 0 for
                                  sigma = p1^2 + p2^2 + p3^2               */
};

typedef struct {
    int kind;
    const double *values;  /* PER_VERTEX / PER_CORNER / GRID values        */
    int fn;                /* ANALYTIC: ORC_FN_*                           */
    double params[8];      /* ANALYTIC parameters                          */
    double origin[3];      /* GRID: position of node (0,0,0)               */
    double spacing[3];     /* GRID: node spacing                           */
    int dims[3];           /* GRID: node counts, x fastest in memory       */
} orc_field;

typedef struct orc_scene orc_scene;

/* Builds the oracle scene (copies all inputs).  Returns NULL on bad input. */
orc_scene *orc_scene_new(int dim, int nv, const double *vertices, int np,
                         const int32_t *prims, const uint8_t *flags,
                         const orc_field *g, const orc_field *h,
                         const orc_field *f);
void orc_scene_free(orc_scene *s);

/* App. B: data of the - side of double-sided primitives (flags 2 =
 * double-sided Dirichlet, 3 = double-sided Neumann).  NONE: g- = g+ and
 * h- = -h+ (a solution continuous across the sheet).  The + side of a
 * primitive is the one its normal n+ points away from. */
void orc_scene_set_minus(orc_scene *s, const orc_field *gm, const orc_field *hm);
int orc_scene_info(const orc_scene *s, int64_t *out /* [8] */);

/* Philox4x32-10 (Salmon et al., SC'11), one block. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);

/* Q.1 closest point on the Dirichlet boundary (brute force).  For each of n
 * points: out_d[i], out_xbar[i*3..], out_prim[i] (-1 and +inf if none). */
void orc_closest_dirichlet(const orc_scene *s, int64_t n, const double *x,
                           double *out_d, double *out_xbar, int32_t *out_prim);

/* Q.2 distance to the closest visibility-silhouette point of the Neumann
 * boundary within rmax (brute force); rmax if there is none.  out_sil is the
 * silhouette primitive index (vertex in 2D, edge in 3D) or -1. */
void orc_silhouette_distance(const orc_scene *s, int64_t n, const double *x,
                             const double *rmax, double *out_d,
                             int32_t *out_sil);

/* Q.3 first hit of the ray o + t v, 0 < t <= tmax, with the Neumann
 * boundary, skipping primitive `skip` (-1 for none). */
void orc_intersect_neumann(const orc_scene *s, int64_t n, const double *o,
                           const double *v, const double *tmax,
                           const int32_t *skip, int32_t *out_hit,
                           double *out_t, int32_t *out_prim);

/* Q.2 and Q.3 with the silhouette threshold moved to tau |v| (1 + |x|_inf)
 * (Q.2) or the segment-parameter / barycentric range widened by tol (Q.3):
 * positive values accept more, negative fewer.  Tests only: an answer
 * decided in single precision within rounding of a threshold lies between
 * the answers for a negative and a positive value. */
void orc_silhouette_distance_tol(const orc_scene *s, int64_t n, const double *x,
                                 const double *rmax, double tau, double *out_d);
void orc_intersect_neumann_tol(const orc_scene *s, int64_t n, const double *o,
                               const double *v, const double *tmax,
                               const int32_t *skip, double tol, int32_t *out_hit,
                               double *out_t);

/* Q.4 hierarchical Neumann sample (Algs. 5-6) for ball (x, r) with uniforms
 * drawn from the Philox stream (seed, ctr0, ctr1, ctr2, slot 1...).  Writes
 * z [3], n_z [3], pdf and the primitive (or -1). */
void orc_neumann_sample(const orc_scene *s, const double *x, double r,
                        uint64_t seed, uint32_t ctr0, uint32_t ctr1,
                        uint32_t ctr2, double *out_z, double *out_nz,
                        double *out_pdf, int32_t *out_prim);

/* Green's function of the ball B(x,R) at distance rho (App. A) and its
 * integral over the ball. */
double orc_green_ball(int dim, double rho, double R);
double orc_green_ball_norm(int dim, double R);
/* Source radius t ~ G_B(x, x + t v)/|G_B| from the uniforms of slot 0. */
double orc_source_radius(int dim, double R, double u1, double u2);

/* Exponentially scaled modified Bessel functions e^-x I0(x), e^-x I1(x),
 * e^x K0(x), e^x K1(x), x > 0, from their integral representations. */
double orc_bessel_i0e(double x);
double orc_bessel_i1e(double x);
double orc_bessel_k0e(double x);
double orc_bessel_k1e(double x);
/* Screened Poisson, sigma > 0 (App. A.2): Green's function of the ball
 * B(x,R) at distance rho, its integral over the ball, and the step weight
 * Q = P^sigma_B / P^free at distance rho <= R. */
double orc_screened_green_ball(int dim, double rho, double R, double sigma);
double orc_screened_green_ball_norm(int dim, double R, double sigma);
double orc_screened_q(int dim, double rho, double R, double sigma);

typedef struct {
    double epsilon, r_min;
    int max_steps;
    uint64_t seed;
    double offset;    /* relative ray-origin offset for on-boundary points */
    double vis_tmax;  /* visibility ray end for the Neumann sample (< 1)   */
    int n_threads;    /* 0 = all cores                                     */
    double sigma;     /* screening coefficient (0: Poisson)                */
    int screen_after; /* steps k >= screen_after solve the screened
                         equation (Tikhonov switch); 0 = every step        */
} orc_params;

/* Runs walks_per_point walks (walk ids first_walk ...) from each point and
 * writes FP64 per-point sums.  Point i draws the random stream of point
 * index point_base + i.  normals/on_neumann may be NULL.  per_walk, if not
 * NULL, receives every walk's estimate [n * walks]. */
int orc_solve(const orc_scene *s, int64_t n, const double *points,
              const double *normals, const uint8_t *on_neumann,
              int walks_per_point, uint32_t first_walk, uint32_t point_base,
              const orc_params *p, double *out_sum, double *out_sumsq,
              int64_t *out_steps, int64_t *out_capped, double *per_walk);

/* One walk with a per-step trace.  Each row has ORC_TRACE_COLS doubles:
 * x0 x1 x2 onNeumann d_D d_sil r hit t_boundary N S.  Returns the number of
 * rows written; *out_value receives the estimate. */
#define ORC_TRACE_COLS 11
int orc_walk_trace(const orc_scene *s, const double *x0, const double *n0,
                   int on_neumann, uint32_t point_index, uint32_t walk_index,
                   const orc_params *p, double *rows, int max_rows,
                   double *out_value, int *out_capped);

/* Exact solution u at n points (for tests). */
void orc_exact_u(int dim, int fn, const double *params, int64_t n,
                 const double *x, double *out);

#ifdef __cplusplus
}
#endif
#endif
