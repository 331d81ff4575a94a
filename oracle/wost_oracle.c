/*
 * FP64 brute-force CPU oracle for walk on stars -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code with the CUDA path.
 *
 * Paper: Sawhney, Miller, Gkioulekas, Crane, "Walk on Stars: A Grid-Free
 * Monte Carlo Method for PDEs with Neumann Boundary Conditions", 2023.
 *
 * What is computed, and where it comes from:
 *   - problem: Sec. 3.2, Eq. (PoissonEquation), mixed Dirichlet/Neumann;
 *   - estimator: Sec. 4.3 (WoSt estimator box) and Sec. 4.7 (final form),
 *     walked as in Alg. 1 (WalkOnStars);
 *   - Green's function of the ball and its integral: App. A.1;
 *   - direction sampling: Sec. 4.4, Eq. (DirectionalSampling); hemisphere
 *     flip on the Neumann boundary: Sec. 4.4.2;
 *   - source sampling: Sec. 4.6;
 *   - queries Q.1-Q.4: Sec. 5.  Q.1-Q.3 here are brute force over every
 *     primitive.  Q.2 uses the silhouette condition of Eq. (SilhouetteDef)
 *     at the closest point of every silhouette candidate (Alg. 3's leaf
 *     test applied to all candidates, without the hierarchy).  Q.4 follows
 *     Algs. 5-6 on a plain median-split binary tree built here.
 *   - random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
 *     random numbers: as easy as 1, 2, 3", SC'11), keyed by the seed, with
 *     counter (walk, point, step, slot).
 *
 * Readings where the paper is ambiguous (each is also listed in the design
 * notes of the repository):
 *   R1 signs: the Green's functions of App. A are positive, so with the
 *      outward normal derivative h the Neumann term is ADDED and the source
 *      term is added with f = -Lap(u): each step adds +N + S (Alg. 1 prints
 *      -N + S with a negative-semidefinite Laplacian; App. A's positive G
 *      fixes the sign used here).
 *   R2 Alg. 3's leaf returns the first silhouette edge below r; the Ensure
 *      line asks for the closest one, so d_sil is the minimum.
 *   R3 r = min(d_D, max(r_min, d_sil)) so that the ball never crosses the
 *      Dirichlet boundary (equal to Alg. 1's form whenever d_D >= r_min).
 *   R4 on the Neumann boundary, Q.2, Q.3 and the visibility ray start from
 *      x - delta n_x (footnote of Sec. 4.4), delta = offset*(1+|x|_inf);
 *      the visibility ray skips z's own primitive and ends at vis_tmax.
 *   R5 at the step cap the walk ends like an epsilon-shell hit: g at the
 *      closest Dirichlet point.
 *   R6 Q.4 child weights: 1/(4 pi d) in 3D (free-space G, Alg. 6); in 2D
 *      the free-space G = log(d)/2pi is not a positive weight, so 1/d.
 *      One fresh uniform per reservoir candidate in the leaf.
 *   R7 2D source radius t = R sqrt(U1 U2); 3D t = R (1/2 + sin(asin(2U-1)/3))
 *      (inverse CDF of Beta(2,2)); both are the normalised G_B of App. A.
 *   R12 a Neumann sample at distance exactly 0 from x contributes nothing.
 *   R14 the star radius is at most the diagonal of the boundary's bounding
 *      box (a ball that large around any point of the box holds the whole
 *      domain); it matters only without a Dirichlet boundary (pure Neumann
 *      problems, Sec. 6.4), where d_D is infinite.
 *   R15 screened steps (sigma > 0, from step screen_after on: the Tikhonov
 *      switch of Sec. 4.1) use G^sigma_B of App. A.2 for the Neumann term,
 *      the unscreened source density with weight |G_B| G^sigma_B / G_B for
 *      the source term, and continue with probability Q^sigma_B(x, x_next)
 *      drawn with the fourth uniform of slot 0 (Russian roulette).
 *   R13 a walk whose position lies outside the bounding box of the
 *      boundary grown by its largest side on every side (or is not finite)
 *      has left the domain: it ends like a capped walk (R5).  Exact
 *      arithmetic never gets there; single precision can, through a gap
 *      between two primitives.
 */
#include "wost_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* small vector helpers (always 3 components; z = 0 in 2D)            */
/* ------------------------------------------------------------------ */
typedef struct { double x, y, z; } V3;

static V3 mk(double x, double y, double z) { V3 r = {x, y, z}; return r; }
static V3 add(V3 a, V3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static V3 sub(V3 a, V3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static V3 scl(V3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static V3 crs(V3 a, V3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double len(V3 a) { return sqrt(dot(a, a)); }
static double maxabs(V3 a) {
    double m = fabs(a.x);
    if (fabs(a.y) > m) m = fabs(a.y);
    if (fabs(a.z) > m) m = fabs(a.z);
    return m;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11): round = two 32x32->64 multiplies, key Weyl   */
/* increments between rounds.                                          */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform in (0,1): the top 23 bits plus one half, scaled by 2^-23.  Every
 * value is exactly representable in single and double precision. */
static double u01(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

typedef struct {
    uint32_t key[2], ctr[4];
    uint32_t buf[4];
    int used;
} stream_t;

static void stream_init(stream_t *st, uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2,
                        uint32_t first_slot) {
    st->key[0] = (uint32_t)seed;
    st->key[1] = (uint32_t)(seed >> 32);
    st->ctr[0] = c0; st->ctr[1] = c1; st->ctr[2] = c2; st->ctr[3] = first_slot;
    st->used = 4;
}
static double stream_next(stream_t *st) {
    if (st->used == 4) {
        orc_philox4x32_10(st->ctr, st->key, st->buf);
        st->ctr[3] += 1;
        st->used = 0;
    }
    return u01(st->buf[st->used++]);
}

/* ------------------------------------------------------------------ */
/* Green's functions (App. A.1)                                        */
/* ------------------------------------------------------------------ */
double orc_green_ball(int dim, double rho, double R) {
    if (dim == 2) return log(R / rho) / (2.0 * M_PI);
    return (1.0 / rho - 1.0 / R) / (4.0 * M_PI);
}
double orc_green_ball_norm(int dim, double R) {
    return dim == 2 ? R * R / 4.0 : R * R / 6.0;
}
double orc_source_radius(int dim, double R, double u1, double u2) {
    if (dim == 2) return R * sqrt(u1 * u2);
    (void)u2;
    return R * (0.5 + sin(asin(2.0 * u1 - 1.0) / 3.0));
}

/* ------------------------------------------------------------------ */
/* Screened Poisson equation (App. A.2)                                */
/* ------------------------------------------------------------------ */
/* Exponentially scaled modified Bessel functions from their integral
 * representations (Abramowitz & Stegun 9.6.19 and 9.6.24):
 *   I_n(x) = (1/pi) int_0^pi e^{x cos t} cos(n t) dt,
 *   K_n(x) = int_0^inf e^{-x cosh t} cosh(n t) dt,
 * by the trapezoidal rule, which converges geometrically for these smooth
 * even integrands (periodic for I, decaying double-exponentially for K). */
#define ORC_BESSEL_N 4096
static double bessel_ie(int n, double x) {
    const double h = M_PI / ORC_BESSEL_N;
    double sum = 0.0;
    for (int j = 0; j <= ORC_BESSEL_N; ++j) {
        double t = j * h, w = (j == 0 || j == ORC_BESSEL_N) ? 0.5 : 1.0;
        sum += w * exp(x * (cos(t) - 1.0)) * (n ? cos(t) : 1.0);
    }
    return sum * h / M_PI;
}
static double bessel_ke(int n, double x) {
    /* the integrand is below e^-750 beyond T */
    const double T = acosh(1.0 + 750.0 / x);
    const double h = T / ORC_BESSEL_N;
    double sum = 0.0;
    for (int j = 0; j <= ORC_BESSEL_N; ++j) {
        double t = j * h, w = (j == 0 || j == ORC_BESSEL_N) ? 0.5 : 1.0;
        sum += w * exp(-x * (cosh(t) - 1.0)) * (n ? cosh(t) : 1.0);
    }
    return sum * h;
}
double orc_bessel_i0e(double x) { return bessel_ie(0, x); }
double orc_bessel_i1e(double x) { return bessel_ie(1, x); }
double orc_bessel_k0e(double x) { return bessel_ke(0, x); }
double orc_bessel_k1e(double x) { return bessel_ke(1, x); }

/* Eq. GreensFnsScreenedPoissonBall, written with the scaled Bessel
 * functions (2D) and exponentials (3D) so that nothing overflows. */
double orc_screened_green_ball(int dim, double rho, double R, double sigma) {
    const double sq = sqrt(sigma), a = R * sq, b = rho * sq;
    if (dim == 2) {
        double k0b = orc_bessel_k0e(b) * exp(-b);
        double i0b_ratio = orc_bessel_i0e(b) * orc_bessel_k0e(a) / orc_bessel_i0e(a) * exp(b - 2.0 * a);
        return (k0b - i0b_ratio) / (2.0 * M_PI);
    }
    /* sinh((R - rho) s) / sinh(R s) */
    double ratio = exp(-b) * (1.0 - exp(-2.0 * (a - b))) / (1.0 - exp(-2.0 * a));
    return ratio / (4.0 * M_PI * rho);
}
/* Eq. GreensFnsNormScreenedPoissonBall */
double orc_screened_green_ball_norm(int dim, double R, double sigma) {
    const double a = R * sqrt(sigma);
    if (dim == 2) return (1.0 - exp(-a) / orc_bessel_i0e(a)) / sigma;
    return (1.0 - 2.0 * a * exp(-a) / (1.0 - exp(-2.0 * a))) / sigma;
}
/* Eq. ScreenedPoissonKernelsSphere: Q at distance rho from the centre */
double orc_screened_q(int dim, double rho, double R, double sigma) {
    const double sq = sqrt(sigma), a = R * sq, b = rho * sq;
    if (dim == 2) {
        double k1b = orc_bessel_k1e(b) * exp(-b);
        double i1b_ratio = orc_bessel_i1e(b) * orc_bessel_k0e(a) / orc_bessel_i0e(a) * exp(b - 2.0 * a);
        return (k1b + i1b_ratio) * b;
    }
    /* (b cosh b - sinh b) e^-a / sinh a */
    double second = ((b - 1.0) * exp(b - 2.0 * a) + (b + 1.0) * exp(-b - 2.0 * a)) / (1.0 - exp(-2.0 * a));
    return exp(-b) * (b + 1.0) + second;
}

/* ------------------------------------------------------------------ */
/* exact solutions used as analytic boundary data                      */
/* ------------------------------------------------------------------ */
static double fn_u(int dim, int fn, const double *p, V3 x) {
    switch (fn) {
    case ORC_FN_EXP_COS: return exp(x.x) * cos(x.y);
    case ORC_FN_SIN2X_COS3Y: return sin(2 * x.x) * cos(3 * x.y);
    case ORC_FN_QUAD3: return x.x * x.x - x.y * x.y + 0.5 * x.z;
    case ORC_FN_BUMP: return (1.0 - dot(x, x)) / (2.0 * dim);
    case ORC_FN_LINEAR: return p[0] + p[1] * x.x + p[2] * x.y + p[3] * x.z;
    case ORC_FN_LOG_RADIAL: {
        double rho = len(sub(x, mk(p[2], p[3], dim == 3 ? p[4] : 0.0)));
        return dim == 2 ? p[0] + p[1] * log(rho) : p[0] + p[1] / rho;
    }
    case ORC_FN_EXP_PLANE: return p[0] * exp(p[1] * x.x + p[2] * x.y + p[3] * x.z);
    default: return 0.0;
    }
}
static V3 fn_grad(int dim, int fn, const double *p, V3 x) {
    switch (fn) {
    case ORC_FN_EXP_COS: return mk(exp(x.x) * cos(x.y), -exp(x.x) * sin(x.y), 0);
    case ORC_FN_SIN2X_COS3Y:
        return mk(2 * cos(2 * x.x) * cos(3 * x.y), -3 * sin(2 * x.x) * sin(3 * x.y), 0);
    case ORC_FN_QUAD3: return mk(2 * x.x, -2 * x.y, 0.5);
    case ORC_FN_BUMP: return scl(x, -1.0 / dim);
    case ORC_FN_LINEAR: return mk(p[1], p[2], p[3]);
    case ORC_FN_LOG_RADIAL: {
        V3 d = sub(x, mk(p[2], p[3], dim == 3 ? p[4] : 0.0));
        double rho = len(d);
        return dim == 2 ? scl(d, p[1] / (rho * rho)) : scl(d, -p[1] / (rho * rho * rho));
    }
    case ORC_FN_EXP_PLANE: {
        double u = p[0] * exp(p[1] * x.x + p[2] * x.y + p[3] * x.z);
        return mk(u * p[1], u * p[2], u * p[3]);
    }
    default: return mk(0, 0, 0);
    }
}
/* -Laplacian(u), the source f under reading R1 */
static double fn_neglap(int dim, int fn, const double *p, V3 x) {
    switch (fn) {
    case ORC_FN_SIN2X_COS3Y: return 13.0 * sin(2 * x.x) * cos(3 * x.y);
    case ORC_FN_BUMP: return 1.0;
    case ORC_FN_EXP_PLANE:
        return -(p[1] * p[1] + p[2] * p[2] + p[3] * p[3]) * p[0] * exp(p[1] * x.x + p[2] * x.y + p[3] * x.z);
    default: (void)dim; return 0.0;
    }
}

void orc_exact_u(int dim, int fn, const double *params, int64_t n, const double *x,
                 double *out) {
    double p[8] = {0};
    if (params) memcpy(p, params, sizeof p);
    for (int64_t i = 0; i < n; ++i) {
        V3 q = mk(x[i * dim], x[i * dim + 1], dim == 3 ? x[i * dim + 2] : 0.0);
        out[i] = fn_u(dim, fn, p, q);
    }
}

/* ------------------------------------------------------------------ */
/* scene                                                               */
/* ------------------------------------------------------------------ */
typedef struct {
    V3 lo, hi;
    int left, right;  /* children (internal) */
    int start, count; /* prim range in tree_prims (leaf: count > 0) */
} onode;

struct orc_scene {
    int dim, nv, np;
    V3 *V;
    int32_t *P;
    uint8_t *flags, *live;
    V3 *nrm;     /* unit outward normal per primitive */
    double *area; /* length (2D) or area (3D) */
    int nD, nN;
    int32_t *Dl, *Nl;
    /* silhouette candidates: 2D vertices (b = -1), 3D edges (a, b) */
    int nsil;
    int32_t *sa, *sb, *snadj, *sf0, *sf1;
    /* Q.4 tree */
    int nnodes;
    onode *nodes;
    int32_t *tprims;
    orc_field g, h, f;
    double *gv, *hv, *fv;
    /* App. B: data of the - side of double-sided primitives (flags 2, 3);
     * kind NONE: g- = g+, h- = -h+ */
    orc_field gm, hm;
    double *gmv, *hmv;
    double blo[3], bhi[3]; /* R13: grown bounding box of the vertices */
    double rmax;           /* R14: diagonal of the vertices' bounding box */
};

static V3 vert(const orc_scene *s, int i) { return s->V[i]; }
static V3 corner(const orc_scene *s, int prim, int k) { return s->V[s->P[prim * s->dim + k]]; }

static double *copy_vals(const orc_field *fd, int n) {
    if (!fd || !fd->values || n <= 0) return NULL;
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    memcpy(d, fd->values, sizeof(double) * (size_t)n);
    return d;
}
static int field_len(const orc_scene *s, const orc_field *fd) {
    if (!fd) return 0;
    switch (fd->kind) {
    case ORC_DATA_PER_VERTEX: return s->nv;
    case ORC_DATA_PER_CORNER: return s->np * s->dim;
    case ORC_DATA_GRID: return fd->dims[0] * fd->dims[1] * (s->dim == 3 ? fd->dims[2] : 1);
    default: return 0;
    }
}

/* --- plain median-split tree over the Neumann primitives (for Q.4) --- */
static V3 prim_centroid(const orc_scene *s, int p) {
    V3 c = mk(0, 0, 0);
    for (int k = 0; k < s->dim; ++k) c = add(c, corner(s, p, k));
    return scl(c, 1.0 / s->dim);
}
static const orc_scene *g_sort_scene;
static int g_sort_axis;
static double axis_of(V3 v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }
static int cmp_centroid(const void *A, const void *B) {
    int a = *(const int32_t *)A, b = *(const int32_t *)B;
    double ca = axis_of(prim_centroid(g_sort_scene, a), g_sort_axis);
    double cb = axis_of(prim_centroid(g_sort_scene, b), g_sort_axis);
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return (a > b) - (a < b);
}
static void box_grow(V3 *lo, V3 *hi, V3 p) {
    if (p.x < lo->x) lo->x = p.x; if (p.y < lo->y) lo->y = p.y; if (p.z < lo->z) lo->z = p.z;
    if (p.x > hi->x) hi->x = p.x; if (p.y > hi->y) hi->y = p.y; if (p.z > hi->z) hi->z = p.z;
}
static int build_node(orc_scene *s, int start, int count) {
    int id = s->nnodes++;
    onode nd;
    nd.lo = mk(INFINITY, INFINITY, INFINITY);
    nd.hi = mk(-INFINITY, -INFINITY, -INFINITY);
    V3 clo = nd.lo, chi = nd.hi;
    for (int i = start; i < start + count; ++i) {
        int p = s->tprims[i];
        for (int k = 0; k < s->dim; ++k) box_grow(&nd.lo, &nd.hi, corner(s, p, k));
        box_grow(&clo, &chi, prim_centroid(s, p));
    }
    nd.left = nd.right = -1;
    nd.start = start;
    nd.count = count;
    s->nodes[id] = nd;
    if (count > 4) {
        V3 ext = sub(chi, clo);
        int axis = 0;
        if (ext.y > ext.x) axis = 1;
        if (s->dim == 3 && ext.z > axis_of(ext, axis)) axis = 2;
        g_sort_scene = s;
        g_sort_axis = axis;
        qsort(s->tprims + start, (size_t)count, sizeof(int32_t), cmp_centroid);
        int half = count / 2;
        int l = build_node(s, start, half);
        int r = build_node(s, start + half, count - half);
        s->nodes[id].left = l;
        s->nodes[id].right = r;
        s->nodes[id].count = 0;
    }
    return id;
}

typedef struct { int32_t a, b, tri; } edge_rec;
static int cmp_edge(const void *A, const void *B) {
    const edge_rec *x = (const edge_rec *)A, *y = (const edge_rec *)B;
    if (x->a != y->a) return (x->a > y->a) - (x->a < y->a);
    if (x->b != y->b) return (x->b > y->b) - (x->b < y->b);
    return (x->tri > y->tri) - (x->tri < y->tri);
}

orc_scene *orc_scene_new(int dim, int nv, const double *vertices, int np, const int32_t *prims,
                         const uint8_t *flags, const orc_field *g, const orc_field *h,
                         const orc_field *f) {
    if ((dim != 2 && dim != 3) || nv <= 0 || np < 0) return NULL;
    for (int i = 0; i < np * dim; ++i)
        if (prims[i] < 0 || prims[i] >= nv) return NULL;
    orc_scene *s = (orc_scene *)calloc(1, sizeof(orc_scene));
    s->dim = dim; s->nv = nv; s->np = np;
    s->V = (V3 *)malloc(sizeof(V3) * (size_t)nv);
    for (int i = 0; i < nv; ++i)
        s->V[i] = mk(vertices[i * dim], vertices[i * dim + 1], dim == 3 ? vertices[i * dim + 2] : 0.0);
    s->P = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np * dim + 1));
    memcpy(s->P, prims, sizeof(int32_t) * (size_t)(np * dim));
    s->flags = (uint8_t *)malloc((size_t)np + 1);
    memcpy(s->flags, flags, (size_t)np);
    s->live = (uint8_t *)calloc((size_t)np + 1, 1);
    s->nrm = (V3 *)malloc(sizeof(V3) * (size_t)(np + 1));
    s->area = (double *)malloc(sizeof(double) * (size_t)(np + 1));
    s->Dl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np + 1));
    s->Nl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np + 1));
    for (int p = 0; p < np; ++p) {
        V3 a = corner(s, p, 0), b = corner(s, p, 1);
        V3 n;
        double A;
        if (dim == 2) {
            V3 t = sub(b, a);
            A = len(t);
            n = A > 0 ? mk(t.y / A, -t.x / A, 0) : mk(0, 0, 0);
        } else {
            V3 c = corner(s, p, 2);
            V3 cr = crs(sub(b, a), sub(c, a));
            double l = len(cr);
            A = 0.5 * l;
            n = l > 0 ? scl(cr, 1.0 / l) : mk(0, 0, 0);
        }
        s->nrm[p] = n;
        s->area[p] = A;
        s->live[p] = A > 0;
        if (!s->live[p]) continue;
        if (flags[p] & 1) s->Nl[s->nN++] = p; /* 1, 3: Neumann (3 double-sided) */
        else s->Dl[s->nD++] = p;            /* 0, 2: Dirichlet (2 double-sided) */
    }
    /* silhouette candidates */
    if (dim == 2) {
        int *cnt = (int *)calloc((size_t)nv, sizeof(int));
        int *f0 = (int *)malloc(sizeof(int) * (size_t)nv), *f1 = (int *)malloc(sizeof(int) * (size_t)nv);
        for (int i = 0; i < s->nN; ++i) {
            int p = s->Nl[i];
            for (int k = 0; k < 2; ++k) {
                int v = s->P[p * 2 + k];
                if (cnt[v] == 0) f0[v] = p;
                else if (cnt[v] == 1) f1[v] = p;
                cnt[v]++;
            }
        }
        s->sa = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
        s->sb = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
        s->snadj = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
        s->sf0 = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
        s->sf1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
        for (int v = 0; v < nv; ++v) {
            if (!cnt[v]) continue;
            int k = s->nsil++;
            s->sa[k] = v; s->sb[k] = -1; s->snadj[k] = cnt[v];
            s->sf0[k] = f0[v]; s->sf1[k] = cnt[v] >= 2 ? f1[v] : -1;
        }
        free(cnt); free(f0); free(f1);
    } else {
        int ne = 3 * s->nN;
        edge_rec *E = (edge_rec *)malloc(sizeof(edge_rec) * (size_t)(ne + 1));
        for (int i = 0; i < s->nN; ++i) {
            int p = s->Nl[i];
            for (int k = 0; k < 3; ++k) {
                int a = s->P[p * 3 + k], b = s->P[p * 3 + (k + 1) % 3];
                E[3 * i + k].a = a < b ? a : b;
                E[3 * i + k].b = a < b ? b : a;
                E[3 * i + k].tri = p;
            }
        }
        qsort(E, (size_t)ne, sizeof(edge_rec), cmp_edge);
        s->sa = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne + 1));
        s->sb = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne + 1));
        s->snadj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne + 1));
        s->sf0 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne + 1));
        s->sf1 = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ne + 1));
        for (int i = 0; i < ne;) {
            int j = i;
            while (j < ne && E[j].a == E[i].a && E[j].b == E[i].b) ++j;
            int k = s->nsil++;
            s->sa[k] = E[i].a; s->sb[k] = E[i].b; s->snadj[k] = j - i;
            s->sf0[k] = E[i].tri; s->sf1[k] = j - i >= 2 ? E[i + 1].tri : -1;
            i = j;
        }
        free(E);
    }
    /* Q.4 tree */
    s->tprims = (int32_t *)malloc(sizeof(int32_t) * (size_t)(s->nN + 1));
    memcpy(s->tprims, s->Nl, sizeof(int32_t) * (size_t)s->nN);
    s->nodes = (onode *)malloc(sizeof(onode) * (size_t)(2 * s->nN + 2));
    s->nnodes = 0;
    if (s->nN > 0) build_node(s, 0, s->nN);
    /* boundary data */
    orc_field none;
    memset(&none, 0, sizeof none);
    s->g = g ? *g : none;
    s->h = h ? *h : none;
    s->f = f ? *f : none;
    s->gv = copy_vals(g, field_len(s, g));
    s->hv = copy_vals(h, field_len(s, h));
    s->fv = copy_vals(f, field_len(s, f));
    s->g.values = s->gv; s->h.values = s->hv; s->f.values = s->fv;
    /* R13: bounding box of the vertices grown by its largest side */
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < nv; ++i) {
        double c[3] = {s->V[i].x, s->V[i].y, s->V[i].z};
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], c[a]);
            hi[a] = fmax(hi[a], c[a]);
        }
    }
    double m = 0.0, d2 = 0.0;
    for (int a = 0; a < dim; ++a) {
        m = fmax(m, hi[a] - lo[a]);
        d2 += (hi[a] - lo[a]) * (hi[a] - lo[a]);
    }
    s->rmax = sqrt(d2);
    for (int a = 0; a < 3; ++a) {
        s->blo[a] = lo[a] - m;
        s->bhi[a] = hi[a] + m;
    }
    return s;
}

/* R13: inside the grown bounding box (false for a non-finite position) */
static int in_bounds(const orc_scene *s, V3 x) {
    int in = x.x >= s->blo[0] && x.x <= s->bhi[0] && x.y >= s->blo[1] && x.y <= s->bhi[1];
    if (s->dim == 3) in = in && x.z >= s->blo[2] && x.z <= s->bhi[2];
    return in;
}

void orc_scene_free(orc_scene *s) {
    if (!s) return;
    free(s->V); free(s->P); free(s->flags); free(s->live); free(s->nrm); free(s->area);
    free(s->Dl); free(s->Nl); free(s->sa); free(s->sb); free(s->snadj); free(s->sf0);
    free(s->sf1); free(s->nodes); free(s->tprims); free(s->gv); free(s->hv); free(s->fv);
    free(s->gmv); free(s->hmv);
    free(s);
}

void orc_scene_set_minus(orc_scene *s, const orc_field *gm, const orc_field *hm) {
    orc_field none;
    memset(&none, 0, sizeof none);
    free(s->gmv); free(s->hmv);
    s->gm = gm ? *gm : none;
    s->hm = hm ? *hm : none;
    s->gmv = copy_vals(gm, field_len(s, gm));
    s->hmv = copy_vals(hm, field_len(s, hm));
    s->gm.values = s->gmv; s->hm.values = s->hmv;
}

int orc_scene_info(const orc_scene *s, int64_t *out) {
    out[0] = s->dim; out[1] = s->nD; out[2] = s->nN; out[3] = s->nsil;
    out[4] = s->nnodes; out[5] = s->np; out[6] = s->nv; out[7] = 0;
    return 0;
}

/* ------------------------------------------------------------------ */
/* primitive geometry                                                  */
/* ------------------------------------------------------------------ */
/* closest point on segment a-b; *t in [0,1] is the position along it */
static V3 closest_on_segment(V3 a, V3 b, V3 x, double *t) {
    V3 e = sub(b, a);
    double ee = dot(e, e);
    double s = ee > 0 ? dot(sub(x, a), e) / ee : 0.0;
    if (s < 0) s = 0;
    if (s > 1) s = 1;
    *t = s;
    return add(a, scl(e, s));
}

/* closest point on primitive p; bary receives the barycentric weights */
static V3 closest_on_prim(const orc_scene *s, int p, V3 x, double bary[3]) {
    V3 a = corner(s, p, 0), b = corner(s, p, 1);
    if (s->dim == 2) {
        double t;
        V3 q = closest_on_segment(a, b, x, &t);
        bary[0] = 1 - t; bary[1] = t; bary[2] = 0;
        return q;
    }
    V3 c = corner(s, p, 2);
    V3 n = s->nrm[p];
    /* projection onto the plane; inside the triangle -> done */
    V3 q = sub(x, scl(n, dot(sub(x, a), n)));
    V3 v0 = sub(b, a), v1 = sub(c, a), v2 = sub(q, a);
    double d00 = dot(v0, v0), d01 = dot(v0, v1), d11 = dot(v1, v1);
    double d20 = dot(v2, v0), d21 = dot(v2, v1);
    double den = d00 * d11 - d01 * d01;
    double lb = (d11 * d20 - d01 * d21) / den;
    double lc = (d00 * d21 - d01 * d20) / den;
    double la = 1 - lb - lc;
    if (la >= 0 && lb >= 0 && lc >= 0) {
        bary[0] = la; bary[1] = lb; bary[2] = lc;
        return q;
    }
    /* otherwise the closest point lies on one of the three edges */
    V3 corners[3] = {a, b, c};
    double best = INFINITY;
    V3 bq = a;
    for (int k = 0; k < 3; ++k) {
        double t;
        V3 e = closest_on_segment(corners[k], corners[(k + 1) % 3], x, &t);
        double d = len(sub(e, x));
        if (d < best) {
            best = d;
            bq = e;
            bary[0] = bary[1] = bary[2] = 0;
            bary[k] = 1 - t;
            bary[(k + 1) % 3] = t;
        }
    }
    return bq;
}

/* first intersection of the ray o + t v, 0 < t <= tmax, with primitive p.
 * tol widens (> 0) or narrows (< 0) the accepted range of the segment
 * parameter / barycentric coordinates; the walk uses the exact test, tol = 0
 * (the parity tests bracket a single-precision answer between tol = +-tau) */
static int ray_prim(const orc_scene *s, int p, V3 o, V3 v, double tmax, double *t_out, double tol) {
    V3 a = corner(s, p, 0), b = corner(s, p, 1);
    if (s->dim == 2) {
        V3 e = sub(b, a), ao = sub(a, o);
        double den = v.x * e.y - v.y * e.x;
        if (den == 0) return 0;
        double t = (ao.x * e.y - ao.y * e.x) / den;
        double u = (ao.x * v.y - ao.y * v.x) / den;
        if (u < -tol || u > 1 + tol || t <= 0 || t > tmax) return 0;
        *t_out = t;
        return 1;
    }
    /* Moller-Trumbore */
    V3 c = corner(s, p, 2);
    V3 e1 = sub(b, a), e2 = sub(c, a);
    V3 pv = crs(v, e2);
    double det = dot(e1, pv);
    if (det == 0) return 0;
    double inv = 1.0 / det;
    V3 tv = sub(o, a);
    double u = dot(tv, pv) * inv;
    if (u < -tol || u > 1 + tol) return 0;
    V3 qv = crs(tv, e1);
    double w = dot(v, qv) * inv;
    if (w < -tol || u + w > 1 + tol) return 0;
    double t = dot(e2, qv) * inv;
    if (t <= 0 || t > tmax) return 0;
    *t_out = t;
    return 1;
}

/* field evaluation on a primitive at barycentric weights */
static double interp_prim(const orc_scene *s, const orc_field *fd, int p, const double bary[3]) {
    double v = 0;
    for (int k = 0; k < s->dim; ++k) {
        double val = fd->kind == ORC_DATA_PER_VERTEX ? fd->values[s->P[p * s->dim + k]]
                                                     : fd->values[p * s->dim + k];
        v += bary[k] * val;
    }
    return v;
}
static void bary_of(const orc_scene *s, int p, V3 q, double bary[3]) {
    closest_on_prim(s, p, q, bary);
}
/* App. B: a double-sided primitive carries data for each of its sides */
static int double_sided(const orc_scene *s, int p) { return s->flags[p] >= 2; }
static double eval_g(const orc_scene *s, int p, V3 q, const double bary[3], int minus) {
    if (minus && (s->gm.kind == ORC_DATA_PER_VERTEX || s->gm.kind == ORC_DATA_PER_CORNER))
        return interp_prim(s, &s->gm, p, bary);
    if (s->g.kind == ORC_DATA_ANALYTIC) return fn_u(s->dim, s->g.fn, s->g.params, q);
    if (s->g.kind == ORC_DATA_PER_VERTEX || s->g.kind == ORC_DATA_PER_CORNER)
        return interp_prim(s, &s->g, p, bary);
    return 0.0;
}
/* h on the + side is du/dn+ (n+ the primitive's normal); on the - side
 * du/dn- with n- = -n+: the given - side data, else -h+ */
static double eval_h(const orc_scene *s, int p, V3 q, int minus) {
    if (s->h.kind == ORC_DATA_ANALYTIC) {
        double hp = dot(fn_grad(s->dim, s->h.fn, s->h.params, q), s->nrm[p]);
        return minus ? -hp : hp;
    }
    double bary[3];
    bary_of(s, p, q, bary);
    if (minus && (s->hm.kind == ORC_DATA_PER_VERTEX || s->hm.kind == ORC_DATA_PER_CORNER))
        return interp_prim(s, &s->hm, p, bary);
    if (s->h.kind == ORC_DATA_PER_VERTEX || s->h.kind == ORC_DATA_PER_CORNER) {
        double hp = interp_prim(s, &s->h, p, bary);
        return minus ? -hp : hp;
    }
    return 0.0;
}
static double grid_eval(const orc_scene *s, V3 y) {
    const orc_field *fd = &s->f;
    double c[3] = {y.x, y.y, y.z};
    int i0[3] = {0, 0, 0};
    double fr[3] = {0, 0, 0};
    int nd = s->dim;
    for (int a = 0; a < nd; ++a) {
        int n = fd->dims[a];
        double gpos = (c[a] - fd->origin[a]) / fd->spacing[a];
        if (gpos < 0) gpos = 0;
        if (gpos > n - 1) gpos = n - 1;
        int i = (int)floor(gpos);
        if (i > n - 2) i = n - 2;
        if (i < 0) i = 0;
        i0[a] = i;
        fr[a] = n >= 2 ? gpos - i : 0.0;
    }
    double acc = 0;
    int ncorner = 1 << nd;
    for (int m = 0; m < ncorner; ++m) {
        double w = 1;
        int idx[3] = {0, 0, 0};
        for (int a = 0; a < nd; ++a) {
            int bit = (m >> a) & 1;
            int n = fd->dims[a];
            idx[a] = i0[a] + (n >= 2 ? bit : 0);
            w *= bit ? fr[a] : 1 - fr[a];
        }
        size_t lin = (size_t)idx[0] + (size_t)fd->dims[0] * ((size_t)idx[1] + (nd == 3 ? (size_t)fd->dims[1] * idx[2] : 0));
        acc += w * fd->values[lin];
    }
    return acc;
}
static double eval_f(const orc_scene *s, V3 y) {
    if (s->f.kind == ORC_DATA_ANALYTIC) return fn_neglap(s->dim, s->f.fn, s->f.params, y);
    if (s->f.kind == ORC_DATA_GRID) return grid_eval(s, y);
    return 0.0;
}

/* ------------------------------------------------------------------ */
/* Q.1 - Q.3, brute force                                              */
/* ------------------------------------------------------------------ */
static double q_closest_dirichlet(const orc_scene *s, V3 x, V3 *xbar, int *prim, double bary[3]) {
    double best = INFINITY;
    *prim = -1;
    for (int i = 0; i < s->nD; ++i) {
        int p = s->Dl[i];
        double b[3];
        V3 q = closest_on_prim(s, p, x, b);
        double d = len(sub(q, x));
        if (d < best) {
            best = d;
            *xbar = q;
            *prim = p;
            bary[0] = b[0]; bary[1] = b[1]; bary[2] = b[2];
        }
    }
    return best;
}

/* Eq. SilhouetteDefinition at the candidate point pe = x + v: (v.n0)(v.n1) <=
 * 0.  tau relaxes (> 0) or tightens (< 0) the threshold to tau |v| (1 +
 * |x|_inf), the size of single-precision rounding in the product; the walk
 * uses tau = 0 */
static int is_silhouette(const orc_scene *s, int k, V3 v, double tau) {
    if (s->snadj[k] != 2) return 1; /* boundary (or non-manifold) edge/vertex */
    double a = dot(v, s->nrm[s->sf0[k]]), b = dot(v, s->nrm[s->sf1[k]]);
    return a * b <= tau;
}

static double q_silhouette_tol(const orc_scene *s, V3 x, double rmax, int *which, double tau) {
    double best = rmax;
    *which = -1;
    for (int k = 0; k < s->nsil; ++k) {
        V3 pe;
        if (s->dim == 2) {
            pe = vert(s, s->sa[k]);
        } else {
            double t;
            pe = closest_on_segment(vert(s, s->sa[k]), vert(s, s->sb[k]), x, &t);
        }
        V3 v = sub(pe, x);
        double d = len(v);
        double scale = 1.0 + fmax(fabs(x.x), fmax(fabs(x.y), fabs(x.z)));
        if (d < best && is_silhouette(s, k, v, tau * d * scale)) {
            best = d;
            *which = k;
        }
    }
    return best;
}
static double q_silhouette(const orc_scene *s, V3 x, double rmax, int *which) {
    return q_silhouette_tol(s, x, rmax, which, 0.0);
}

static int q_intersect_neumann_tol(const orc_scene *s, V3 o, V3 v, double tmax, int skip, double *t_out,
                                   int *prim, double tol) {
    double best = tmax;
    int hit = 0;
    *prim = -1;
    for (int i = 0; i < s->nN; ++i) {
        int p = s->Nl[i];
        if (p == skip) continue;
        double t;
        if (ray_prim(s, p, o, v, best, &t, tol)) {
            best = t;
            hit = 1;
            *prim = p;
        }
    }
    *t_out = best;
    return hit;
}
static int q_intersect_neumann(const orc_scene *s, V3 o, V3 v, double tmax, int skip, double *t_out,
                               int *prim) {
    return q_intersect_neumann_tol(s, o, v, tmax, skip, t_out, prim, 0.0);
}

/* ------------------------------------------------------------------ */
/* Q.4: Algs. 5-6 on the median-split tree                             */
/* ------------------------------------------------------------------ */
static int aabb_meets_ball(const onode *nd, V3 x, double r) {
    double c[3] = {x.x, x.y, x.z}, lo[3] = {nd->lo.x, nd->lo.y, nd->lo.z},
           hi[3] = {nd->hi.x, nd->hi.y, nd->hi.z};
    double d2 = 0;
    for (int a = 0; a < 3; ++a) {
        double e = 0;
        if (c[a] < lo[a]) e = lo[a] - c[a];
        else if (c[a] > hi[a]) e = c[a] - hi[a];
        d2 += e * e;
    }
    return d2 <= r * r;
}
static double child_weight(const orc_scene *s, const onode *nd, V3 x, double r) {
    if (!aabb_meets_ball(nd, x, r)) return 0.0;
    V3 c = scl(add(nd->lo, nd->hi), 0.5);
    double d = len(sub(c, x));
    if (d < 1e-12) d = 1e-12;
    return s->dim == 3 ? 1.0 / (4.0 * M_PI * d) : 1.0 / d;
}

static int q_neumann_sample(const orc_scene *s, V3 x, double r, stream_t *st, V3 *z, double *pdf) {
    *pdf = 0;
    if (s->nnodes == 0) return -1;
    int node = 0;
    double pdf_T = 1.0;
    /* Alg. 6: descend through one random child, weighted by proximity */
    while (s->nodes[node].count == 0) {
        const onode *L = &s->nodes[s->nodes[node].left], *R = &s->nodes[s->nodes[node].right];
        double wL = child_weight(s, L, x, r), wR = child_weight(s, R, x, r);
        double tot = wL + wR;
        if (!(tot > 0)) return -1;
        double pL = wL / tot;
        if (stream_next(st) < pL) {
            pdf_T *= pL;
            node = s->nodes[node].left;
        } else {
            pdf_T *= 1 - pL;
            node = s->nodes[node].right;
        }
    }
    /* leaf: pick one primitive meeting the ball, proportionally to area */
    const onode *lf = &s->nodes[node];
    double total = 0, pdf_t = 0;
    int chosen = -1;
    for (int i = lf->start; i < lf->start + lf->count; ++i) {
        int p = s->tprims[i];
        double b[3];
        V3 q = closest_on_prim(s, p, x, b);
        if (len(sub(q, x)) <= r) {
            total += s->area[p];
            if (stream_next(st) * total < s->area[p]) {
                chosen = p;
                pdf_t = pdf_T * s->area[p];
            }
        }
    }
    if (chosen < 0) return -1;
    pdf_t /= total;
    /* Alg. 5: uniform point on the chosen primitive */
    V3 a = corner(s, chosen, 0), b = corner(s, chosen, 1);
    if (s->dim == 2) {
        double u = stream_next(st);
        *z = add(a, scl(sub(b, a), u));
    } else {
        V3 c = corner(s, chosen, 2);
        double u1 = stream_next(st), u2 = stream_next(st);
        double su = sqrt(u1);
        *z = add(add(scl(a, 1 - su), scl(b, su * (1 - u2))), scl(c, su * u2));
    }
    *pdf = pdf_t / s->area[chosen];
    return chosen;
}

/* ------------------------------------------------------------------ */
/* public query wrappers                                               */
/* ------------------------------------------------------------------ */
static V3 load_pt(int dim, const double *x, int64_t i) {
    return mk(x[i * dim], x[i * dim + 1], dim == 3 ? x[i * dim + 2] : 0.0);
}

void orc_closest_dirichlet(const orc_scene *s, int64_t n, const double *x, double *out_d,
                           double *out_xbar, int32_t *out_prim) {
    for (int64_t i = 0; i < n; ++i) {
        V3 xb = mk(0, 0, 0);
        int p;
        double b[3];
        out_d[i] = q_closest_dirichlet(s, load_pt(s->dim, x, i), &xb, &p, b);
        out_xbar[i * 3] = xb.x; out_xbar[i * 3 + 1] = xb.y; out_xbar[i * 3 + 2] = xb.z;
        out_prim[i] = p;
    }
}
void orc_silhouette_distance(const orc_scene *s, int64_t n, const double *x, const double *rmax,
                             double *out_d, int32_t *out_sil) {
    for (int64_t i = 0; i < n; ++i) {
        int w;
        out_d[i] = q_silhouette(s, load_pt(s->dim, x, i), rmax[i], &w);
        out_sil[i] = w;
    }
}
/* the same brute-force queries with relaxed / tightened thresholds (tests
 * only: a single-precision answer decided within rounding of a threshold
 * must lie between the answers for -tau and +tau) */
void orc_silhouette_distance_tol(const orc_scene *s, int64_t n, const double *x, const double *rmax,
                                 double tau, double *out_d) {
    for (int64_t i = 0; i < n; ++i) {
        int w;
        out_d[i] = q_silhouette_tol(s, load_pt(s->dim, x, i), rmax[i], &w, tau);
    }
}
void orc_intersect_neumann_tol(const orc_scene *s, int64_t n, const double *o, const double *v,
                               const double *tmax, const int32_t *skip, double tol, int32_t *out_hit,
                               double *out_t) {
    for (int64_t i = 0; i < n; ++i) {
        double t;
        int p;
        out_hit[i] = q_intersect_neumann_tol(s, load_pt(s->dim, o, i), load_pt(s->dim, v, i), tmax[i],
                                             skip ? skip[i] : -1, &t, &p, tol);
        out_t[i] = t;
    }
}
void orc_intersect_neumann(const orc_scene *s, int64_t n, const double *o, const double *v,
                           const double *tmax, const int32_t *skip, int32_t *out_hit,
                           double *out_t, int32_t *out_prim) {
    for (int64_t i = 0; i < n; ++i) {
        double t;
        int p;
        out_hit[i] = q_intersect_neumann(s, load_pt(s->dim, o, i), load_pt(s->dim, v, i), tmax[i],
                                         skip ? skip[i] : -1, &t, &p);
        out_t[i] = t;
        out_prim[i] = p;
    }
}
void orc_neumann_sample(const orc_scene *s, const double *x, double r, uint64_t seed, uint32_t c0,
                        uint32_t c1, uint32_t c2, double *out_z, double *out_nz, double *out_pdf,
                        int32_t *out_prim) {
    stream_t st;
    stream_init(&st, seed, c0, c1, c2, 1);
    V3 z = mk(0, 0, 0);
    double pdf;
    int p = q_neumann_sample(s, load_pt(s->dim, x, 0), r, &st, &z, &pdf);
    out_z[0] = z.x; out_z[1] = z.y; out_z[2] = z.z;
    V3 nz = p >= 0 ? s->nrm[p] : mk(0, 0, 0);
    out_nz[0] = nz.x; out_nz[1] = nz.y; out_nz[2] = nz.z;
    *out_pdf = pdf;
    *out_prim = p;
}

/* ------------------------------------------------------------------ */
/* Alg. 1, iterated instead of recursed                                */
/* ------------------------------------------------------------------ */
static V3 sample_direction(int dim, double u1, double u2) {
    if (dim == 2) {
        double th = 2.0 * M_PI * u1;
        return mk(cos(th), sin(th), 0);
    }
    double zc = 1.0 - 2.0 * u1;
    double rr = sqrt(fmax(0.0, 1.0 - zc * zc));
    double ph = 2.0 * M_PI * u2;
    return mk(rr * cos(ph), rr * sin(ph), zc);
}

static double walk(const orc_scene *s, V3 x, V3 nx, int onN, uint32_t pidx, uint32_t widx,
                   const orc_params *pr, int *steps_out, int *capped_out, double *rows,
                   int max_rows, int *nrows) {
    const int dim = s->dim;
    double acc = 0.0;
    int k = 0;
    *capped_out = 0;
    if (nrows) *nrows = 0;
    for (;; ++k) {
        /* distance to the Dirichlet boundary (Q.1) */
        V3 xbar = mk(0, 0, 0);
        int primD;
        double bary[3] = {0, 0, 0};
        int lost = !in_bounds(s, x); /* R13 */
        double dD = q_closest_dirichlet(s, x, &xbar, &primD, bary);
        int last = dD < pr->epsilon || k + 1 >= pr->max_steps || lost;
        if (last) {
            /* epsilon shell: return g at the closest point; R5, R13: same at
             * the cap and outside the grown bounding box */
            if (dD >= pr->epsilon) *capped_out = 1;
            /* App. B: the - side's data when x lies on the side of a
             * double-sided primitive that its normal n+ points into */
            int minus = primD >= 0 && double_sided(s, primD) && !(dot(sub(xbar, x), s->nrm[primD]) > 0);
            if (primD >= 0) acc += eval_g(s, primD, xbar, bary, minus);
            if (rows && *nrows < max_rows) {
                double *row = rows + (size_t)(*nrows) * ORC_TRACE_COLS;
                row[0] = x.x; row[1] = x.y; row[2] = x.z; row[3] = onN; row[4] = dD;
                row[5] = NAN; row[6] = NAN; row[7] = 0; row[8] = NAN; row[9] = 0; row[10] = 0;
                ++*nrows;
            }
            break;
        }
        /* R4: offset query origin when on the Neumann boundary */
        double delta = pr->offset * (1.0 + maxabs(x));
        V3 xq = onN ? sub(x, scl(nx, delta)) : x;
        /* distance to the visibility silhouette (Q.2) within d_D */
        int silk;
        double dsil = q_silhouette(s, xq, dD, &silk);
        /* star radius (R3), at most the scene's diameter (R14) */
        double r = fmin(fmin(dD, fmax(pr->r_min, dsil)), s->rmax);
        /* screening coefficient of this step (Tikhonov switch, Sec. 4.1) */
        double sig = (pr->sigma > 0 && k >= pr->screen_after) ? pr->sigma : 0.0;
        /* direction, hemisphere about -n_x on the Neumann boundary */
        uint32_t key[2] = {(uint32_t)pr->seed, (uint32_t)(pr->seed >> 32)};
        uint32_t ctr[4] = {widx, pidx, (uint32_t)k, 0u}, w4[4];
        orc_philox4x32_10(ctr, key, w4);
        double u1 = u01(w4[0]), u2 = u01(w4[1]), u3 = u01(w4[2]), u4 = u01(w4[3]);
        V3 v = sample_direction(dim, u1, u2);
        if (onN && dot(nx, v) > 0) v = scl(v, -1.0);
        /* first hit with the Neumann part of the star boundary (Q.3) */
        double th;
        int hprim;
        int hit = q_intersect_neumann(s, xq, v, r, -1, &th, &hprim);
        V3 p, np = mk(0, 0, 0);
        if (hit) {
            p = add(xq, scl(v, th));
            np = s->nrm[hprim];
            /* App. B: at a double-sided sheet the walk stays on the side it
             * came from: the outward normal there is the one it moves along */
            if (double_sided(s, hprim) && dot(v, np) < 0) np = scl(np, -1.0);
        } else {
            p = add(x, scl(v, r));
        }
        /* Neumann contribution from a separate sample z (Q.4) */
        stream_t st;
        stream_init(&st, pr->seed, widx, pidx, (uint32_t)k, 1);
        V3 z = mk(0, 0, 0);
        double pdf;
        int zprim = q_neumann_sample(s, x, r, &st, &z, &pdf);
        double Nterm = 0.0;
        if (zprim >= 0 && pdf > 0) {
            double dz = len(sub(z, x));
            /* R12: a sample at zero distance from x (G infinite, a set of
             * measure zero reached only through rounding) is skipped */
            if (dz < r && dz > 0) {
                double tvis;
                int vp;
                int occluded = q_intersect_neumann(s, xq, sub(z, xq), pr->vis_tmax, zprim, &tvis, &vp);
                if (!occluded) {
                    double alpha = onN ? 0.5 : 1.0;
                    double G = sig > 0 ? orc_screened_green_ball(dim, dz, r, sig) : orc_green_ball(dim, dz, r);
                    /* App. B: the data of the side of a double-sided sheet
                     * that faces the query point xq (which lies off the
                     * boundary on the walk's side, R4) */
                    int minus = double_sided(s, zprim) && !(dot(sub(z, xq), s->nrm[zprim]) > 0);
                    Nterm = G * eval_h(s, zprim, z, minus) / (alpha * pdf);
                }
            }
        }
        /* source contribution, reusing the direction v */
        double Sterm = 0.0;
        double ts = orc_source_radius(dim, r, dim == 2 ? u2 : u3, u3);
        if (s->f.kind != ORC_DATA_NONE) {
            double tb = len(sub(p, x));
            if (ts < tb) {
                /* y drawn from G_B / |G_B|; under screening the estimate is
                 * G^sigma_B(x,y) f(y) / pdf(y) = |G_B| (G^sigma_B / G_B)(ts) f(y) */
                double w = orc_green_ball_norm(dim, r);
                if (sig > 0) w *= orc_screened_green_ball(dim, ts, r, sig) / orc_green_ball(dim, ts, r);
                Sterm = w * eval_f(s, add(x, scl(v, ts)));
            }
        }
        /* R1: each step adds the Neumann and source terms */
        acc += Nterm + Sterm;
        if (rows && *nrows < max_rows) {
            double *row = rows + (size_t)(*nrows) * ORC_TRACE_COLS;
            row[0] = x.x; row[1] = x.y; row[2] = x.z; row[3] = onN; row[4] = dD;
            row[5] = dsil; row[6] = r; row[7] = hit; row[8] = len(sub(p, x));
            row[9] = Nterm; row[10] = Sterm;
            ++*nrows;
        }
        /* screened step (App. A.2): the walk continues to p with probability
         * Q^sigma_B(x, p) (Russian roulette with the fourth uniform of slot 0)
         * and is otherwise absorbed, contributing nothing more */
        if (sig > 0 && u4 >= orc_screened_q(dim, len(sub(p, x)), r, sig)) break;
        x = p;
        nx = np;
        onN = hit;
    }
    *steps_out = k + 1;
    return acc;
}

int orc_walk_trace(const orc_scene *s, const double *x0, const double *n0, int on_neumann,
                   uint32_t point_index, uint32_t walk_index, const orc_params *p, double *rows,
                   int max_rows, double *out_value, int *out_capped) {
    int steps, nrows = 0;
    V3 x = load_pt(s->dim, x0, 0);
    V3 n = n0 ? load_pt(s->dim, n0, 0) : mk(0, 0, 0);
    *out_value = walk(s, x, n, on_neumann, point_index, walk_index, p, &steps, out_capped, rows,
                      max_rows, &nrows);
    return nrows;
}

/* ------------------------------------------------------------------ */
/* multi-threaded solve                                                */
/* ------------------------------------------------------------------ */
typedef struct {
    const orc_scene *s;
    int64_t n;
    const double *points, *normals;
    const uint8_t *onN;
    int walks;
    uint32_t first_walk;
    uint32_t point_base;
    const orc_params *p;
    double *sum, *sumsq, *per_walk;
    int64_t *steps, *capped;
    int64_t next;
    pthread_mutex_t mu;
} job_t;

static void *worker(void *arg) {
    job_t *J = (job_t *)arg;
    const int dim = J->s->dim;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t i = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (i >= J->n) break;
        V3 x0 = load_pt(dim, J->points, i);
        V3 n0 = J->normals ? load_pt(dim, J->normals, i) : mk(0, 0, 0);
        int on = J->onN ? J->onN[i] != 0 : 0;
        double sm = 0, sq = 0;
        int64_t st = 0, cp = 0;
        for (int j = 0; j < J->walks; ++j) {
            int steps, capped;
            double val = walk(J->s, x0, n0, on, J->point_base + (uint32_t)i, J->first_walk + (uint32_t)j, J->p, &steps,
                              &capped, NULL, 0, NULL);
            sm += val;
            sq += val * val;
            st += steps;
            cp += capped;
            if (J->per_walk) J->per_walk[i * J->walks + j] = val;
        }
        J->sum[i] = sm;
        J->sumsq[i] = sq;
        J->steps[i] = st;
        J->capped[i] = cp;
    }
    return NULL;
}

int orc_solve(const orc_scene *s, int64_t n, const double *points, const double *normals,
              const uint8_t *on_neumann, int walks_per_point, uint32_t first_walk,
              uint32_t point_base, const orc_params *p, double *out_sum, double *out_sumsq,
              int64_t *out_steps, int64_t *out_capped, double *per_walk) {
    job_t J;
    J.point_base = point_base;
    J.s = s; J.n = n; J.points = points; J.normals = normals; J.onN = on_neumann;
    J.walks = walks_per_point; J.first_walk = first_walk; J.p = p;
    J.sum = out_sum; J.sumsq = out_sumsq; J.steps = out_steps; J.capped = out_capped;
    J.per_walk = per_walk; J.next = 0;
    pthread_mutex_init(&J.mu, NULL);
    int nt = p->n_threads > 0 ? p->n_threads : (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nt < 1) nt = 1;
    if (nt > 512) nt = 512;
    pthread_t th[512];
    for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, worker, &J);
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J.mu);
    return nt;
}
