/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for 3D-BBS
 * (arxiv 2310.10023).  TEST INFRASTRUCTURE ONLY: the product path never
 * includes, links or calls it.  Build: gcc -O2 -ffp-contract=off
 * -fno-fast-math (FP32 products and sums must round one by one).
 *
 * Every function names the passage of the paper it follows.  Where the paper
 * is silent or ambiguous the reading taken is stated beside the code.
 * All functions are pinned by the CPU tests (closed forms, set definitions,
 * brute force on tiny inputs, planted poses).
 */
#define _POSIX_C_SOURCE 199309L
#include "oracle.h"
#ifdef _OPENMP
#include <omp.h>
#endif

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

/* ======================================================================== */
/* small helpers                                                             */
/* ======================================================================== */

/* floor(x / 2^l) for a signed integer, written as plain floor division */
static int64_t floordiv_pow2(int64_t x, int l)
{
    int64_t d = (int64_t)1 << l;
    if (x >= 0) return x / d;
    return -((-x + d - 1) / d);
}

static double now_ms(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec * 1e3 + (double)ts.tv_nsec * 1e-6;
}

/* ======================================================================== */
/* Pose grid: Sec. III-B Eq. (2)-(5), Sec. III-D Eq. (12) and (14)           */
/* ======================================================================== */

/* Eq. (2): delta(r) = arccos(1 - r^2 / (2 d_max^2)).  Reading: the argument is
 * clamped to [-1, 1] (for r > 2 d_max the paper's formula is undefined; the
 * clamp gives delta = pi there).  d_max <= 0 also gives pi. */
double orc_delta(double r, double d_max)
{
    if (!(d_max > 0.0)) return acos(-1.0);
    double x = 1.0 - (r * r) / (2.0 * d_max * d_max);
    if (x < -1.0) x = -1.0;
    if (x > 1.0) x = 1.0;
    return acos(x);
}

/* d_max reading: the maximum range of the scan is taken from the data, as the
 * largest Euclidean norm of a scan point (FP64, fixed order). */
double orc_scan_dmax(const float* s, int64_t k)
{
    double m = 0.0;
    for (int64_t i = 0; i < k; ++i) {
        double x = s[3 * i], y = s[3 * i + 1], z = s[3 * i + 2];
        double d = sqrt((x * x + y * y) + z * z);
        if (d > m) m = d;
    }
    return m;
}

int orc_grid_build(double r, int levels, double d_max, const orc_ranges* rg,
                   uint32_t flags, orc_grid* g)
{
    if (!(r > 0.0) || levels < 1 || levels > ORC_MAX_LEVELS) return ORC_EINVAL;
    memset(g, 0, sizeof(*g));
    g->levels = levels;
    g->r = r;
    g->d_max = d_max;
    g->flags = flags;
    for (int i = 0; i < 3; ++i) {
        if (!(rg->ang_hi[i] >= rg->ang_lo[i])) return ORC_EINVAL;
        if (!(rg->hi[i] >= rg->lo[i])) return ORC_EINVAL;
        g->ang_lo[i] = rg->ang_lo[i];
        g->ang_range[i] = rg->ang_hi[i] - rg->ang_lo[i];
    }
    for (int l = 0; l < levels; ++l) {
        int src = (flags & ORC_TRANSLATION_ONLY) ? 0 : l;
        double rl = ldexp(r, src);              /* r_l = 2^l r, Sec. III-C */
        g->delta[l] = orc_delta(rl, d_max);     /* Eq. (2)               */
        for (int i = 0; i < 3; ++i) {
            double W = g->ang_range[i];
            /* Eq. (12): delta' = W / ceil(W / delta).  A zero-width range
             * (reading) has one segment of width 0. */
            int64_t n = 1;
            if (W > 0.0) {
                double q = ceil(W / g->delta[l]);
                n = (int64_t)q;
                if (n < 1) n = 1;
            }
            g->N[l][i] = n;
            g->dprime[l][i] = W / (double)n;
        }
    }
    /* Eq. (14): a = ceil(delta'(r_l) / delta'(r_{l-1})) when delta'(r_{l-1}) is
     * smaller than the range, else 1.  Reading: delta'_l / delta'_{l-1} equals
     * N_{l-1} / N_l exactly, so the ceiling is taken in integers to avoid a
     * rounding of the FP64 quotient pushing an exact integer ratio up by one. */
    for (int l = 1; l < levels; ++l)
        for (int i = 0; i < 3; ++i) {
            int64_t np = g->N[l][i], nc = g->N[l - 1][i];
            if ((flags & ORC_TRANSLATION_ONLY) || nc <= 1) g->a[l][i] = 1;
            else g->a[l][i] = (nc + np - 1) / np;
        }
    /* Eq. (3)-(5) in 3-D: w_min = floor(W_min / r_lmax), w_max = ceil(W_max / r_lmax) */
    double rmax = ldexp(r, levels - 1);
    for (int i = 0; i < 3; ++i) {
        double a = floor(rg->lo[i] / rmax), b = ceil(rg->hi[i] / rmax);
        if (!(fabs(a) < 1e15) || !(fabs(b) < 1e15)) return ORC_EKEYRANGE;
        g->wmin[i] = (int64_t)a;
        g->wmax[i] = (int64_t)b;
        /* every leaf translation index must stay within +-2^20 fine voxels */
        int64_t tlo = g->wmin[i] * ((int64_t)1 << (levels - 1));
        int64_t thi = (g->wmax[i] + 1) * ((int64_t)1 << (levels - 1));
        if (tlo < -((int64_t)1 << 20) || thi > ((int64_t)1 << 20)) return ORC_EKEYRANGE;
    }
    return ORC_OK;
}

/* Angle of segment index c.  Reading: the segment centre W_min + (c + 1/2) delta'
 * (the paper gives no offset); ORC_ANGLE_LOWER_EDGE selects W_min + c delta'. */
double orc_angle(const orc_grid* g, int level, int axis, int64_t c)
{
    double dp = g->dprime[level][axis];
    if (g->flags & ORC_ANGLE_LOWER_EDGE) return g->ang_lo[axis] + (double)c * dp;
    return g->ang_lo[axis] + ((double)c + 0.5) * dp;
}

/* Sec. III-A: x = [x, y, z, alpha, beta, gamma] with roll, pitch, yaw.
 * Reading: R = Rz(gamma) Ry(beta) Rx(alpha).  Entries in FP64 in a fixed
 * order, then A = fl32(R / r) so that floor(A s) is the fine voxel key. */
void orc_rotation(const orc_grid* g, int level, int64_t ia, int64_t ib, int64_t ig, float A[9])
{
    double al = orc_angle(g, level, 0, ia);
    double be = orc_angle(g, level, 1, ib);
    double ga = orc_angle(g, level, 2, ig);
    double ca = cos(al), sa = sin(al);
    double cb = cos(be), sb = sin(be);
    double cg = cos(ga), sg = sin(ga);
    double R[9];
    R[0] = cg * cb;
    R[1] = (cg * sb) * sa - sg * ca;
    R[2] = (cg * sb) * ca + sg * sa;
    R[3] = sg * cb;
    R[4] = (sg * sb) * sa + cg * ca;
    R[5] = (sg * sb) * ca - cg * sa;
    R[6] = -sb;
    R[7] = cb * sa;
    R[8] = cb * ca;
    for (int i = 0; i < 9; ++i) A[i] = (float)(R[i] / g->r);
}

/* Rotational children of angle index c at level l (Eq. (13), (14)): the
 * half-open index range [*lo, *hi) at level l-1.
 *
 * Reading: Eq. (13) writes the children as a*c + j, j < a.  That nests the
 * level grids only when N_{l-1} = a N_l; otherwise (N_{l-1} = 155, N_l = 77
 * gives a = 3) the children of the last parents lie far outside the parent's
 * segment and its score bounds nothing.  The reading taken: the children of
 * segment c are the level-(l-1) segments whose centres lie inside segment c,
 * i.e. the c' with floor((c' + 1/2) N_l / N_{l-1}) = c.  This equals a*c + j
 * whenever N_{l-1} = a N_l, gives at most a children (a = ceil of the step
 * ratio, Eq. (14)) and gives every level-(l-1) index exactly one parent.
 * ORC_CHILD_LITERAL selects the literal a*c + j, dropping indices >= N_{l-1}. */
static int64_t child_lo(int64_t np, int64_t nc, int64_t c)
{
    /* smallest c' with (2c' + 1) np >= 2 c nc */
    int64_t num = 2 * c * nc - np;
    if (num <= 0) return 0;
    return (num + 2 * np - 1) / (2 * np);
}

void orc_child_range(const orc_grid* g, int l, int axis, int64_t c, int64_t* lo, int64_t* hi)
{
    int64_t np = g->N[l][axis], nc = g->N[l - 1][axis];
    if (g->flags & ORC_CHILD_LITERAL) {
        int64_t a = g->a[l][axis];
        *lo = a * c;
        *hi = a * c + a;
        if (*lo > nc) *lo = nc;
        if (*hi > nc) *hi = nc;
        return;
    }
    *lo = child_lo(np, nc, c);
    *hi = child_lo(np, nc, c + 1);
    if (*hi > nc) *hi = nc;
}

/* Number of children of a node: 8 translations (2c + j, Eq. (13)) times the
 * rotational children of each angle axis. */
int64_t orc_num_children(const orc_grid* g, const int32_t node[7])
{
    int l = node[6];
    if (l <= 0) return 0;
    int64_t n = 8;
    for (int i = 0; i < 3; ++i) {
        int64_t lo, hi;
        orc_child_range(g, l, i, node[3 + i], &lo, &hi);
        n *= (hi - lo);
    }
    return n;
}

/* children in canonical order (alpha, beta, gamma, x, y, z), Eq. (13) */
int64_t orc_children(const orc_grid* g, const int32_t p[7], int32_t* out, int64_t cap)
{
    int l = p[6];
    if (l <= 0) return 0;
    int64_t lo[3], hi[3];
    for (int i = 0; i < 3; ++i) orc_child_range(g, l, i, p[3 + i], &lo[i], &hi[i]);
    int64_t cnt = 0;
    for (int64_t ca = lo[0]; ca < hi[0]; ++ca)
        for (int64_t cb = lo[1]; cb < hi[1]; ++cb)
            for (int64_t cg = lo[2]; cg < hi[2]; ++cg)
                for (int jx = 0; jx < 2; ++jx)
                    for (int jy = 0; jy < 2; ++jy)
                        for (int jz = 0; jz < 2; ++jz) {
                            if (cnt < cap) {
                                int32_t* c = out + 7 * cnt;
                                c[0] = 2 * p[0] + jx;
                                c[1] = 2 * p[1] + jy;
                                c[2] = 2 * p[2] + jz;
                                c[3] = (int32_t)ca;
                                c[4] = (int32_t)cb;
                                c[5] = (int32_t)cg;
                                c[6] = l - 1;
                            }
                            ++cnt;
                        }
    return cnt;
}

/* ======================================================================== */
/* Sparse hash voxel maps: Sec. III-C, Eq. (10)                              */
/* ======================================================================== */

typedef struct {
    int32_t x, y, z;
    int32_t used;
} orc_slot;

typedef struct {
    orc_slot* slot;
    int64_t T;          /* number of buckets (T_l)       */
    int64_t count;      /* stored voxels                 */
    int64_t collisions; /* voxels not in their home slot */
} orc_table;

struct orc_maps {
    int levels;
    double r;
    uint32_t flags;
    double lo[3], hi[3];
    orc_table lv[ORC_MAX_LEVELS];
};

/* f(v): the paper cites an unresolvable reference for the tuple hash.  Any
 * function gives the same occupancy, so this uses the XOR-of-primes spatial
 * hash of Teschner et al. (2003); hash(v) = f(v) mod T_l, Eq. (10). */
static uint64_t orc_f(int32_t x, int32_t y, int32_t z)
{
    return ((uint64_t)(uint32_t)x * 73856093ull) ^ ((uint64_t)(uint32_t)y * 19349663ull) ^
           ((uint64_t)(uint32_t)z * 83492791ull);
}

/* Open addressing (Sec. III-C): when a bucket is taken by another voxel the
 * bucket index is incremented until an empty one is found.  Returns 1 if the
 * voxel was inserted, 0 if already present. */
static int table_insert(orc_table* t, int32_t x, int32_t y, int32_t z)
{
    int64_t h = (int64_t)(orc_f(x, y, z) % (uint64_t)t->T);
    int64_t i = h;
    for (;;) {
        orc_slot* s = &t->slot[i];
        if (!s->used) {
            s->x = x; s->y = y; s->z = z; s->used = 1;
            t->count++;
            if (i != h) t->collisions++;
            return 1;
        }
        if (s->x == x && s->y == y && s->z == z) return 0;
        i = (i + 1 == t->T) ? 0 : i + 1;
    }
}

static int table_contains(const orc_table* t, int32_t x, int32_t y, int32_t z)
{
    int64_t i = (int64_t)(orc_f(x, y, z) % (uint64_t)t->T);
    for (;;) {
        const orc_slot* s = &t->slot[i];
        if (!s->used) return 0;
        if (s->x == x && s->y == y && s->z == z) return 1;
        i = (i + 1 == t->T) ? 0 : i + 1;
    }
}

static int table_init(orc_table* t, int64_t T)
{
    t->slot = (orc_slot*)calloc((size_t)T, sizeof(orc_slot));
    if (!t->slot) return ORC_ENOMEM;
    t->T = T;
    t->count = 0;
    t->collisions = 0;
    return ORC_OK;
}

/* growable set used only to de-duplicate keys while building a level */
static int set_add(orc_table* t, int32_t x, int32_t y, int32_t z)
{
    if ((t->count + 1) * 2 > t->T) {
        orc_table n;
        if (table_init(&n, 2 * t->T + 1)) return ORC_ENOMEM;
        for (int64_t i = 0; i < t->T; ++i)
            if (t->slot[i].used) table_insert(&n, t->slot[i].x, t->slot[i].y, t->slot[i].z);
        free(t->slot);
        *t = n;
    }
    table_insert(t, x, y, z);
    return ORC_OK;
}

/* "we seek T_l until the hash collision rate becomes small (e.g. 0.1%)".
 * Reading: T_l starts at 2n+1 and grows as T <- 2T+1 until the fraction of
 * voxels outside their home bucket is at most 0.1%, stopping at load 1/4. */
static int table_from_keys(orc_table* out, const int32_t* keys, int64_t n)
{
    int64_t T = 2 * n + 1;
    for (;;) {
        orc_table t;
        if (table_init(&t, T)) return ORC_ENOMEM;
        for (int64_t i = 0; i < n; ++i) table_insert(&t, keys[3 * i], keys[3 * i + 1], keys[3 * i + 2]);
        if (n == 0 || (double)t.collisions <= 0.001 * (double)n || T >= 4 * n) {
            *out = t;
            return ORC_OK;
        }
        free(t.slot);
        T = 2 * T + 1;
    }
}

/* keys stored in a set, in table order */
static int64_t set_keys(const orc_table* t, int32_t* out)
{
    int64_t c = 0;
    for (int64_t i = 0; i < t->T; ++i)
        if (t->slot[i].used) {
            out[3 * c] = t->slot[i].x;
            out[3 * c + 1] = t->slot[i].y;
            out[3 * c + 2] = t->slot[i].z;
            ++c;
        }
    return c;
}

/* Map keys (Sec. III-C): v = floor(x / r_l).  Reading: the fine key
 * u = floor(fl32(m * fl32(1/r))) is computed once and the level-l key is
 * floor(u / 2^l) in integers, the same identity used for scan points.
 * Level l stores B_l plus the dilation V_add = {v - j, j in {0,1}^3} of every
 * occupied voxel (Sec. III-C, last paragraph).  Reading: level 0 is dilated
 * as well unless ORC_LEAF_UNDILATED is set. */
int orc_maps_build(const float* xyz, int64_t n, float r_f, int levels, uint32_t flags,
                   orc_maps** out)
{
    *out = NULL;
    if (!(r_f > 0.0f) || levels < 1 || levels > ORC_MAX_LEVELS || n < 0) return ORC_EINVAL;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (!isfinite(xyz[i])) return ORC_EINVAL;
    orc_maps* m = (orc_maps*)calloc(1, sizeof(orc_maps));
    if (!m) return ORC_ENOMEM;
    m->levels = levels;
    m->r = (double)r_f;
    m->flags = flags;
    for (int i = 0; i < 3; ++i) { m->lo[i] = INFINITY; m->hi[i] = -INFINITY; }
    for (int64_t p = 0; p < n; ++p)
        for (int i = 0; i < 3; ++i) {
            double v = xyz[3 * p + i];
            if (v < m->lo[i]) m->lo[i] = v;
            if (v > m->hi[i]) m->hi[i] = v;
        }
    if (n == 0) for (int i = 0; i < 3; ++i) { m->lo[i] = 0.0; m->hi[i] = 0.0; }

    const float rho = (float)(1.0 / (double)r_f);
    const int32_t KMAX = (1 << 20) - 4;
    orc_table b0;
    if (table_init(&b0, 1023)) { free(m); return ORC_ENOMEM; }
    int rc = ORC_OK;
    for (int64_t p = 0; p < n && rc == ORC_OK; ++p) {
        int32_t u[3];
        for (int i = 0; i < 3; ++i) {
            float q = xyz[3 * p + i] * rho;
            float f = floorf(q);
            if (!(f >= -(float)KMAX && f <= (float)KMAX)) { rc = ORC_EKEYRANGE; break; }
            u[i] = (int32_t)f;
        }
        if (rc == ORC_OK) rc = set_add(&b0, u[0], u[1], u[2]);
    }
    if (rc != ORC_OK) { free(b0.slot); free(m); return rc; }
    int64_t nb0 = b0.count;
    int32_t* k0 = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(nb0 > 0 ? nb0 : 1));
    if (!k0) { free(b0.slot); free(m); return ORC_ENOMEM; }
    set_keys(&b0, k0);
    free(b0.slot);

    /* exact-bound mode: a wider dilation at every level above the leaves */
    const int ee = (flags & ORC_EXACT_BOUND) ? ORC_EXACT_E(flags) : 0;
    if ((flags & ORC_EXACT_BOUND) && ee < 1) { free(k0); free(m); return ORC_EINVAL; }
    for (int l = 0; l < levels && rc == ORC_OK; ++l) {
        int dilate = !(l == 0 && (flags & ORC_LEAF_UNDILATED));
        const int jlo = l > 0 ? -ee : 0, jhi = l > 0 ? 1 + ee : 1;
        orc_table d;
        if (table_init(&d, 1023)) { rc = ORC_ENOMEM; break; }
        for (int64_t i = 0; i < nb0 && rc == ORC_OK; ++i) {
            int32_t vx = (int32_t)floordiv_pow2(k0[3 * i], l);
            int32_t vy = (int32_t)floordiv_pow2(k0[3 * i + 1], l);
            int32_t vz = (int32_t)floordiv_pow2(k0[3 * i + 2], l);
            if (!dilate) { rc = set_add(&d, vx, vy, vz); continue; }
            for (int jx = jlo; jx <= jhi && rc == ORC_OK; ++jx)
                for (int jy = jlo; jy <= jhi && rc == ORC_OK; ++jy)
                    for (int jz = jlo; jz <= jhi && rc == ORC_OK; ++jz)
                        rc = set_add(&d, vx - jx, vy - jy, vz - jz);
        }
        if (rc != ORC_OK) { free(d.slot); break; }
        int64_t nd = d.count;
        int32_t* kd = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)(nd > 0 ? nd : 1));
        if (!kd) { free(d.slot); rc = ORC_ENOMEM; break; }
        set_keys(&d, kd);
        free(d.slot);
        rc = table_from_keys(&m->lv[l], kd, nd);
        free(kd);
    }
    free(k0);
    if (rc != ORC_OK) { orc_maps_free(m); return rc; }
    *out = m;
    return ORC_OK;
}

/* Exact-bound mode.  A node at level l with rotation R_p (segment-centre
 * angles) and any leaf below it with rotation R_d: along the chain of
 * ancestors each child's angle lies within half a parent segment of the
 * parent's (centre reading; a whole segment with the lower-edge reading), so
 * per axis |angle_d - angle_p| <= sum_{k=1..l} delta'_k / 2 and the rotation
 * between them is at most the sum over the three axes, theta_l (the angle of
 * R_p^T R_d is bounded by the sum of the axis angles).  A scan point s then
 * moves by at most theta_l |s| <= theta_l d_max in metres (d_max: the larger of
 * the grid's and the scan's largest norm), theta_l d_max / r fine voxels;
 * the floors and the FP32 rounding of the keys add less than 2.  With the
 * translational offset t in [0, 2^l) of the leaf, the parent's level-l key is
 * the leaf's minus j with j in [-e, 1 + e] per axis, e = ceil((theta_l d_max / r
 * + 2) / 2^l): the dilation {v - j} then keeps every leaf hit a parent hit. */
int orc_exact_dilation(const orc_grid* g, double scan_norm_max)
{
    const double dmax = scan_norm_max > g->d_max ? scan_norm_max : g->d_max;
    if (g->flags & ORC_CHILD_LITERAL) return -1;
    const double half = (g->flags & ORC_ANGLE_LOWER_EDGE) ? 1.0 : 0.5;
    int e = 0;
    double sum[3] = {0.0, 0.0, 0.0};
    for (int l = 1; l < g->levels; ++l) {
        double theta = 0.0;
        for (int i = 0; i < 3; ++i) {
            /* a single segment at both levels: the child is the parent's angle */
            if (!(g->N[l][i] == 1 && g->N[l - 1][i] == 1)) sum[i] += half * g->dprime[l][i];
            theta += sum[i];
        }
        const double E = theta * dmax / g->r + 2.0;
        const int el = (int)ceil(E / ldexp(1.0, l));
        if (el > e) e = el;
    }
    return e;
}

void orc_maps_free(orc_maps* m)
{
    if (!m) return;
    for (int l = 0; l < ORC_MAX_LEVELS; ++l) free(m->lv[l].slot);
    free(m);
}

int orc_maps_levels(const orc_maps* m) { return m->levels; }
int64_t orc_maps_count(const orc_maps* m, int l) { return m->lv[l].count; }
int64_t orc_maps_table_size(const orc_maps* m, int l) { return m->lv[l].T; }
int64_t orc_maps_collisions(const orc_maps* m, int l) { return m->lv[l].collisions; }

int64_t orc_maps_keys(const orc_maps* m, int l, int32_t* out, int64_t cap)
{
    if (cap < m->lv[l].count) return -1;
    return set_keys(&m->lv[l], out);
}

int orc_maps_contains(const orc_maps* m, int l, int32_t x, int32_t y, int32_t z)
{
    return table_contains(&m->lv[l], x, y, z);
}

void orc_maps_bbox(const orc_maps* m, double lo[3], double hi[3])
{
    for (int i = 0; i < 3; ++i) { lo[i] = m->lo[i]; hi[i] = m->hi[i]; }
}

/* ======================================================================== */
/* Score: Sec. III-C Eq. (11)                                                */
/* ======================================================================== */

/* Fine key of point s under the scaled matrix A: u_i = floor(q_i) with
 * q_i = ((A_i0 s_x + A_i1 s_y) + A_i2 s_z), every product and sum rounded to
 * FP32 on its own (no FMA). */
static void fine_key(const float A[9], const float* s, int64_t u[3])
{
    for (int i = 0; i < 3; ++i) {
        float p0 = A[3 * i] * s[0];
        float p1 = A[3 * i + 1] * s[1];
        float p2 = A[3 * i + 2] * s[2];
        float q = (p0 + p1) + p2;
        u[i] = (int64_t)floorf(q);
    }
}

/* score(c) = sum_k H^{c_l}(T_{x_c} s_k), Eq. (11).  x_c translates by c * r_l;
 * reading: the translation is applied in the integer key domain, so the key
 * at level l is floor((u + c * 2^l) / 2^l) with u the fine key. */
int32_t orc_score(const orc_maps* m, const orc_grid* g, const float* scan, int64_t k,
                  const int32_t c[7])
{
    int l = c[6];
    float A[9];
    orc_rotation(g, l, c[3], c[4], c[5], A);
    int64_t T[3] = {(int64_t)c[0] * ((int64_t)1 << l), (int64_t)c[1] * ((int64_t)1 << l),
                    (int64_t)c[2] * ((int64_t)1 << l)};
    int32_t score = 0;
    for (int64_t p = 0; p < k; ++p) {
        int64_t u[3];
        fine_key(A, scan + 3 * p, u);
        int64_t vx = floordiv_pow2(u[0] + T[0], l);
        int64_t vy = floordiv_pow2(u[1] + T[1], l);
        int64_t vz = floordiv_pow2(u[2] + T[2], l);
        if (vx < INT32_MIN || vx > INT32_MAX || vy < INT32_MIN || vy > INT32_MAX ||
            vz < INT32_MIN || vz > INT32_MAX)
            continue;
        score += table_contains(&m->lv[l], (int32_t)vx, (int32_t)vy, (int32_t)vz);
    }
    return score;
}

static int node_valid(const orc_grid* g, const int32_t c[7])
{
    int l = c[6];
    if (l < 0 || l >= g->levels) return 0;
    for (int i = 0; i < 3; ++i) {
        if (c[3 + i] < 0 || c[3 + i] >= g->N[l][i]) return 0;
        int64_t t = (int64_t)c[i] * ((int64_t)1 << l);
        if (t < -((int64_t)1 << 20) || t > ((int64_t)1 << 20)) return 0;
    }
    return 1;
}

int orc_score_nodes(const orc_maps* m, const orc_grid* g, const float* scan, int64_t k,
                    const int32_t* nodes, int64_t n, int32_t* scores)
{
    for (int64_t i = 0; i < n; ++i)
        if (!node_valid(g, nodes + 7 * i)) return ORC_EINVAL;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) scores[i] = orc_score(m, g, scan, k, nodes + 7 * i);
    return ORC_OK;
}

/* Threads of the OpenMP build (liborc_mt.so); the plain build has one and
 * returns 1. */
int orc_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ======================================================================== */
/* Best-first batched BnB: Sec. III-E, Algorithm 2                           */
/* ======================================================================== */

typedef struct { int32_t c[7]; } node7;

typedef struct {
    node7* v;
    int64_t n, cap;
} nodevec;

static int vec_push(nodevec* a, const int32_t c[7])
{
    if (a->n == a->cap) {
        int64_t nc = a->cap ? 2 * a->cap : 16;
        node7* nv = (node7*)realloc(a->v, sizeof(node7) * (size_t)nc);
        if (!nv) return ORC_ENOMEM;
        a->v = nv;
        a->cap = nc;
    }
    memcpy(a->v[a->n].c, c, sizeof(int32_t) * 7);
    a->n++;
    return ORC_OK;
}

/* lexicographic order on (c_x, c_y, c_z, c_alpha, c_beta, c_gamma) */
static int lex_less(const int32_t* a, const int32_t* b)
{
    for (int i = 0; i < 6; ++i) {
        if (a[i] < b[i]) return 1;
        if (a[i] > b[i]) return 0;
    }
    return 0;
}

/* Scores of a list of nodes (Eq. (11)) into out[].  The scores are
 * independent of one another: built with OpenMP (liborc_mt.so, the CPU
 * multi-thread rows of Table I) they are computed in parallel; the callers
 * consume them in list order either way, so the search is the same. */
static void score_list(const orc_maps* m, const orc_grid* g, const float* scan, int64_t k, const node7* v,
                       int64_t n, int32_t* out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) out[i] = orc_score(m, g, scan, k, v[i].c);
}

/* Every child (Eq. (13)) of the parents P in parent order, with the index of
 * its parent, and their scores. */
typedef struct {
    nodevec kids;
    int64_t* parent;
    int32_t* score;
    int64_t cap;
} childset;

static int children_scored(const orc_maps* m, const orc_grid* g, const float* scan, int64_t k, const nodevec* P,
                           childset* C)
{
    C->kids.n = 0;
    int64_t total = 0;
    for (int64_t i = 0; i < P->n; ++i) total += orc_num_children(g, P->v[i].c);
    if (C->kids.cap < total) {
        node7* nv = (node7*)realloc(C->kids.v, sizeof(node7) * (size_t)total);
        if (!nv) return ORC_ENOMEM;
        C->kids.v = nv;
        C->kids.cap = total;
    }
    if (C->cap < total) {
        int64_t* np = (int64_t*)realloc(C->parent, sizeof(int64_t) * (size_t)total);
        if (!np) return ORC_ENOMEM;
        C->parent = np;
        int32_t* ns = (int32_t*)realloc(C->score, sizeof(int32_t) * (size_t)total);
        if (!ns) return ORC_ENOMEM;
        C->score = ns;
        C->cap = total;
    }
    for (int64_t i = 0; i < P->n; ++i) {
        const int64_t nk = orc_num_children(g, P->v[i].c);
        orc_children(g, P->v[i].c, &C->kids.v[C->kids.n].c[0], nk);
        for (int64_t j = 0; j < nk; ++j) C->parent[C->kids.n + j] = i;
        C->kids.n += nk;
    }
    score_list(m, g, scan, k, C->kids.v, C->kids.n, C->score);
    return ORC_OK;
}

static void childset_free(childset* C)
{
    free(C->kids.v);
    free(C->parent);
    free(C->score);
}

/* The frontier F: nodes bucketed by integer score (the queue "sorted by
 * score" of Algorithm 2). */
typedef struct {
    nodevec* b;     /* b[s], s = 0..K */
    int64_t K;
    int64_t size;
    int64_t top;    /* every bucket above top is empty */
} frontier;

static int fr_push(frontier* f, int32_t s, const int32_t c[7])
{
    int rc = vec_push(&f->b[s], c);
    if (rc) return rc;
    f->size++;
    if (s > f->top) f->top = s;
    return ORC_OK;
}

static void fr_clear(frontier* f)
{
    for (int64_t s = 0; s <= f->K; ++s) f->b[s].n = 0;
    f->size = 0;
    f->top = -1;
}

/* Canonical iteration (the paper leaves ties, the end-of-queue flush and the
 * pop order within a batch open; the reading fixed here is reproduced exactly
 * by the GPU path):
 *
 *   best = ceil(theta K) - 1, match unset
 *   F = { c in C_lmax : score(c) > best }
 *   repeat:
 *     P = {}
 *     while F is not empty and children(P) < b:
 *       s = highest score in F, B = all nodes of F with score s (removed)
 *       if s <= best: clear F, stop popping
 *       if B holds a leaf: best = s, match = lexmin leaf of B, clear F, stop popping
 *       P = P + B
 *     if P is empty: done
 *     score every child of P (Eq. 13); keep those with score > best in F
 *
 * Only popping a leaf changes best, so the order in which a batch's children
 * are scored and inserted cannot change the outcome. */
/* Sec. IV-A checks how often the approximate rotational bound fails: a
 * child scoring above its parent (whose score was to bound it), and by how
 * much relative to the child's score.  Counted over every child scored while
 * branching. */
static void bound_check(orc_result* res, int32_t parent, int32_t child)
{
    res->children_scored++;
    if (child > parent) {
        res->bound_violations++;
        res->bound_excess += (double)(child - parent) / (double)child;
    }
}

/* Depth-first batched iteration (Table I's DFS search strategy; the paper
 * gives no batched form of it, so this reading fixes one): F is kept per
 * level, and nodes are taken deepest level first and, within a level,
 * highest score first, in whole (level, score) buckets.
 *
 *   best = ceil(theta K) - 1, match unset, F = { c in C_lmax : score(c) > best }
 *   repeat:
 *     if F holds leaves: s = their highest score (> best), best = s,
 *       match = lexmin leaf of score s; drop every node of F with score <= best
 *       (every leaf among them)
 *     P = {}
 *     for l = 1 .. l_max, and within l for s from the highest score down,
 *       while children(P) < b: P = P + the nodes of F at (l, s) (removed)
 *     if P is empty: done
 *     score every child of P (Eq. 13); keep those with score > best in F
 *
 * best changes only at the start of an iteration, so the order in which a
 * batch's children are scored and inserted cannot change the outcome.  Every
 * node kept scores above best, so with an exact bound the result's score is
 * the exhaustive optimum, as for the best-first order; the match may differ
 * among equal scores. */
static int dfs_search(const orc_maps* m, const orc_grid* g, const float* scan, int64_t k, int64_t batch,
                      int64_t max_frontier, frontier* FL, int32_t* best_io, int32_t match[7], int* found,
                      orc_result* res)
{
    const int L = g->levels;
    int32_t best = *best_io;
    nodevec P = {0};
    childset C = {{0}, 0, 0, 0};
    int32_t* Ps = NULL;   /* score of each popped parent */
    int64_t Ps_cap = 0;
    int rc = ORC_OK;
    for (;;) {
        int64_t size = 0;
        for (int l = 0; l < L; ++l) size += FL[l].size;
        if (size > res->peak_frontier) res->peak_frontier = size;
        if (max_frontier > 0 && size > max_frontier) { rc = ORC_ENOMEM; break; }
        /* leaves first: the best of them sets best and the match */
        if (FL[0].size > 0) {
            while (FL[0].top >= 0 && FL[0].b[FL[0].top].n == 0) FL[0].top--;
            const int32_t s = (int32_t)FL[0].top;
            const nodevec* B = &FL[0].b[s];
            int32_t lm[7];
            for (int64_t i = 0; i < B->n; ++i)
                if (i == 0 || lex_less(B->v[i].c, lm)) memcpy(lm, B->v[i].c, sizeof(lm));
            best = s;
            memcpy(match, lm, sizeof(lm));
            *found = 1;
            for (int l = 0; l < L; ++l)
                for (int64_t t = 0; t <= best && t <= FL[l].K; ++t) {
                    FL[l].size -= FL[l].b[t].n;
                    FL[l].b[t].n = 0;
                }
        }
        /* parents: deepest level first, highest score first */
        P.n = 0;
        int64_t nchild = 0;
        for (int l = 1; l < L && nchild < batch && !rc; ++l) {
            frontier* F = &FL[l];
            for (int64_t s = F->top; s > best && nchild < batch && !rc; --s) {
                nodevec* B = &F->b[s];
                if (B->n == 0) continue;
                if (Ps_cap < P.n + B->n) {
                    int64_t nc = 2 * (P.n + B->n);
                    int32_t* np = (int32_t*)realloc(Ps, sizeof(int32_t) * (size_t)nc);
                    if (!np) { rc = ORC_ENOMEM; break; }
                    Ps = np;
                    Ps_cap = nc;
                }
                for (int64_t i = 0; i < B->n && !rc; ++i) {
                    Ps[P.n] = (int32_t)s;
                    rc = vec_push(&P, B->v[i].c);
                    nchild += orc_num_children(g, B->v[i].c);
                }
                F->size -= B->n;
                B->n = 0;
            }
        }
        if (rc || P.n == 0) break;
        res->iterations++;
        res->parents_branched += P.n;
        rc = children_scored(m, g, scan, k, &P, &C);
        for (int64_t j = 0; j < C.kids.n && !rc; ++j) {
            const int32_t s = C.score[j];
            res->nodes_scored++;
            bound_check(res, Ps[C.parent[j]], s);
            if (s > best) rc = fr_push(&FL[C.kids.v[j].c[6]], s, C.kids.v[j].c);
        }
    }
    free(P.v);
    free(Ps);
    childset_free(&C);
    *best_io = best;
    return rc;
}

int orc_localize(const orc_maps* m, const float* scan, int64_t k, const orc_ranges* rg,
                 double score_frac, int64_t batch, double d_max, uint32_t flags,
                 int64_t max_frontier, orc_result* res)
{
    double t0 = now_ms();
    memset(res, 0, sizeof(*res));
    res->num_points = (int32_t)k;
    if (k < 0 || batch < 1 || !(score_frac > 0.0 && score_frac <= 1.0)) return res->status = ORC_EINVAL;
    for (int64_t i = 0; i < 3 * k; ++i)
        if (!isfinite(scan[i]) || fabs((double)scan[i]) > ldexp(m->r, 18)) return res->status = ORC_EINVAL;
    if (flags & ORC_PRUNE_GE) return res->status = ORC_EINVAL;
    if (k == 0) { res->status = ORC_NOT_FOUND; return ORC_NOT_FOUND; }

    double dm = d_max > 0.0 ? d_max : orc_scan_dmax(scan, k);
    orc_grid g;
    int rc = orc_grid_build(m->r, m->levels, dm, rg, flags, &g);
    if (rc) return res->status = rc;
    if (m->flags & ORC_EXACT_BOUND) {   /* the maps' dilation must cover this grid */
        const int need = orc_exact_dilation(&g, orc_scan_dmax(scan, k));
        if (need < 0 || need > ORC_EXACT_E(m->flags)) return res->status = ORC_EINVAL;
    }

    const int lmax = m->levels - 1;
    int32_t best = (int32_t)ceil(score_frac * (double)k) - 1;
    int32_t match[7] = {0};
    int found = 0;

    const int dfs = (flags & ORC_SEARCH_DFS) != 0;
    const int nfr = dfs ? m->levels : 1;   /* depth-first: one frontier per level */
    frontier* FL = (frontier*)calloc((size_t)nfr, sizeof(frontier));
    if (!FL) return res->status = ORC_ENOMEM;
    for (int l = 0; l < nfr; ++l) {
        FL[l].K = k;
        FL[l].top = -1;
        FL[l].b = (nodevec*)calloc((size_t)k + 1, sizeof(nodevec));
        if (!FL[l].b) {
            for (int j = 0; j < l; ++j) free(FL[j].b);
            free(FL);
            return res->status = ORC_ENOMEM;
        }
    }
    frontier F = FL[0];   /* best-first: the one frontier */
    nodevec P = {0};
    childset C = {{0}, 0, 0, 0};
    int32_t* Ps = NULL;   /* score of each popped parent (the bucket it came from) */
    int64_t Ps_cap = 0;

    /* initial set C_lmax (Sec. III-D): all translations of Eq. (3)-(5) times
     * all rotations at l_max */
    int32_t c[7];
    c[6] = lmax;
    nodevec init = {0};
    for (int64_t x = g.wmin[0]; x <= g.wmax[0] && !rc; ++x)
        for (int64_t y = g.wmin[1]; y <= g.wmax[1] && !rc; ++y)
            for (int64_t z = g.wmin[2]; z <= g.wmax[2] && !rc; ++z)
                for (int64_t ia = 0; ia < g.N[lmax][0] && !rc; ++ia)
                    for (int64_t ib = 0; ib < g.N[lmax][1] && !rc; ++ib)
                        for (int64_t ig = 0; ig < g.N[lmax][2] && !rc; ++ig) {
                            c[0] = (int32_t)x; c[1] = (int32_t)y; c[2] = (int32_t)z;
                            c[3] = (int32_t)ia; c[4] = (int32_t)ib; c[5] = (int32_t)ig;
                            rc = vec_push(&init, c);
                        }
    int32_t* init_score = rc ? NULL : (int32_t*)malloc(sizeof(int32_t) * (size_t)(init.n > 0 ? init.n : 1));
    if (!rc && !init_score) rc = ORC_ENOMEM;
    if (!rc) score_list(m, &g, scan, k, init.v, init.n, init_score);
    for (int64_t i = 0; i < init.n && !rc; ++i) {
        res->nodes_scored++;
        if (init_score[i] > best) rc = fr_push(dfs ? &FL[lmax] : &F, init_score[i], init.v[i].c);
    }
    free(init.v);
    free(init_score);
    if (F.size > res->peak_frontier) res->peak_frontier = F.size;

    if (dfs && !rc) rc = dfs_search(m, &g, scan, k, batch, max_frontier, FL, &best, match, &found, res);
    while (!rc && !dfs) {
        if (max_frontier > 0 && F.size > max_frontier) { rc = ORC_ENOMEM; break; }
        P.n = 0;
        int64_t nchild = 0;
        while (F.size > 0 && nchild < batch) {
            while (F.top >= 0 && F.b[F.top].n == 0) F.top--;
            int32_t s = (int32_t)F.top;
            if (s <= best) { fr_clear(&F); break; }
            nodevec* B = &F.b[s];
            int has_leaf = 0;
            int32_t lm[7];
            for (int64_t i = 0; i < B->n; ++i)
                if (B->v[i].c[6] == 0) {
                    if (!has_leaf || lex_less(B->v[i].c, lm)) memcpy(lm, B->v[i].c, sizeof(lm));
                    has_leaf = 1;
                }
            if (has_leaf) {
                best = s;
                memcpy(match, lm, sizeof(match));
                found = 1;
                fr_clear(&F);
                break;
            }
            if (Ps_cap < P.n + B->n) {
                int64_t nc = 2 * (P.n + B->n);
                int32_t* np = (int32_t*)realloc(Ps, sizeof(int32_t) * (size_t)nc);
                if (!np) { rc = ORC_ENOMEM; break; }
                Ps = np;
                Ps_cap = nc;
            }
            for (int64_t i = 0; i < B->n && !rc; ++i) {
                Ps[P.n] = s;
                rc = vec_push(&P, B->v[i].c);
                nchild += orc_num_children(&g, B->v[i].c);
            }
            F.size -= B->n;
            B->n = 0;
        }
        if (rc || P.n == 0) break;
        res->iterations++;
        res->parents_branched += P.n;
        rc = children_scored(m, &g, scan, k, &P, &C);
        for (int64_t j = 0; j < C.kids.n && !rc; ++j) {
            const int32_t s = C.score[j];
            res->nodes_scored++;
            bound_check(res, Ps[C.parent[j]], s);
            if (s > best) rc = fr_push(&F, s, C.kids.v[j].c);
        }
        if (F.size > res->peak_frontier) res->peak_frontier = F.size;
    }

    if (!dfs) FL[0] = F;
    for (int l = 0; l < nfr; ++l) {
        for (int64_t s = 0; s <= k; ++s) free(FL[l].b[s].v);
        free(FL[l].b);
    }
    free(FL);
    free(P.v);
    free(Ps);
    childset_free(&C);
    res->probes = res->nodes_scored * k;
    res->ms_total = now_ms() - t0;
    if (rc) return res->status = rc;
    res->best_score = best;
    if (found) {
        memcpy(res->node, match, sizeof(match));
        res->found = 1;
        for (int i = 0; i < 3; ++i) res->pose[i] = (double)match[i] * g.r;   /* x_c = r_l c, l = 0 */
        for (int i = 0; i < 3; ++i) res->pose[3 + i] = orc_angle(&g, 0, i, match[3 + i]);
        res->status = ORC_OK;
    } else {
        res->status = ORC_NOT_FOUND;
    }
    return res->status;
}

/* ======================================================================== */
/* Exhaustive search: Eq. (1) over the leaf set of the grid                  */
/* ======================================================================== */

/* The leaves are every level-0 node below C_lmax: translations
 * [w_min 2^lmax, (w_max + 1) 2^lmax - 1] per axis, all level-0 rotations. */
int orc_brute_force(const orc_maps* m, const orc_grid* g, const float* scan, int64_t k,
                    int32_t* best_score, int32_t best_node[7])
{
    const int lmax = g->levels - 1;
    int64_t tlo[3], thi[3];
    for (int i = 0; i < 3; ++i) {
        tlo[i] = g->wmin[i] * ((int64_t)1 << lmax);
        thi[i] = (g->wmax[i] + 1) * ((int64_t)1 << lmax) - 1;
    }
    int64_t* u = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(k > 0 ? k : 1));
    if (!u) return ORC_ENOMEM;
    int32_t best = -1;
    int32_t bn[7] = {0};
    for (int64_t ia = 0; ia < g->N[0][0]; ++ia)
        for (int64_t ib = 0; ib < g->N[0][1]; ++ib)
            for (int64_t ig = 0; ig < g->N[0][2]; ++ig) {
                float A[9];
                orc_rotation(g, 0, ia, ib, ig, A);
                for (int64_t p = 0; p < k; ++p) fine_key(A, scan + 3 * p, u + 3 * p);
                for (int64_t x = tlo[0]; x <= thi[0]; ++x)
                    for (int64_t y = tlo[1]; y <= thi[1]; ++y)
                        for (int64_t z = tlo[2]; z <= thi[2]; ++z) {
                            int32_t s = 0;
                            for (int64_t p = 0; p < k; ++p)
                                s += table_contains(&m->lv[0], (int32_t)(u[3 * p] + x),
                                                    (int32_t)(u[3 * p + 1] + y),
                                                    (int32_t)(u[3 * p + 2] + z));
                            int32_t cand[7] = {(int32_t)x, (int32_t)y, (int32_t)z, (int32_t)ia,
                                               (int32_t)ib, (int32_t)ig, 0};
                            if (s > best || (s == best && lex_less(cand, bn))) {
                                best = s;
                                memcpy(bn, cand, sizeof(bn));
                            }
                        }
            }
    free(u);
    *best_score = best;
    memcpy(best_node, bn, sizeof(bn));
    return ORC_OK;
}
