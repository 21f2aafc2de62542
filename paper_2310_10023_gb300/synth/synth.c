/*
 * synth.c -- seeded synthetic maps and LiDAR scans for 3D-BBS workloads.
 *
 * This module only produces inputs: scenes of axis-aligned boxes, surface
 * samples of them (the map point cloud), and scans ray-cast from a planted
 * sensor pose.  It contains none of the localization method's arithmetic
 * (no voxel keys, hash maps, pose grids or scores) and is shared by the
 * oracle tests and the GPU tests/benchmark as the single source of inputs.
 *
 * Random numbers: MT19937-64 (Matsumoto and Nishimura's 64-bit Mersenne
 * Twister, written out from its published recurrence), 53-bit uniforms
 * u = (x >> 11) * 2^-53, and Box-Muller normals, so the data is reproducible
 * from the seed alone.
 *
 * Sensor pose convention: world point = R s + t with
 * R = Rz(yaw) Ry(pitch) Rx(roll); a scan holds sensor-frame points s.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#if defined(__GNUC__)
#define SYN_API __attribute__((visibility("default")))
#else
#define SYN_API
#endif

/* ------------------------------------------------------------------------ */
/* MT19937-64                                                                */
/* ------------------------------------------------------------------------ */
#define MT_N 312
#define MT_M 156
typedef struct {
    uint64_t mt[MT_N];
    int i;
} syn_rng;

static void rng_seed(syn_rng* r, uint64_t seed)
{
    r->mt[0] = seed;
    for (int i = 1; i < MT_N; ++i)
        r->mt[i] = 6364136223846793005ull * (r->mt[i - 1] ^ (r->mt[i - 1] >> 62)) + (uint64_t)i;
    r->i = MT_N;
}

static uint64_t rng_next(syn_rng* r)
{
    const uint64_t UPPER = 0xFFFFFFFF80000000ull, LOWER = 0x7FFFFFFFull;
    const uint64_t MATRIX_A = 0xB5026F5AA96619E9ull;
    if (r->i >= MT_N) {
        for (int k = 0; k < MT_N; ++k) {
            uint64_t x = (r->mt[k] & UPPER) | (r->mt[(k + 1) % MT_N] & LOWER);
            uint64_t xa = x >> 1;
            if (x & 1ull) xa ^= MATRIX_A;
            r->mt[k] = r->mt[(k + MT_M) % MT_N] ^ xa;
        }
        r->i = 0;
    }
    uint64_t x = r->mt[r->i++];
    x ^= (x >> 29) & 0x5555555555555555ull;
    x ^= (x << 17) & 0x71D67FFFEDA60000ull;
    x ^= (x << 37) & 0xFFF7EEE000000000ull;
    x ^= x >> 43;
    return x;
}

static double rng_u(syn_rng* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static double rng_range(syn_rng* r, double a, double b) { return a + (b - a) * rng_u(r); }
static double rng_normal(syn_rng* r)
{
    double u1 = 1.0 - rng_u(r); /* (0, 1] */
    double u2 = rng_u(r);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* exposed for the generator's own reproducibility test */
SYN_API void syn_mt64(uint64_t seed, int64_t n, uint64_t* out)
{
    syn_rng r;
    rng_seed(&r, seed);
    for (int64_t i = 0; i < n; ++i) out[i] = rng_next(&r);
}

/* ------------------------------------------------------------------------ */
/* scenes of boxes                                                           */
/* ------------------------------------------------------------------------ */
enum { F_NX = 1, F_PX = 2, F_NY = 4, F_PY = 8, F_NZ = 16, F_PZ = 32, F_ALL_BUT_BOTTOM = 47 };

typedef struct {
    double lo[3], hi[3];
    unsigned faces; /* which faces are sampled into the map */
} box;

typedef struct {
    box* b;
    int n, cap;
    double lo[3], hi[3];     /* scene extent used for planting poses   */
} scene;

static void add_box(scene* s, double x0, double y0, double z0, double x1, double y1, double z1,
                    unsigned faces)
{
    if (s->n == s->cap) {
        s->cap = s->cap ? 2 * s->cap : 64;
        s->b = (box*)realloc(s->b, sizeof(box) * (size_t)s->cap);
    }
    box* b = &s->b[s->n++];
    b->lo[0] = x0; b->lo[1] = y0; b->lo[2] = z0;
    b->hi[0] = x1; b->hi[1] = y1; b->hi[2] = z1;
    b->faces = faces;
}

/* cfg 1: 20 x 20 x 5 m room, floor and 4 walls, 10 random boxes */
static void scene_room(scene* s)
{
    syn_rng r;
    rng_seed(&r, 1001);
    add_box(s, 0, 0, -0.2, 20, 20, 0, F_PZ);
    add_box(s, -0.2, 0, 0, 0, 20, 5, F_PX);
    add_box(s, 20, 0, 0, 20.2, 20, 5, F_NX);
    add_box(s, 0, -0.2, 0, 20, 0, 5, F_PY);
    add_box(s, 0, 20, 0, 20, 20.2, 5, F_NY);
    for (int i = 0; i < 10; ++i) {
        double sx = rng_range(&r, 0.5, 3.0), sy = rng_range(&r, 0.5, 3.0), sz = rng_range(&r, 0.5, 3.0);
        double x = rng_range(&r, 0.5, 19.5 - sx), y = rng_range(&r, 0.5, 19.5 - sy);
        add_box(s, x, y, 0, x + sx, y + sy, sz, F_ALL_BUT_BOTTOM);
    }
    s->lo[0] = 0; s->lo[1] = 0; s->lo[2] = 0;
    s->hi[0] = 20; s->hi[1] = 20; s->hi[2] = 5;
}

/* a wall along x (constant y band) from x0 to x1 with one door gap */
static void wall_x(scene* s, syn_rng* r, double x0, double x1, double y, double h)
{
    double t = 0.1, dw = 1.5, dh = 2.2;
    double d = rng_range(r, x0 + 1.0, x1 - 1.0 - dw);
    add_box(s, x0, y - t, 0, d, y + t, h, F_NY | F_PY | F_NX | F_PX);
    add_box(s, d + dw, y - t, 0, x1, y + t, h, F_NY | F_PY | F_NX | F_PX);
    add_box(s, d, y - t, dh, d + dw, y + t, h, F_NY | F_PY | F_NZ);
}

static void wall_y(scene* s, syn_rng* r, double y0, double y1, double x, double h)
{
    double t = 0.1, dw = 1.5, dh = 2.2;
    double d = rng_range(r, y0 + 1.0, y1 - 1.0 - dw);
    add_box(s, x - t, y0, 0, x + t, d, h, F_NX | F_PX | F_NY | F_PY);
    add_box(s, x - t, d + dw, 0, x + t, y1, h, F_NX | F_PX | F_NY | F_PY);
    add_box(s, x - t, d, dh, x + t, d + dw, h, F_NX | F_PX | F_NZ);
}

/* cfg 2: 100 x 60 x 10 m multi-room floor: floor, ceiling, outer walls, a
 * 5 x 4 room grid of inner walls with door gaps, 150 clutter boxes */
static void scene_indoor(scene* s)
{
    syn_rng r;
    rng_seed(&r, 1002);
    const double X = 100, Y = 60, H = 10;
    add_box(s, 0, 0, -0.2, X, Y, 0, F_PZ);
    add_box(s, 0, 0, H, X, Y, H + 0.2, F_NZ);
    add_box(s, -0.2, 0, 0, 0, Y, H, F_PX);
    add_box(s, X, 0, 0, X + 0.2, Y, H, F_NX);
    add_box(s, 0, -0.2, 0, X, 0, H, F_PY);
    add_box(s, 0, Y, 0, X, Y + 0.2, H, F_NY);
    for (int i = 1; i < 5; ++i)          /* walls at x = 20, 40, 60, 80 */
        for (int j = 0; j < 4; ++j) wall_y(s, &r, 15.0 * j, 15.0 * (j + 1), 20.0 * i, H);
    for (int j = 1; j < 4; ++j)          /* walls at y = 15, 30, 45 */
        for (int i = 0; i < 5; ++i) wall_x(s, &r, 20.0 * i, 20.0 * (i + 1), 15.0 * j, H);
    for (int i = 0; i < 150; ++i) {
        double sx = rng_range(&r, 0.3, 2.5), sy = rng_range(&r, 0.3, 2.5), sz = rng_range(&r, 0.5, 2.5);
        double x = rng_range(&r, 0.5, X - 0.5 - sx), y = rng_range(&r, 0.5, Y - 0.5 - sy);
        add_box(s, x, y, 0, x + sx, y + sy, sz, F_ALL_BUT_BOTTOM);
    }
    s->lo[0] = 0; s->lo[1] = 0; s->lo[2] = 0;
    s->hi[0] = X; s->hi[1] = Y; s->hi[2] = H;
}

/* cfg 3: 800 x 800 x 40 m city: ground, 10 x 10 blocks of 60 m with 20 m
 * streets, up to 4 buildings per block, street poles and tree clusters */
static void scene_city(scene* s)
{
    syn_rng r;
    rng_seed(&r, 1003);
    add_box(s, 0, 0, -0.5, 800, 800, 0, F_PZ);
    for (int bi = 0; bi < 10; ++bi)
        for (int bj = 0; bj < 10; ++bj) {
            double ox = 10 + 80.0 * bi, oy = 10 + 80.0 * bj;
            for (int q = 0; q < 4; ++q) {
                double qx = ox + 30.0 * (q & 1), qy = oy + 30.0 * (q >> 1);
                if (rng_u(&r) < 0.15) {   /* park: a tree cluster */
                    int nt = 3 + (int)(rng_u(&r) * 4);
                    for (int t = 0; t < nt; ++t) {
                        double tx = rng_range(&r, qx + 3, qx + 27), ty = rng_range(&r, qy + 3, qy + 27);
                        add_box(s, tx - 0.25, ty - 0.25, 0, tx + 0.25, ty + 0.25, 3, F_NX | F_PX | F_NY | F_PY);
                        add_box(s, tx - 1.5, ty - 1.5, 3, tx + 1.5, ty + 1.5, 6, F_ALL_BUT_BOTTOM | F_NZ);
                    }
                    continue;
                }
                double x0 = qx + rng_range(&r, 1, 5), y0 = qy + rng_range(&r, 1, 5);
                double x1 = qx + 30 - rng_range(&r, 1, 5), y1 = qy + 30 - rng_range(&r, 1, 5);
                double h = rng_range(&r, 6, 40);
                add_box(s, x0, y0, 0, x1, y1, h, F_ALL_BUT_BOTTOM);
            }
            /* poles every 20 m along the block's south and west edges */
            for (int p = 0; p < 3; ++p) {
                double px = ox + 10 + 20.0 * p, py = oy - 2.0;
                add_box(s, px - 0.15, py - 0.15, 0, px + 0.15, py + 0.15, 8, F_NX | F_PX | F_NY | F_PY | F_PZ);
                add_box(s, ox - 2.15, oy + 10 + 20.0 * p - 0.15, 0, ox - 1.85, oy + 10 + 20.0 * p + 0.15, 8,
                        F_NX | F_PX | F_NY | F_PY | F_PZ);
            }
        }
    s->lo[0] = 0; s->lo[1] = 0; s->lo[2] = 0;
    s->hi[0] = 800; s->hi[1] = 800; s->hi[2] = 40;
}

static int make_scene(int cfg, scene* s)
{
    memset(s, 0, sizeof(*s));
    switch (cfg) {
    case 1: scene_room(s); return 0;
    case 2: scene_indoor(s); return 0;
    case 3: scene_city(s); return 0;
    default: return -1;
    }
}

/* ------------------------------------------------------------------------ */
/* map point clouds: samples of the box faces                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    float* p;
    int64_t n, cap;
} cloud;

static void cloud_add(cloud* c, double x, double y, double z)
{
    if (c->n == c->cap) {
        c->cap = c->cap ? 2 * c->cap : 4096;
        c->p = (float*)realloc(c->p, sizeof(float) * 3 * (size_t)c->cap);
    }
    c->p[3 * c->n] = (float)x;
    c->p[3 * c->n + 1] = (float)y;
    c->p[3 * c->n + 2] = (float)z;
    c->n++;
}

/* face f of box b: fixed axis, fixed coordinate, the two in-plane axes */
static void face_geom(const box* b, int f, int* ax, double* at, int* u, int* v)
{
    *ax = f / 2;
    *at = (f & 1) ? b->hi[*ax] : b->lo[*ax];
    *u = (*ax + 1) % 3;
    *v = (*ax + 2) % 3;
}

/* lattice samples at multiples of h inside each sampled face */
static void sample_lattice(const scene* s, double h, cloud* c)
{
    for (int i = 0; i < s->n; ++i)
        for (int f = 0; f < 6; ++f) {
            if (!(s->b[i].faces & (1u << f))) continue;
            int ax, u, v;
            double at;
            face_geom(&s->b[i], f, &ax, &at, &u, &v);
            int64_t u0 = (int64_t)ceil(s->b[i].lo[u] / h - 1e-9), u1 = (int64_t)floor(s->b[i].hi[u] / h + 1e-9);
            int64_t v0 = (int64_t)ceil(s->b[i].lo[v] / h - 1e-9), v1 = (int64_t)floor(s->b[i].hi[v] / h + 1e-9);
            for (int64_t a = u0; a <= u1; ++a)
                for (int64_t b = v0; b <= v1; ++b) {
                    double p[3];
                    p[ax] = at;
                    p[u] = (double)a * h;
                    p[v] = (double)b * h;
                    cloud_add(c, p[0], p[1], p[2]);
                }
        }
}

/* n_total uniform samples spread over the sampled faces by area */
static void sample_random(const scene* s, int64_t n_total, uint64_t seed, cloud* c)
{
    syn_rng r;
    rng_seed(&r, seed);
    double area = 0;
    for (int i = 0; i < s->n; ++i)
        for (int f = 0; f < 6; ++f) {
            if (!(s->b[i].faces & (1u << f))) continue;
            int ax, u, v;
            double at;
            face_geom(&s->b[i], f, &ax, &at, &u, &v);
            area += (s->b[i].hi[u] - s->b[i].lo[u]) * (s->b[i].hi[v] - s->b[i].lo[v]);
        }
    for (int i = 0; i < s->n; ++i)
        for (int f = 0; f < 6; ++f) {
            if (!(s->b[i].faces & (1u << f))) continue;
            int ax, u, v;
            double at;
            face_geom(&s->b[i], f, &ax, &at, &u, &v);
            double fa = (s->b[i].hi[u] - s->b[i].lo[u]) * (s->b[i].hi[v] - s->b[i].lo[v]);
            int64_t m = (int64_t)floor((double)n_total * fa / area + 0.5);
            for (int64_t k = 0; k < m; ++k) {
                double p[3];
                p[ax] = at;
                p[u] = rng_range(&r, s->b[i].lo[u], s->b[i].hi[u]);
                p[v] = rng_range(&r, s->b[i].lo[v], s->b[i].hi[v]);
                cloud_add(c, p[0], p[1], p[2]);
            }
        }
}

/* ------------------------------------------------------------------------ */
/* ray casting                                                               */
/* ------------------------------------------------------------------------ */
static double ray_box(const double o[3], const double d[3], const box* b)
{
    double t0 = 0.0, t1 = INFINITY;
    for (int i = 0; i < 3; ++i) {
        if (fabs(d[i]) < 1e-15) {
            if (o[i] < b->lo[i] || o[i] > b->hi[i]) return INFINITY;
            continue;
        }
        double inv = 1.0 / d[i];
        double a = (b->lo[i] - o[i]) * inv, c = (b->hi[i] - o[i]) * inv;
        if (a > c) { double t = a; a = c; c = t; }
        if (a > t0) t0 = a;
        if (c < t1) t1 = c;
        if (t0 > t1) return INFINITY;
    }
    return t0 > 1e-6 ? t0 : INFINITY;
}

static void rot_zyx(double roll, double pitch, double yaw, double R[9])
{
    double ca = cos(roll), sa = sin(roll), cb = cos(pitch), sb = sin(pitch), cg = cos(yaw), sg = sin(yaw);
    R[0] = cg * cb; R[1] = cg * sb * sa - sg * ca; R[2] = cg * sb * ca + sg * sa;
    R[3] = sg * cb; R[4] = sg * sb * sa + cg * ca; R[5] = sg * sb * ca - cg * sa;
    R[6] = -sb;     R[7] = cb * sa;                R[8] = cb * ca;
}

static int inside_any(const scene* s, const double p[3], double margin)
{
    for (int i = 0; i < s->n; ++i) {
        const box* b = &s->b[i];
        if (p[0] > b->lo[0] - margin && p[0] < b->hi[0] + margin && p[1] > b->lo[1] - margin &&
            p[1] < b->hi[1] + margin && p[2] > b->lo[2] - margin && p[2] < b->hi[2] + margin)
            return 1;
    }
    return 0;
}

typedef struct {
    int beams;
    double vfov_deg;      /* beams spread evenly over [-vfov, +vfov]     */
    double hres_deg;
    double max_range;
} lidar;

/* sensor-frame hits of all rays from pose (t, R) */
static void cast_scan(const scene* s, const lidar* L, const double t[3], const double R[9], cloud* out)
{
    /* only boxes that can be within range */
    int* near = (int*)malloc(sizeof(int) * (size_t)(s->n > 0 ? s->n : 1));
    int nn = 0;
    for (int i = 0; i < s->n; ++i) {
        double d2 = 0;
        for (int k = 0; k < 3; ++k) {
            double e = 0;
            if (t[k] < s->b[i].lo[k]) e = s->b[i].lo[k] - t[k];
            else if (t[k] > s->b[i].hi[k]) e = t[k] - s->b[i].hi[k];
            d2 += e * e;
        }
        if (d2 <= L->max_range * L->max_range) near[nn++] = i;
    }
    int naz = (int)floor(360.0 / L->hres_deg + 0.5);
    for (int bi = 0; bi < L->beams; ++bi) {
        double el = L->beams > 1 ? (-L->vfov_deg + 2.0 * L->vfov_deg * bi / (L->beams - 1)) : 0.0;
        el *= 3.141592653589793 / 180.0;
        for (int a = 0; a < naz; ++a) {
            double az = (double)a * L->hres_deg * 3.141592653589793 / 180.0;
            double ds[3] = {cos(el) * cos(az), cos(el) * sin(az), sin(el)};
            double dw[3];
            for (int i = 0; i < 3; ++i) dw[i] = R[3 * i] * ds[0] + R[3 * i + 1] * ds[1] + R[3 * i + 2] * ds[2];
            double best = INFINITY;
            for (int j = 0; j < nn; ++j) {
                double h = ray_box(t, dw, &s->b[near[j]]);
                if (h < best) best = h;
            }
            if (best <= L->max_range) cloud_add(out, best * ds[0], best * ds[1], best * ds[2]);
        }
    }
    free(near);
}

/* voxel-grid filter (centroid per voxel), as used by the paper to reduce scans */
typedef struct {
    int64_t key[3];
    int64_t idx;
} vk;

static int vk_cmp(const void* a, const void* b)
{
    const vk* x = (const vk*)a;
    const vk* y = (const vk*)b;
    for (int i = 0; i < 3; ++i) {
        if (x->key[i] < y->key[i]) return -1;
        if (x->key[i] > y->key[i]) return 1;
    }
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static void voxel_filter(const cloud* in, double v, cloud* out)
{
    out->n = 0;
    if (in->n == 0) return;
    vk* a = (vk*)malloc(sizeof(vk) * (size_t)in->n);
    for (int64_t i = 0; i < in->n; ++i) {
        for (int k = 0; k < 3; ++k) a[i].key[k] = (int64_t)floor((double)in->p[3 * i + k] / v);
        a[i].idx = i;
    }
    qsort(a, (size_t)in->n, sizeof(vk), vk_cmp);
    int64_t i = 0;
    while (i < in->n) {
        int64_t j = i;
        double sx = 0, sy = 0, sz = 0;
        while (j < in->n && memcmp(a[j].key, a[i].key, sizeof(a[i].key)) == 0) {
            sx += in->p[3 * a[j].idx];
            sy += in->p[3 * a[j].idx + 1];
            sz += in->p[3 * a[j].idx + 2];
            ++j;
        }
        double c = (double)(j - i);
        cloud_add(out, sx / c, sy / c, sz / c);
        i = j;
    }
    free(a);
}

/* pick the voxel size whose filtered cloud is closest to `target` points */
static void voxel_filter_to(const cloud* in, int64_t target, cloud* out)
{
    if (in->n <= target) {
        out->n = 0;
        for (int64_t i = 0; i < in->n; ++i) cloud_add(out, in->p[3 * i], in->p[3 * i + 1], in->p[3 * i + 2]);
        return;
    }
    double lo = 0.005, hi = 20.0;
    for (int it = 0; it < 40; ++it) {
        double mid = sqrt(lo * hi);
        voxel_filter(in, mid, out);
        if (out->n > target) lo = mid; else hi = mid;
    }
    voxel_filter(in, lo, out); /* the smallest size found that keeps >= target points */
}

/* keep m of the points, chosen uniformly (partial Fisher-Yates) */
static void random_subset(cloud* c, int64_t m, syn_rng* r)
{
    if (m >= c->n) return;
    for (int64_t i = 0; i < m; ++i) {
        int64_t j = i + (int64_t)(rng_u(r) * (double)(c->n - i));
        if (j >= c->n) j = c->n - 1;
        for (int k = 0; k < 3; ++k) {
            float t = c->p[3 * i + k];
            c->p[3 * i + k] = c->p[3 * j + k];
            c->p[3 * j + k] = t;
        }
    }
    c->n = m;
}

/* ------------------------------------------------------------------------ */
/* public entry points                                                       */
/* ------------------------------------------------------------------------ */
SYN_API void syn_free(void* p) { free(p); }

/* scene extent (m) of a config's map */
SYN_API int syn_scene_extent(int cfg, double lo[3], double hi[3])
{
    scene s;
    if (make_scene(cfg, &s)) return -1;
    for (int i = 0; i < 3; ++i) { lo[i] = s.lo[i]; hi[i] = s.hi[i]; }
    free(s.b);
    return 0;
}

/* map cloud of config cfg: 1 = 5 cm lattice (~0.35 M), 2 = ~5 M random,
 * 3 = ~40 M random; n_override > 0 replaces the random count */
SYN_API int syn_map(int cfg, int64_t n_override, float** xyz, int64_t* n)
{
    scene s;
    if (make_scene(cfg, &s)) return -1;
    cloud c = {0};
    if (cfg == 1) sample_lattice(&s, 0.05, &c);
    else sample_random(&s, n_override > 0 ? n_override : (cfg == 2 ? 5000000 : 40000000), 1100 + (uint64_t)cfg, &c);
    free(s.b);
    *xyz = c.p;
    *n = c.n;
    return 0;
}

/* Scan number `index` of config cfg.  k_target > 0 asks for exactly that many
 * points (64-beam pattern, voxel filter then a uniform subset); 0 gives the
 * config's own scan.  pose[6] = planted (x, y, z, roll, pitch, yaw). */
SYN_API int syn_scan(int cfg, int index, int64_t k_target, float** xyz, int64_t* k, double pose[6])
{
    scene s;
    if (make_scene(cfg, &s)) return -1;
    syn_rng rp, rn;
    rng_seed(&rp, 2000000ull + 1000ull * (uint64_t)cfg + (uint64_t)index);
    rng_seed(&rn, 3000000ull + 1000ull * (uint64_t)cfg + (uint64_t)index);

    double z = cfg == 3 ? 2.0 : 1.0;
    double rp_max = (cfg == 2 ? 3.0 : 2.0) * 3.141592653589793 / 180.0;
    double plo[2], phi[2];
    if (cfg == 3) { plo[0] = plo[1] = 200.0; phi[0] = phi[1] = 600.0; }
    else { plo[0] = s.lo[0] + 0.5; plo[1] = s.lo[1] + 0.5; phi[0] = s.hi[0] - 0.5; phi[1] = s.hi[1] - 0.5; }
    double t[3];
    for (int tries = 0; tries < 10000; ++tries) {
        t[0] = rng_range(&rp, plo[0], phi[0]);
        t[1] = rng_range(&rp, plo[1], phi[1]);
        t[2] = z;
        if (!inside_any(&s, t, 0.4)) break;
    }
    double roll = rng_range(&rp, -rp_max, rp_max);
    double pitch = rng_range(&rp, -rp_max, rp_max);
    double yaw = rng_range(&rp, 0.0, 6.283185307179586);
    double R[9];
    rot_zyx(roll, pitch, yaw, R);
    pose[0] = t[0]; pose[1] = t[1]; pose[2] = t[2];
    pose[3] = roll; pose[4] = pitch; pose[5] = yaw;

    lidar L;
    double sigma = 0.03, drop = 0.0;
    int64_t target;
    if (k_target > 0) {
        L.beams = 64; L.vfov_deg = 15.0; L.hres_deg = 0.2; L.max_range = cfg == 3 ? 100.0 : 50.0;
        target = k_target;
    } else if (cfg == 1) {
        L.beams = 32; L.vfov_deg = 15.0; L.hres_deg = 0.2; L.max_range = 50.0;
        target = 1000; sigma = 0.02;
    } else if (cfg == 2) {
        L.beams = 16; L.vfov_deg = 15.0; L.hres_deg = 0.2; L.max_range = 50.0;
        target = 8889; drop = 0.10;     /* ~8 k points after the 10% drop */
    } else {
        L.beams = 64; L.vfov_deg = 22.5; L.hres_deg = 0.2; L.max_range = 100.0;
        target = 20000;
    }
    cloud hits = {0}, pts = {0};
    cast_scan(&s, &L, t, R, &hits);
    free(s.b);
    if (cfg == 1 && k_target <= 0) {
        random_subset(&hits, target, &rn);
        pts = hits;
        hits.p = NULL;
    } else {
        voxel_filter_to(&hits, k_target > 0 ? (target + target / 5) : target, &pts);
        if (k_target > 0) random_subset(&pts, target, &rn);
    }
    free(hits.p);
    for (int64_t i = 0; i < 3 * pts.n; ++i) pts.p[i] = (float)((double)pts.p[i] + sigma * rng_normal(&rn));
    if (drop > 0) {
        int64_t w = 0;
        for (int64_t i = 0; i < pts.n; ++i) {
            if (rng_u(&rn) < drop) continue;
            for (int k2 = 0; k2 < 3; ++k2) pts.p[3 * w + k2] = pts.p[3 * i + k2];
            ++w;
        }
        pts.n = w;
    }
    *xyz = pts.p;
    *k = pts.n;
    return 0;
}

/* Poisson arrival trace: n requests at rate lam (1/s), scan sizes
 * log-uniform in [kmin, kmax]; arrivals in seconds from 0. */
SYN_API void syn_trace(uint64_t seed, double lam, int64_t n, int64_t kmin, int64_t kmax,
                       double* arrival, int64_t* ks)
{
    syn_rng r;
    rng_seed(&r, seed);
    double t = 0;
    for (int64_t i = 0; i < n; ++i) {
        t += -log(1.0 - rng_u(&r)) / lam;
        arrival[i] = t;
        double lk = log((double)kmin) + (log((double)kmax) - log((double)kmin)) * rng_u(&r);
        ks[i] = (int64_t)floor(exp(lk) + 0.5);
    }
}
