// bbs_internal.cuh -- shared internals of libbbs (GPU 3D-BBS, arxiv 2310.10023).
//
// Layout of a level map H^l (Sec. III-C) in HBM: an open-addressing hash
// table (linear probing, Eq. (10)) whose buckets are 32-byte "bricks".  A
// brick covers the 4 x 4 x 4 voxels 4b + [0,4)^3 and stores the occupancy
// of the overlapping 5 x 5 x 5 block 4b + [0,5)^3 as five 25-bit planes, so
// the 2 x 2 x 2 voxel block v + {0,1}^3 of ANY voxel v lies inside the single
// brick floor(v / 4).  One probe -- one 32-byte L2 sector -- therefore
// answers membership for all eight translational siblings of a branched node
// (children 2c + j, Eq. (13)) at once.  Membership is exact; the hash
// function and table size change speed only, never a score.
#pragma once

#include <cuda_runtime.h>
#include <cstring>
#include <stdint.h>

#include "bbs.h"

namespace bbs {

constexpr int32_t KEY_LIMIT = 1 << 20;         // voxel keys live in [-2^20, 2^20)
constexpr int32_t MAP_KEY_MAX = (1 << 20) - 4; // |fine map key| bound (BBS_EKEYRANGE beyond)
constexpr int32_t BRICK_BIAS = 1 << 19;        // brick coordinates in [-2^19, 2^19)
constexpr unsigned long long EMPTY_KEY = ~0ull;
constexpr int MAX_LEVELS = BBS_MAX_LEVELS;

struct __align__(32) Brick {
    unsigned long long key;  // packed brick coordinates, EMPTY_KEY when free
    uint32_t plane[5];       // plane z: bit (x + 5 y) = voxel 4b + (x, y, z) occupied
    uint32_t pad;
};
static_assert(sizeof(Brick) == 32, "brick must be one 32-byte sector");

// Read-only view of one level's table passed to kernels by value.
//
// Two bucket layouts.  "Wide": a 64-bit absolute brick key and the five
// planes (two 16-byte loads per probe).  "Compact", used whenever the level's
// voxels fit in 8192 x 8192 x 4092 keys: bricks are indexed relative to
// `base` (a multiple of 4 at least 4 below the smallest stored key) and packed
// into 32 bits (x 11, y 11, z 10 bits); each 16-byte half of the bucket repeats
// the key and holds the three planes a query can need, [key, p0, p1, p2 |
// key, p2, p3, p4], so a probe is ONE 16-byte load of half (oz >> 1).  A query
// block outside [base, base + rmax] cannot touch a stored voxel and is a miss
// without any load.
struct LevelView {
    const Brick* slots;
    uint32_t shift;   // home slot = hash >> shift   (table size 2^(32 - shift))
    uint32_t mask;    // hashed: table size - 1; dense: index of the zero brick past the box; bytes: last cell
    int32_t maxp;     // longest probe distance of any stored brick
    int32_t layout;   // LAYOUT_WIDE, LAYOUT_COMPACT or LAYOUT_DENSE
    int32_t base[3];  // compact, dense: key origin (multiple of 4)
    uint32_t rmax[3]; // compact, dense: largest relative key a query block may start at
    uint32_t nby, nbz; // dense: bricks along y and z (x: rmax[0] / 4 + 1); bytes: keys (rmax + 2)
};

// Level table layouts.  Wide: open addressing over 32-byte bricks with a
// 64-bit brick key.  Compact: open addressing, a 32-bit relative brick key
// repeated in each 16-byte half.  Dense: every brick of the level's key box
// at index (bx * nby + by) * nbz + bz (relative brick coordinates), no key:
// one load per query; chosen when the box is small enough.
// Bytes: one byte per key of the box (x slowest), bit jx + 2 jy + 4 jz set
// when key + (jx, jy, jz) is in the level's set: the 8 children of a key
// block in one byte load; the box reaches one key past rmax on every axis,
// an empty key that out-of-box queries are clamped to.
enum { LAYOUT_WIDE = 0, LAYOUT_COMPACT = 1, LAYOUT_DENSE = 2, LAYOUT_BYTES = 3 };

constexpr uint32_t CEMPTY = 0xFFFFFFFFu;

__host__ __device__ __forceinline__ uint32_t cbrick_pack(uint32_t bx, uint32_t by, uint32_t bz)
{
    return bx | (by << 11) | (bz << 22);
}

__host__ __device__ __forceinline__ uint32_t cbrick_hash(uint32_t key) { return key * 0x9E3779B1u; }

// Compact probe of relative brick (bx, by, bz), half `h` (0: planes 0-2, 1: planes 2-4).
// On success w = {key, plane a, plane a+1, plane a+2} with a = 2h.
__device__ __forceinline__ bool probe_compact(const LevelView& L, uint32_t key, int h, uint4& w)
{
    const uint32_t s = cbrick_hash(key) >> L.shift;
    w = __ldg(reinterpret_cast<const uint4*>(L.slots + s) + h);   // the home bucket: almost every probe ends here
    if (w.x == key) return true;
    if (w.x == CEMPTY) return false;
    for (int p = 1; p <= L.maxp; ++p) {
        const uint4* q = reinterpret_cast<const uint4*>(L.slots + ((s + (uint32_t)p) & L.mask)) + h;
        w = __ldg(q);
        if (w.x == key) return true;
        if (w.x == CEMPTY) return false;
    }
    return false;
}

// Search grid passed to kernels by value.
struct DevGrid {
    int32_t levels;
    uint32_t flags;
    int32_t N[MAX_LEVELS][3];    // angle segments per level and axis
    int32_t a[MAX_LEVELS][3];    // Eq. (14) divisions (index l: from l to l-1)
    int32_t cs_off[MAX_LEVELS][3];   // first (cos, sin) entry of each level and axis
    double r;                    // voxel size of level 0
    double inv_r;                // fl64(1 / r)
};

// fl32(fl64(x / r)).  q = fl64(x * fl64(1/r)) lies within 3 units in the last
// place of x / r, so fl32(q) is the float of the exact quotient unless q sits
// near a float rounding midpoint (its low 29 bits within 64 of 2^28) or
// outside the normal float range; those cases divide exactly.  Both tests
// read q's bits (integer work): |q| in [2^-120, 2^120) is a biased exponent
// in [1023 - 120, 1023 + 120) (zero, subnormals, infinities and NaN fall
// outside).
__device__ __forceinline__ float div_r_f32(double x, double r, double inv_r)
{
    const double q = __dmul_rn(x, inv_r);
    const uint32_t lo = (uint32_t)__double2loint(q) & 0x1FFFFFFFu;
    const uint32_t d = lo > 0x10000000u ? lo - 0x10000000u : 0x10000000u - lo;
    const uint32_t e = ((uint32_t)__double2hiint(q) >> 20) & 0x7FFu;
    if (d > 64u && e - (1023u - 120u) < 240u) return __double2float_rn(q);
    return __double2float_rn(__ddiv_rn(x, r));
}

// Entry e (row-major) of A = fl32(R / r) for rotation `rot` at level l: the
// same products and sums as rotation_rows, one entry per call
__device__ __forceinline__ float rotation_entry(const double2* __restrict__ cs, const DevGrid& g, int l, uint32_t rot, int e)
{
    const uint32_t ng = (uint32_t)g.N[l][2], nb = (uint32_t)g.N[l][1];
    const uint32_t q1 = rot / ng, ig = rot - q1 * ng, ia = q1 / nb, ib = q1 - ia * nb;
    const double2 A_ = cs[g.cs_off[l][0] + (int32_t)ia];
    const double2 B_ = cs[g.cs_off[l][1] + (int32_t)ib];
    const double2 G_ = cs[g.cs_off[l][2] + (int32_t)ig];
    const double ca = A_.x, sa = A_.y, cb = B_.x, sb = B_.y, cg = G_.x, sg = G_.y;
    double x;
    switch (e) {
        case 0: x = __dmul_rn(cg, cb); break;
        case 1: x = __dsub_rn(__dmul_rn(__dmul_rn(cg, sb), sa), __dmul_rn(sg, ca)); break;
        case 2: x = __dadd_rn(__dmul_rn(__dmul_rn(cg, sb), ca), __dmul_rn(sg, sa)); break;
        case 3: x = __dmul_rn(sg, cb); break;
        case 4: x = __dadd_rn(__dmul_rn(__dmul_rn(sg, sb), sa), __dmul_rn(cg, ca)); break;
        case 5: x = __dsub_rn(__dmul_rn(__dmul_rn(sg, sb), ca), __dmul_rn(cg, sa)); break;
        case 6: x = -sb; break;
        case 7: x = __dmul_rn(cb, sa); break;
        default: x = __dmul_rn(cb, ca); break;
    }
    return div_r_f32(x, g.r, g.inv_r);
}

// A = fl32(R / r) of rotation `rot` at level l (row-major, 9 entries), with
// R = Rz(gamma) Ry(beta) Rx(alpha) of the segment angles (Sec. III-A) formed
// in FP64 from the host cos / sin table cs, every product and sum rounded
__device__ __forceinline__ void rotation_rows(const double2* __restrict__ cs, const DevGrid& g, int l, uint32_t rot,
                                              float A[9])
{
    const uint32_t ng = (uint32_t)g.N[l][2], nb = (uint32_t)g.N[l][1];
    const uint32_t q1 = rot / ng, ig = rot - q1 * ng, ia = q1 / nb, ib = q1 - ia * nb;
    const double2 A_ = cs[g.cs_off[l][0] + (int32_t)ia];
    const double2 B_ = cs[g.cs_off[l][1] + (int32_t)ib];
    const double2 G_ = cs[g.cs_off[l][2] + (int32_t)ig];
    const double ca = A_.x, sa = A_.y, cb = B_.x, sb = B_.y, cg = G_.x, sg = G_.y;
    double R[9];
    R[0] = __dmul_rn(cg, cb);
    R[1] = __dsub_rn(__dmul_rn(__dmul_rn(cg, sb), sa), __dmul_rn(sg, ca));
    R[2] = __dadd_rn(__dmul_rn(__dmul_rn(cg, sb), ca), __dmul_rn(sg, sa));
    R[3] = __dmul_rn(sg, cb);
    R[4] = __dadd_rn(__dmul_rn(__dmul_rn(sg, sb), sa), __dmul_rn(cg, ca));
    R[5] = __dsub_rn(__dmul_rn(__dmul_rn(sg, sb), ca), __dmul_rn(cg, sa));
    R[6] = -sb;
    R[7] = __dmul_rn(cb, sa);
    R[8] = __dmul_rn(cb, ca);
    for (int i = 0; i < 9; ++i) A[i] = div_r_f32(R[i], g.r, g.inv_r);
}

// ---- the same rows without FP64 arithmetic ----------------------------------
// A value held as h + l in two floats (double-float).  FP64 runs at a small
// fraction of the FP32 rate on this part, so the search's own row formation
// takes the rows of rotation_rows from FP32 operations and falls back to
// rotation_rows only where those cannot decide the result.
struct DF {
    float h, l;
};

// x as h + l: h its leading 24 significand bits (truncated, exact), l the
// remaining 29 bits rounded to a float, so |h + l - x| <= 2^-47 |x|.  Integer
// work and one conversion.  ok becomes false unless x is zero or a normal
// number with |x| in [2^-60, 2^30) (the cos / sin of an angle a rounding
// residue away from a multiple of pi/2 lies near 1e-16: kept; a product of
// two such stays in the FP32 normal range, and the absolute error of its low
// part, which may fall below it, is far below the tolerance of any entry it
// feeds).
__device__ __forceinline__ DF df_split(double x, bool& ok)
{
    const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
    const uint32_t sgn = hi & 0x80000000u;
    if (((hi & 0x7FFFFFFFu) | lo) == 0u) return DF{__uint_as_float(sgn), 0.0f};
    const int e = (int)((hi >> 20) & 0x7FFu) - 1023;
    ok = ok && e >= -60 && e < 30;
    const int ec = e < -60 ? -60 : (e >= 30 ? 29 : e);   // keeps the bit patterns below well-formed
    const uint32_t hb = sgn | ((uint32_t)(ec + 127) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29);
    // the low 29 significand bits weigh 2^(e - 52) each
    const float l = __fmul_rn(__uint2float_rn(lo & 0x1FFFFFFFu), __uint_as_float((uint32_t)(ec - 52 + 127) << 23));
    return DF{__uint_as_float(hb), sgn ? -l : l};
}

// a * b: h = fl(a.h b.h), l = its exact error plus the cross terms (a.l b.l
// dropped); relative error below 2^-45 for inputs of 2^-47 and unnormalized
// products of this function
__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return DF{p, e};
}

// exact sum of two floats: s + t = a + b
__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF{s, t};
}

// a + b, normalized (|l| <= ulp(h) / 2)
__device__ __forceinline__ DF df_add(DF a, DF b)
{
    const DF s = two_sum(a.h, b.h);
    return two_sum(s.h, __fadd_rn(__fadd_rn(s.l, a.l), b.l));
}

// fl32 of a real y known to lie within D of h + l (h + l normalized with h
// the float nearest to it): h itself unless y may lie across a rounding
// boundary of h (or h is zero, tiny or huge), which clears ok
__device__ __forceinline__ float df_round(DF v, float D, bool& ok)
{
    const uint32_t hb = __float_as_uint(v.h);
    const uint32_t eb = hb & 0x7F800000u;
    ok = ok && eb >= (40u << 23) && eb < (215u << 23);
    // half the spacing of the floats around h; the gap below a power of two is half as wide
    float half = __uint_as_float((eb < (40u << 23) ? (40u << 23) : eb) - (24u << 23));
    if ((hb & 0x7FFFFFu) == 0u) half = __fmul_rn(half, 0.5f);
    ok = ok && __fadd_rn(fabsf(v.l), D) < half;
    return v.h;
}

// A = fl32(R / r) of rotation `rot` at level l, equal bit for bit to
// rotation_rows wherever this returns true.  Every entry of R is formed from
// double-float copies of the FP64 cos / sin values with FP32 operations
// (error-free products by FMA, error-free sums): the result lies within
// D = 2^-40 (|V| + (|t1| + |t2|) / r) of fl64(R_i / r) (V the double-float
// quotient, t1 and t2 the two product terms of a sum entry; the actual error,
// FP64 roundings of R included, stays below 2^-42 of the same quantity), and
// where every real within D of V rounds to one float, that float is
// fl32(fl64(R_i / r)), the value rotation_rows returns (its quotient test only
// chooses how that value is reached).  A term with an exactly zero factor
// (sin 0) is an exact signed zero in both arithmetics, formed here with the
// same IEEE sign rules (products, and the sum of two zero terms).  Otherwise,
// and for inputs or entries out of range or too close to a rounding
// boundary, it returns false and the caller forms the rows in FP64.
__device__ __forceinline__ bool rotation_rows_df(const double2* __restrict__ cs, const DevGrid& g, int l, uint32_t rot,
                                                 float A[9])
{
    const uint32_t ng = (uint32_t)g.N[l][2], nb = (uint32_t)g.N[l][1];
    const uint32_t q1 = rot / ng, ig = rot - q1 * ng, ia = q1 / nb, ib = q1 - ia * nb;
    const double2 A_ = cs[g.cs_off[l][0] + (int32_t)ia];
    const double2 B_ = cs[g.cs_off[l][1] + (int32_t)ib];
    const double2 G_ = cs[g.cs_off[l][2] + (int32_t)ig];
    bool ok = true;
    const DF ca = df_split(A_.x, ok), sa = df_split(A_.y, ok), cb = df_split(B_.x, ok), sb = df_split(B_.y, ok);
    const DF cg = df_split(G_.x, ok), sg = df_split(G_.y, ok), ir = df_split(g.inv_r, ok);
    constexpr float TOL = 9.094947e-13f;    // 2^-40
    // 2^-100: a sum entry's terms must reach it together; a term far below
    // (two sines a rounding residue from zero) may lose bits to the FP32
    // range, an absolute error far below the tolerance
    constexpr float TINY = 7.888609e-31f;
    const float irh = fabsf(ir.h);
    // a product entry x y, then the quotient
    auto prod = [&](DF x, DF y) -> float {
        if (x.h == 0.0f || y.h == 0.0f) return __fmul_rn(__fmul_rn(x.h, y.h), irh);   // exact signed zero
        DF v = df_mul(df_mul(x, y), ir);
        v = two_sum(v.h, v.l);
        return df_round(v, __fmul_rn(TOL, fabsf(v.h)), ok);
    };
    // a sum entry (x1 y1) z1 + s x2 y2 (s = -1 when neg), then the quotient
    auto sum = [&](DF x1, DF y1, DF z1, DF x2, DF y2, bool neg) -> float {
        const bool zero1 = x1.h == 0.0f || y1.h == 0.0f || z1.h == 0.0f, zero2 = x2.h == 0.0f || y2.h == 0.0f;
        const DF t1 = df_mul(df_mul(x1, y1), z1);
        DF t2 = df_mul(x2, y2);
        if (neg) t2 = DF{-t2.h, -t2.l};
        if (zero1 && zero2) return __fmul_rn(__fadd_rn(t1.h, t2.h), irh);   // two zero terms: exact signed zero
        ok = ok && __fadd_rn(fabsf(t1.h), fabsf(t2.h)) >= TINY;
        DF v = df_mul(df_add(t1, t2), ir);
        v = two_sum(v.h, v.l);
        const float D = __fmul_rn(TOL, __fadd_rn(fabsf(v.h), __fmul_rn(__fadd_rn(fabsf(t1.h), fabsf(t2.h)), irh)));
        return df_round(v, D, ok);
    };
    A[0] = prod(cg, cb);
    A[1] = sum(cg, sb, sa, sg, ca, true);
    A[2] = sum(cg, sb, ca, sg, sa, false);
    A[3] = prod(sg, cb);
    A[4] = sum(sg, sb, sa, cg, ca, false);
    A[5] = sum(sg, sb, ca, cg, sa, true);
    A[6] = prod(DF{-sb.h, -sb.l}, DF{1.0f, 0.0f});   // R6 = -sb exactly
    A[7] = prod(cb, sa);
    A[8] = prod(cb, ca);
    return ok;
}

// The rows the search and the pose grid use: rotation_rows_df, and the FP64
// formation for the rare rotations it cannot decide (the same bits either way)
__device__ __forceinline__ void search_rows(const double2* __restrict__ cs, const DevGrid& g, int l, uint32_t rot,
                                            float A[9])
{
    if (!rotation_rows_df(cs, g, l, rot, A)) rotation_rows(cs, g, l, rot, A);
}

// Node / task record in HBM: translation indices and (rotation index << 5 | level).
struct __align__(16) NodeRec {
    int32_t cx, cy, cz;
    uint32_t rl;
};

__host__ __device__ __forceinline__ uint32_t rl_pack(uint32_t rot, int level) { return (rot << 5) | (uint32_t)level; }

// Lexicographic order of leaves (Algorithm 2's tie rule among equal scores):
// translation indices (c_x, c_y, c_z) first, as one 63-bit key of biased
// 21-bit fields (leaf translations lie in [-2^20, 2^20)), then the rotation
// index, whose order equals (c_alpha, c_beta, c_gamma) order.
__host__ __device__ __forceinline__ unsigned long long lex_translation(const NodeRec& n)
{
    return ((unsigned long long)(uint32_t)(n.cx + KEY_LIMIT) << 42) | ((unsigned long long)(uint32_t)(n.cy + KEY_LIMIT) << 21) |
           (unsigned long long)(uint32_t)(n.cz + KEY_LIMIT);
}
__host__ __device__ __forceinline__ int rl_level(uint32_t rl) { return (int)(rl & 31u); }
__host__ __device__ __forceinline__ uint32_t rl_rot(uint32_t rl) { return rl >> 5; }

__host__ __device__ __forceinline__ unsigned long long brick_pack(int32_t bx, int32_t by, int32_t bz)
{
    return ((unsigned long long)(uint32_t)(bx + BRICK_BIAS) << 40) |
           ((unsigned long long)(uint32_t)(by + BRICK_BIAS) << 20) |
           (unsigned long long)(uint32_t)(bz + BRICK_BIAS);
}

// 32-bit mix of the three brick coordinates; the table uses the top bits.
__host__ __device__ __forceinline__ uint32_t brick_hash(int32_t bx, int32_t by, int32_t bz)
{
    uint32_t h = (uint32_t)bx * 0x9E3779B1u ^ (uint32_t)by * 0x85EBCA77u ^ (uint32_t)bz * 0xC2B2AE3Du;
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    return h;
}

__device__ __forceinline__ bool key_in_range(int32_t k)
{
    return (uint32_t)(k + KEY_LIMIT) < (uint32_t)(2 * KEY_LIMIT);
}

// Find brick (bx, by, bz).  On success lo = {key, plane0, plane1},
// hi = {plane2, plane3, plane4, pad}.  Bounded by the table's longest probe.
__device__ __forceinline__ bool probe_brick(const LevelView& L, int32_t bx, int32_t by, int32_t bz,
                                            uint4& lo, uint4& hi)
{
    const unsigned long long key = brick_pack(bx, by, bz);
    uint32_t s = brick_hash(bx, by, bz) >> L.shift;
    for (int p = 0; p <= L.maxp; ++p) {
        const uint4* q = reinterpret_cast<const uint4*>(L.slots + ((s + (uint32_t)p) & L.mask));
        lo = __ldg(q);
        hi = __ldg(q + 1);
        const unsigned long long k = ((unsigned long long)lo.y << 32) | lo.x;
        if (k == key) return true;
        if (k == EMPTY_KEY) return false;
    }
    return false;
}

__device__ __forceinline__ uint32_t brick_plane(const uint4& lo, const uint4& hi, int z)
{
    uint32_t p = lo.z;
    p = (z == 1) ? lo.w : p;
    p = (z == 2) ? hi.x : p;
    p = (z == 3) ? hi.y : p;
    p = (z == 4) ? hi.z : p;
    return p;
}

// Occupancy of voxel key k at one level (bbs_score_batch).
__device__ __forceinline__ uint32_t voxel_bit(const LevelView& L, int32_t kx, int32_t ky, int32_t kz)
{
    if (L.layout == LAYOUT_BYTES) {
        const uint32_t rx = (uint32_t)(kx - L.base[0]), ry = (uint32_t)(ky - L.base[1]), rz = (uint32_t)(kz - L.base[2]);
        if (rx > L.rmax[0] || ry > L.rmax[1] || rz > L.rmax[2]) return 0u;
        const uint8_t* b = reinterpret_cast<const uint8_t*>(L.slots);
        return __ldg(b + ((size_t)rx * L.nby + ry) * L.nbz + rz) & 1u;
    }
    if (L.layout == LAYOUT_DENSE) {
        const uint32_t rx = (uint32_t)(kx - L.base[0]), ry = (uint32_t)(ky - L.base[1]), rz = (uint32_t)(kz - L.base[2]);
        if (rx > L.rmax[0] || ry > L.rmax[1] || rz > L.rmax[2]) return 0u;
        const uint32_t idx = ((rx >> 2) * L.nby + (ry >> 2)) * L.nbz + (rz >> 2);
        const int oz = (int)(rz & 3u);
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(L.slots + idx) + (oz >> 1));
        return (((oz & 1) ? w.z : w.y) >> ((rx & 3u) + 5u * (ry & 3u))) & 1u;
    }
    if (L.layout == LAYOUT_COMPACT) {
        const uint32_t rx = (uint32_t)(kx - L.base[0]), ry = (uint32_t)(ky - L.base[1]), rz = (uint32_t)(kz - L.base[2]);
        if (rx > L.rmax[0] || ry > L.rmax[1] || rz > L.rmax[2]) return 0u;
        uint4 w;
        const int oz = (int)(rz & 3u);
        if (!probe_compact(L, cbrick_pack(rx >> 2, ry >> 2, rz >> 2), oz >> 1, w)) return 0u;
        return (((oz & 1) ? w.z : w.y) >> ((rx & 3u) + 5u * (ry & 3u))) & 1u;
    }
    if (!(key_in_range(kx) && key_in_range(ky) && key_in_range(kz))) return 0u;
    uint4 lo, hi;
    if (!probe_brick(L, kx >> 2, ky >> 2, kz >> 2, lo, hi)) return 0u;
    return (brick_plane(lo, hi, kz & 3) >> ((kx & 3) + 5 * (ky & 3))) & 1u;
}

// Fine voxel key: u_i = floor(((A_i0 s_x + A_i1 s_y) + A_i2 s_z)), every
// product and sum rounded to FP32 on its own (no FMA), then an exact floor.
__device__ __forceinline__ int32_t fine_key(float4 row, float4 s)
{
    const float q = __fadd_rn(__fadd_rn(__fmul_rn(row.x, s.x), __fmul_rn(row.y, s.y)), __fmul_rn(row.z, s.z));
    return __float2int_rd(q);
}

// Rotational children of angle index c at level l: [lo, hi) at level l - 1.
// Default: the finer segments whose centres fall inside segment c, i.e. the
// smallest c' with (2c' + 1) N_l >= 2 c N_{l-1} starts the range; with
// BBS_CHILD_LITERAL the printed a*c + j, j < a, clipped to N_{l-1}.
__host__ __device__ __forceinline__ int64_t child_first(int64_t np, int64_t nc, int64_t c)
{
    const int64_t num = 2 * c * nc - np;
    return num <= 0 ? 0 : (num + 2 * np - 1) / (2 * np);
}

__host__ __device__ __forceinline__ void child_range(const DevGrid& g, int l, int ax, int32_t c, int32_t& lo,
                                                     int32_t& hi)
{
    const int64_t np = g.N[l][ax], nc = g.N[l - 1][ax];
    if (g.flags & BBS_CHILD_LITERAL) {
        const int64_t a = g.a[l][ax];
        int64_t x = a * c, y = a * c + a;
        lo = (int32_t)(x < nc ? x : nc);
        hi = (int32_t)(y < nc ? y : nc);
        return;
    }
    const int64_t x = child_first(np, nc, c);
    int64_t y = child_first(np, nc, (int64_t)c + 1);
    lo = (int32_t)(x < nc ? x : nc);
    hi = (int32_t)(y < nc ? y : nc);
}

// number of children of a node at level l (0 for leaves): 8 translations
// times the rotational children of each axis
__host__ __device__ __forceinline__ int64_t node_children(const DevGrid& g, int l, uint32_t rot)
{
    if (l <= 0) return 0;
    const int32_t ng = g.N[l][2], nb = g.N[l][1];
    const int32_t cg = (int32_t)(rot % (uint32_t)ng);
    const int32_t cb = (int32_t)((rot / (uint32_t)ng) % (uint32_t)nb);
    const int32_t ca = (int32_t)(rot / ((uint32_t)ng * (uint32_t)nb));
    int32_t lo, hi;
    int64_t n = 8;
    child_range(g, l, 0, ca, lo, hi);
    n *= (hi - lo);
    child_range(g, l, 1, cb, lo, hi);
    n *= (hi - lo);
    child_range(g, l, 2, cg, lo, hi);
    n *= (hi - lo);
    return n;
}

// Programmatic dependent launch (sm_90+): a kernel launched with it may start
// while its predecessor in the stream still runs; pdl_wait() blocks until the
// predecessor has completed and its writes are visible (a no-op without the
// launch attribute), and pdl_trigger() lets the successor's CTAs be
// scheduled once every CTA of this grid has triggered or exited.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---- host side ------------------------------------------------------------

// launch `k` on `st`, with the programmatic-dependent-launch attribute when pdl
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, bool pdl, Args... args)
{
    cudaLaunchConfig_t cfg;
    std::memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, ((KArgs)args)...);
}

int set_error(int code, const char* fmt, ...);
void clear_error();

#define BBS_CUDA_TRY(call)                                                                              \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            return ::bbs::set_error(BBS_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                                    __LINE__);                                                          \
    } while (0)

#define BBS_TRY(expr)           \
    do {                        \
        int rc_ = (expr);       \
        if (rc_ < 0) return rc_; \
    } while (0)

// Per-level host record of a built map.
struct LevelTable {
    Brick* slots;
    int log2T;
    int32_t maxp;
    int32_t layout;
    int32_t base[3];
    uint32_t rmax[3];
    uint32_t nby, nbz;
    int64_t n_slots;     // buckets (hashed), bricks of the box + 1 zero brick (dense), keys (bytes)
    int64_t n_bricks;
    int64_t n_voxels;
    int64_t displaced;   // bricks not in their home slot
};

}  // namespace bbs

struct bbs_maps {
    int device;
    int levels;
    float r;
    uint32_t flags;
    double lo[3], hi[3];
    bbs::LevelTable lv[BBS_MAX_LEVELS];
    void* arena;          // one device allocation holding every level table
    size_t arena_bytes;
};

namespace bbs {

inline LevelView level_view(const bbs_maps* m, int l)
{
    LevelView v;
    v.slots = m->lv[l].slots;
    v.shift = (uint32_t)(32 - m->lv[l].log2T);
    v.mask = (m->lv[l].layout == LAYOUT_DENSE || m->lv[l].layout == LAYOUT_BYTES)
                 ? (uint32_t)(m->lv[l].n_slots - 1)
                 : (uint32_t)((1ull << m->lv[l].log2T) - 1ull);
    v.maxp = m->lv[l].maxp;
    v.layout = m->lv[l].layout;
    for (int i = 0; i < 3; ++i) {
        v.base[i] = m->lv[l].base[i];
        v.rmax[i] = m->lv[l].rmax[i];
    }
    v.nby = m->lv[l].nby;
    v.nbz = m->lv[l].nbz;
    return v;
}

// every level a byte grid: the scoring kernel's byte-grid-only variant applies
inline bool maps_all_bytes(const bbs_maps* m)
{
    for (int l = 0; l < m->levels; ++l)
        if (m->lv[l].layout != LAYOUT_BYTES) return false;
    return m->levels > 0;
}

// Host pose grid (Sec. III-B Eq. (2)-(5), Sec. III-D Eq. (12)-(14)).
struct HostGrid {
    int levels;
    double r;
    double d_max;
    uint32_t flags;
    double ang_lo[3], ang_range[3];
    double delta[MAX_LEVELS];
    double dprime[MAX_LEVELS][3];
    int64_t N[MAX_LEVELS][3];
    int64_t a[MAX_LEVELS][3];
    int64_t wmin[3], wmax[3];
    int64_t nrot[MAX_LEVELS];
    int64_t rot_off[MAX_LEVELS];
    int64_t total_rot;
    int64_t cs_off[MAX_LEVELS][3];   // first (cos, sin) entry of each level and axis
    int64_t n_cs;                    // segment angles of all levels and axes
};

int grid_build(double r, int levels, double d_max, const bbs_ranges* rg, uint32_t flags, HostGrid* g);
double grid_angle(const HostGrid& g, int level, int axis, int64_t c);
DevGrid dev_grid(const HostGrid& g);
void default_ranges(const bbs_maps* m, bbs_ranges* rg);

// Per-call scan + grid state on the device.
// Scan points staged per CTA by the scoring kernel; the scan's chunk boxes
// are kept at this granularity.
constexpr int SCAN_CHUNK = 1568;

struct ScanState {
    float4* scan;      // K points, w = 0
    float4* cbox;      // per SCAN_CHUNK-point chunk: (min x, y, z, 0), (max x, y, z, 0)
    int64_t k;
    double d_max;
    double norm_max;   // the scan's largest point norm
    HostGrid grid;
    double2* cs;       // (cos, sin) of every segment angle, host libm, FP64
    float4* rot;       // 3 float4 rows per rotation of the top level l_max
    int64_t h2d, d2h;  // bytes copied while preparing
    int32_t angles_pending;   // the levels below the top still lack their (cos, sin) entries
};

// Pack the scan, build its pose grid, upload the (cos, sin) table and the top
// level's rotation rows.  defer_lower leaves the levels below the top to
// scan_finish_angles (they are needed from the first branching on).
int scan_prepare(const bbs_maps* m, const float* xyz, int64_t k, int is_device, const bbs_ranges* rg,
                 const bbs_opts* opts, cudaStream_t st, ScanState* out, bool defer_lower = false);
int scan_finish_angles(ScanState* s, cudaStream_t st);
// extra dilation the exact-bound mode needs for this grid and scan (-1: none can)
int exact_dilation_needed(const HostGrid& g, double norm_max);
// the 3 x float4 rows of every rotation of `level` -> out
cudaError_t launch_level_rows(const ScanState& s, int level, float4* out, cudaStream_t st);
void scan_release(ScanState* s, cudaStream_t st);

// GICP refinement (gicp.cu)
int gicp_target_build(const float* xyz, int64_t n, int is_device, float r, cudaStream_t st, bbs_gicp_target** out);
void gicp_target_free(bbs_gicp_target* t);
int gicp_target_info(const bbs_gicp_target* t, int64_t* n_voxels, int64_t* table_size, int32_t* max_probe);
int gicp_target_device(const bbs_gicp_target* t);
int gicp_run(const bbs_gicp_target* tg, const float* xyz, int64_t k, int is_device, const double R0[9],
             const double t0[3], const bbs_gicp_opts* o, bbs_gicp_result* res);
int gicp_linearize(const bbs_gicp_target* tg, const float* xyz, int64_t k, int is_device, const double R[9],
                   const double t[3], const bbs_gicp_opts* o, double H[36], double g[6], double* cost, int64_t* n,
                   int32_t* vox, uint8_t* found);

// kernels launched from more than one translation unit
int launch_score_nodes(const bbs_maps* m, const ScanState& s, const int32_t* d_nodes, int64_t n, int32_t* d_scores,
                       int* d_err, cudaStream_t st);

}  // namespace bbs
