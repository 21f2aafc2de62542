// gicp.cu -- local fine registration after the branch-and-bound result
// (Sec. IV: the BnB estimate seeds a generalized-ICP refinement).
//
// Target: the map cloud grouped by fine voxel key (the level-0 quantization),
// each voxel standing for the centroid of its points, kept in an
// open-addressing table whose per-voxel sums are fixed-point integers (exact,
// so the centroids do not depend on the order of the atomic adds).  Per
// linearization, one thread per scan point: transform the point (FP64, each
// operation rounded on its own), take the nearest centroid of the occupied
// voxels of the 3 x 3 x 3 block around it (kept within tau), form the
// target's normalized covariance from the centroids of the block around that
// voxel, and add the point's Gauss-Newton terms (J^T M J, J^T M d, d^T M d
// with J = [ [p]_x | -I ], M = (C_t + R C_s R^T)^-1) to per-CTA partial sums,
// reduced in a fixed order.  The source covariances come once per scan from
// the scan points within rho (one warp per point).  The host solves the 6 x 6 system and applies
// the step p -> Exp(w) p + v.
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "bbs_internal.cuh"

namespace bbs {

namespace {

constexpr int GT = 64;          // threads per CTA: a scan of 8 k points spreads over 128 SMs
constexpr int NACC = 29;        // H (21 upper-triangle entries), g (6), cost, count
constexpr double FIX = 4294967296.0;   // 2^32: fixed-point scale of the centroid sums
constexpr unsigned long long GEMPTY = ~0ull;

// one voxel of the target: key (21 bits per axis, offset 2^20), point count,
// sums of rint((x - u r) 2^32) per axis while building; then the centroid
// u r + (sum / count) 2^-32 in place of the sums, and in place of the count
// the voxel's row of the covariance array
struct GicpSlot {
    unsigned long long key;
    unsigned long long count;
    long long sum[3];
};

struct TargetView {
    const GicpSlot* slots;
    const double* cov;   // per voxel: C_t (xx, xy, xz, yy, yz, zz), row in the slot's count word
    uint32_t shift, mask;
    int32_t maxp;
    int32_t pad;
    double r;
};

__host__ __device__ __forceinline__ unsigned long long voxel_pack(int32_t x, int32_t y, int32_t z)
{
    return ((unsigned long long)(uint32_t)(x + KEY_LIMIT) << 42) | ((unsigned long long)(uint32_t)(y + KEY_LIMIT) << 21) |
           (unsigned long long)(uint32_t)(z + KEY_LIMIT);
}

struct Pose {
    double R[9];
    double t[3];
};

__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }

// the slot of voxel (x, y, z), or null when the voxel is empty
__device__ __forceinline__ const GicpSlot* target_slot(const TargetView& T, int32_t x, int32_t y, int32_t z)
{
    if (!(key_in_range(x) && key_in_range(y) && key_in_range(z))) return nullptr;
    const unsigned long long key = voxel_pack(x, y, z);
    const uint32_t s = brick_hash(x, y, z) >> T.shift;
    for (int p = 0; p <= T.maxp; ++p) {
        const GicpSlot* q = T.slots + ((s + (uint32_t)p) & T.mask);
        const unsigned long long k = q->key;
        if (k == key) return q;
        if (k == GEMPTY) return nullptr;
    }
    return nullptr;
}

// centroid of voxel (x, y, z) (stored in the slot after the build); false when empty
__device__ __forceinline__ bool target_centroid(const TargetView& T, int32_t x, int32_t y, int32_t z, double c[3])
{
    const GicpSlot* q = target_slot(T, x, y, z);
    if (!q) return false;
    for (int a = 0; a < 3; ++a) c[a] = __longlong_as_double(q->sum[a]);
    return true;
}

// every map point into its voxel: key, count and fixed-point sums; st[0]
// overflow (a probe beyond the limit), st[1] key range, st[2] longest probe,
// st[3] voxels
__global__ void target_insert_kernel(const float* __restrict__ xyz, int64_t n, float rho, double r, GicpSlot* slots,
                                     uint32_t shift, uint32_t mask, int plimit, int* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
        int32_t u[3];
        long long fx[3];
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
            const float q = floorf(__fmul_rn(x[a], rho));
            ok = ok && q >= -(float)KEY_LIMIT && q < (float)KEY_LIMIT;   // also false for NaN
            u[a] = ok ? (int32_t)q : 0;
        }
        if (!ok) {
            atomicOr(&st[1], 1);
            continue;
        }
        for (int a = 0; a < 3; ++a) fx[a] = __double2ll_rn(dmul(dsub((double)x[a], dmul((double)u[a], r)), FIX));
        const unsigned long long key = voxel_pack(u[0], u[1], u[2]);
        const uint32_t s0 = brick_hash(u[0], u[1], u[2]) >> shift;
        int p = 0;
        for (; p < plimit; ++p) {
            GicpSlot* q = slots + ((s0 + (uint32_t)p) & mask);
            const unsigned long long prev = atomicCAS(&q->key, GEMPTY, key);
            if (prev == GEMPTY || prev == key) {
                if (prev == GEMPTY) atomicAdd(&st[3], 1);
                atomicAdd(&q->count, 1ull);
                for (int a = 0; a < 3; ++a) atomicAdd((unsigned long long*)&q->sum[a], (unsigned long long)fx[a]);
                atomicMax(&st[2], p);
                break;
            }
        }
        if (p == plimit) atomicOr(&st[0], 1);
    }
}

// the sums of every occupied slot replaced by the centroid
__global__ void target_centroid_kernel(GicpSlot* slots, int64_t T, double r)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x) {
        GicpSlot& q = slots[i];
        if (q.key == GEMPTY) continue;
        const double n = (double)q.count;
        const int32_t u[3] = {(int32_t)((q.key >> 42) & 0x1FFFFF) - KEY_LIMIT, (int32_t)((q.key >> 21) & 0x1FFFFF) - KEY_LIMIT,
                              (int32_t)(q.key & 0x1FFFFF) - KEY_LIMIT};
        for (int a = 0; a < 3; ++a)
            q.sum[a] = __double_as_longlong(dadd(dmul((double)u[a], r), __ddiv_rn(__ddiv_rn((double)q.sum[a], n), FIX)));
    }
}

__global__ void target_clear_kernel(GicpSlot* slots, int64_t T)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x) {
        slots[i].key = GEMPTY;
        slots[i].count = 0;
        slots[i].sum[0] = slots[i].sum[1] = slots[i].sum[2] = 0;
    }
}

// r^2 (S / tr S + eps I), or r^2 I when tr S = 0; S and C as xx, xy, xz, yy, yz, zz
__device__ __forceinline__ void normalized(const double S[6], double r, double eps, double C[6])
{
    const double tr = dadd(dadd(S[0], S[3]), S[5]);
    const double r2 = dmul(r, r);
    for (int k = 0; k < 6; ++k) {
        const bool diag = k == 0 || k == 3 || k == 5;
        double v;
        if (tr > 0.0) {
            v = __ddiv_rn(S[k], tr);
            if (diag) v = dadd(v, eps);
        } else {
            v = diag ? 1.0 : 0.0;
        }
        C[k] = dmul(v, r2);
    }
}

// Every occupied slot its own row of the covariance array (one atomic per
// warp); row_slot[row] = slot, and the row in the slot's count word.
__global__ void target_rows_kernel(GicpSlot* slots, int64_t nslots, unsigned long long* rows, int64_t* row_slot)
{
    const int lane = threadIdx.x & 31;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x; i0 < nslots; i0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        const bool occ = i < nslots && slots[i].key != GEMPTY;
        const uint32_t ball = __ballot_sync(0xffffffffu, occ);
        if (!ball) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(rows, (unsigned long long)__popc(ball));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (occ) {
            const unsigned long long row = base + __popc(ball & ((1u << lane) - 1u));
            slots[i].count = row;
            row_slot[row] = i;
        }
    }
}

// Per occupied voxel (one thread per row, so every lane of a warp has a
// voxel: FP64 runs at a small fraction of the FP32 rate on this part), the
// shape S / tr S of the centroids of the occupied voxels of its 3 x 3 x 3
// block, sums in (dx, dy, dz) order, or -1 in the first entry when
// tr S = 0.  C_t = r^2 (shape + eps I) is formed at use, so eps stays a
// per-call option.
__global__ void target_cov_kernel(TargetView T, const int64_t* __restrict__ row_slot, int64_t nrows, double* cov)
{
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < nrows; row += (int64_t)gridDim.x * blockDim.x) {
        const GicpSlot& q = T.slots[row_slot[row]];
        const int32_t v[3] = {(int32_t)((q.key >> 42) & 0x1FFFFF) - KEY_LIMIT, (int32_t)((q.key >> 21) & 0x1FFFFF) - KEY_LIMIT,
                              (int32_t)(q.key & 0x1FFFFF) - KEY_LIMIT};
        double cnt = 0.0, sx = 0.0, sy = 0.0, sz = 0.0;
        uint32_t occ = 0;
        int bit = 0;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz, ++bit) {
                    double c[3];
                    if (!target_centroid(T, v[0] + dx, v[1] + dy, v[2] + dz, c)) continue;
                    occ |= 1u << bit;
                    cnt = dadd(cnt, 1.0);
                    sx = dadd(sx, c[0]);
                    sy = dadd(sy, c[1]);
                    sz = dadd(sz, c[2]);
                }
        const double mx = __ddiv_rn(sx, cnt), my = __ddiv_rn(sy, cnt), mz = __ddiv_rn(sz, cnt);
        double S[6] = {0, 0, 0, 0, 0, 0};
        bit = 0;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz, ++bit) {
                    double c[3];
                    if (!(occ >> bit & 1u) || !target_centroid(T, v[0] + dx, v[1] + dy, v[2] + dz, c)) continue;
                    const double ex = dsub(c[0], mx), ey = dsub(c[1], my), ez = dsub(c[2], mz);
                    S[0] = dadd(S[0], dmul(ex, ex));
                    S[1] = dadd(S[1], dmul(ex, ey));
                    S[2] = dadd(S[2], dmul(ex, ez));
                    S[3] = dadd(S[3], dmul(ey, ey));
                    S[4] = dadd(S[4], dmul(ey, ez));
                    S[5] = dadd(S[5], dmul(ez, ez));
                }
        for (int k = 0; k < 6; ++k) S[k] = __ddiv_rn(S[k], cnt);
        const double tr = dadd(dadd(S[0], S[3]), S[5]);
        for (int k = 0; k < 6; ++k) cov[6 * row + k] = tr > 0.0 ? __ddiv_rn(S[k], tr) : (k == 0 ? -1.0 : 0.0);
    }
}

// C_t = r^2 (shape + eps I), or r^2 I for an isolated voxel, as normalized() forms it
__device__ __forceinline__ void target_cov_at_use(const double* shape, double r, double eps, double C[6])
{
    const double r2 = dmul(r, r);
    const bool iso = shape[0] < 0.0;
    for (int k = 0; k < 6; ++k) {
        const bool diag = k == 0 || k == 3 || k == 5;
        const double v = iso ? (diag ? 1.0 : 0.0) : (diag ? dadd(shape[k], eps) : shape[k]);
        C[k] = dmul(v, r2);
    }
}

// Source covariances: scan points within rho of point i (FP64 distance of the
// exact coordinate differences, the point itself included).  One warp per
// point: lane l takes the points l, l + 32, ..., and the lanes' sums meet in
// a fixed butterfly (deterministic; the order differs from a sequential sum
// only by FP64 rounding).  An FP32 distance prefilter skips pairs that lie
// clearly outside (the FP32 value is within 1e-6 relative of the FP64 one).
__device__ __forceinline__ double warp_sum_d(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) source_cov_kernel(const float* __restrict__ xyz, int64_t k, double rho2,
                                                         float rho2_skip, double r, double eps, double* __restrict__ Cs)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= k) return;   // uniform per warp
    const float fx = xyz[3 * i], fy = xyz[3 * i + 1], fz = xyz[3 * i + 2];
    const double sx = fx, sy = fy, sz = fz;
    double cnt = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
    for (int64_t j = lane; j < k; j += 32) {
        const float tx = xyz[3 * j], ty = xyz[3 * j + 1], tz = xyz[3 * j + 2];
        const float ex = fx - tx, ey = fy - ty, ez = fz - tz;
        if (ex * ex + ey * ey + ez * ez > rho2_skip) continue;
        const double dx = dsub(sx, (double)tx), dy = dsub(sy, (double)ty), dz = dsub(sz, (double)tz);
        if (dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz)) > rho2) continue;
        cnt = dadd(cnt, 1.0);
        ax = dadd(ax, (double)tx);
        ay = dadd(ay, (double)ty);
        az = dadd(az, (double)tz);
    }
    cnt = warp_sum_d(cnt);
    const double mx = __ddiv_rn(warp_sum_d(ax), cnt), my = __ddiv_rn(warp_sum_d(ay), cnt),
                 mz = __ddiv_rn(warp_sum_d(az), cnt);
    double S[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t j = lane; j < k; j += 32) {
        const float tx = xyz[3 * j], ty = xyz[3 * j + 1], tz = xyz[3 * j + 2];
        const float ex = fx - tx, ey = fy - ty, ez = fz - tz;
        if (ex * ex + ey * ey + ez * ez > rho2_skip) continue;
        const double dx = dsub(sx, (double)tx), dy = dsub(sy, (double)ty), dz = dsub(sz, (double)tz);
        if (dadd(dadd(dmul(dx, dx), dmul(dy, dy)), dmul(dz, dz)) > rho2) continue;
        const double qx = dsub((double)tx, mx), qy = dsub((double)ty, my), qz = dsub((double)tz, mz);
        S[0] = dadd(S[0], dmul(qx, qx));
        S[1] = dadd(S[1], dmul(qx, qy));
        S[2] = dadd(S[2], dmul(qx, qz));
        S[3] = dadd(S[3], dmul(qy, qy));
        S[4] = dadd(S[4], dmul(qy, qz));
        S[5] = dadd(S[5], dmul(qz, qz));
    }
    for (int q = 0; q < 6; ++q) S[q] = __ddiv_rn(warp_sum_d(S[q]), cnt);
    if (lane) return;
    double C[6];
    normalized(S, r, eps, C);
    for (int q = 0; q < 6; ++q) Cs[6 * i + q] = C[q];
}

__device__ __forceinline__ int32_t clamp_key(double f)
{
    return (int32_t)fmax(fmin(f, (double)(1 << 21)), -(double)(1 << 21));
}

// 3 x 3 symmetric inverse (xx, xy, xz, yy, yz, zz) by the adjugate
__device__ __forceinline__ void sym_inverse(const double C[6], double M[6])
{
    const double a = C[0], b = C[1], c = C[2], d = C[3], e = C[4], f = C[5];
    const double A0 = d * f - e * e, A1 = c * e - b * f, A2 = b * e - c * d;
    const double det = a * A0 + b * A1 + c * A2;
    const double inv = 1.0 / det;
    M[0] = A0 * inv;
    M[1] = A1 * inv;
    M[2] = A2 * inv;
    M[3] = (a * f - c * c) * inv;
    M[4] = (b * c - a * e) * inv;
    M[5] = (a * d - b * b) * inv;
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One linearization: every point's terms, summed per CTA into partial[block][NACC]
__global__ void __launch_bounds__(GT) linearize_kernel(TargetView TG, const float* __restrict__ xyz,
                                                       const double* __restrict__ Cs, int64_t k, Pose T, double r,
                                                       double tau2, double eps, double* __restrict__ partial,
                                                       int32_t* __restrict__ vox_out, uint8_t* __restrict__ found_out)
{
    __shared__ double wsum[GT / 32][NACC];
    const int64_t i = (int64_t)blockIdx.x * GT + threadIdx.x;
    double acc[NACC];
    for (int q = 0; q < NACC; ++q) acc[q] = 0.0;
    if (i < k) {
        const double s[3] = {(double)xyz[3 * i], (double)xyz[3 * i + 1], (double)xyz[3 * i + 2]};
        double p[3];
        for (int a = 0; a < 3; ++a)
            p[a] = dadd(dadd(dadd(dmul(T.R[3 * a], s[0]), dmul(T.R[3 * a + 1], s[1])), dmul(T.R[3 * a + 2], s[2])),
                        T.t[a]);
        int32_t base[3];
        for (int a = 0; a < 3; ++a) base[a] = clamp_key(floor(__ddiv_rn(p[a], r)));
        // nearest centroid of the block's occupied voxels, first in (dx, dy, dz) order on ties
        double best = INFINITY;
        int32_t bv[3] = {0, 0, 0};
        double bc[3] = {0.0, 0.0, 0.0};
        const GicpSlot* bslot = nullptr;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    const int32_t w[3] = {base[0] + dx, base[1] + dy, base[2] + dz};
                    const GicpSlot* q = target_slot(TG, w[0], w[1], w[2]);
                    if (!q) continue;
                    double c[3], e[3];
                    for (int a = 0; a < 3; ++a) c[a] = __longlong_as_double(q->sum[a]);
                    for (int a = 0; a < 3; ++a) e[a] = dsub(p[a], c[a]);
                    const double d2 = dadd(dadd(dmul(e[0], e[0]), dmul(e[1], e[1])), dmul(e[2], e[2]));
                    if (d2 < best) {
                        best = d2;
                        bslot = q;
                        for (int a = 0; a < 3; ++a) bv[a] = w[a], bc[a] = c[a];
                    }
                }
        const bool found = best <= tau2;
        if (vox_out) {
            vox_out[3 * i] = bv[0];
            vox_out[3 * i + 1] = bv[1];
            vox_out[3 * i + 2] = bv[2];
            found_out[i] = found ? 1 : 0;
        }
        if (found) {
            // target covariance: the voxel's shape, formed at the build
            double Ct[6];
            target_cov_at_use(TG.cov + 6 * bslot->count, r, eps, Ct);
            // C = C_t + R C_s R^T
            const double* cs = Cs + 6 * i;
            const double Csf[3][3] = {{cs[0], cs[1], cs[2]}, {cs[1], cs[3], cs[4]}, {cs[2], cs[4], cs[5]}};
            double RC[3][3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    RC[a][b] = T.R[3 * a] * Csf[0][b] + T.R[3 * a + 1] * Csf[1][b] + T.R[3 * a + 2] * Csf[2][b];
            const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
            double C[6];
            for (int q = 0; q < 6; ++q)
                C[q] = Ct[q] + RC[ia[q]][0] * T.R[3 * ib[q]] + RC[ia[q]][1] * T.R[3 * ib[q] + 1] +
                       RC[ia[q]][2] * T.R[3 * ib[q] + 2];
            double M[6];
            sym_inverse(C, M);
            const double Mf[3][3] = {{M[0], M[1], M[2]}, {M[1], M[3], M[4]}, {M[2], M[4], M[5]}};
            double d[3];
            for (int a = 0; a < 3; ++a) d[a] = bc[a] - p[a];
            // J = [ [p]_x | -I ]
            const double J[3][6] = {{0.0, -p[2], p[1], -1.0, 0.0, 0.0},
                                    {p[2], 0.0, -p[0], 0.0, -1.0, 0.0},
                                    {-p[1], p[0], 0.0, 0.0, 0.0, -1.0}};
            double JtM[6][3];
            for (int u = 0; u < 6; ++u)
                for (int b = 0; b < 3; ++b) JtM[u][b] = J[0][u] * Mf[0][b] + J[1][u] * Mf[1][b] + J[2][u] * Mf[2][b];
            int q = 0;
            for (int u = 0; u < 6; ++u)
                for (int v = u; v < 6; ++v, ++q) acc[q] = JtM[u][0] * J[0][v] + JtM[u][1] * J[1][v] + JtM[u][2] * J[2][v];
            for (int u = 0; u < 6; ++u) acc[21 + u] = JtM[u][0] * d[0] + JtM[u][1] * d[1] + JtM[u][2] * d[2];
            double Md[3];
            for (int a = 0; a < 3; ++a) Md[a] = Mf[a][0] * d[0] + Mf[a][1] * d[1] + Mf[a][2] * d[2];
            acc[27] = d[0] * Md[0] + d[1] * Md[1] + d[2] * Md[2];
            acc[28] = 1.0;
        }
    }
    // fixed-order sums: warps, then the CTA's warps in order
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int q = 0; q < NACC; ++q) {
        const double v = warp_sum(acc[q]);
        if (lane == 0) wsum[w][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < NACC) {
        double v = 0.0;
        for (int j = 0; j < GT / 32; ++j) v += wsum[j][threadIdx.x];
        partial[(int64_t)blockIdx.x * NACC + threadIdx.x] = v;
    }
}

// the CTAs' partial sums: warp q adds value q, lane l the CTAs l, l + 32, ...,
// then the lanes in a fixed tree (deterministic)
__global__ void __launch_bounds__(NACC * 32) reduce_partials_kernel(const double* __restrict__ partial, int nblk,
                                                                   double* __restrict__ out)
{
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v = 0.0;
    for (int b = lane; b < nblk; b += 32) v += partial[(int64_t)b * NACC + q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) out[q] = v;
}

// 6 x 6 solve H x = -g by Cholesky (H symmetric positive definite); false if not
bool solve6(const double H[36], const double g[6], double x[6])
{
    double Lm[36] = {0};
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = H[6 * i + j];
            for (int q = 0; q < j; ++q) s -= Lm[6 * i + q] * Lm[6 * j + q];
            if (i == j) {
                if (!(s > 0.0)) return false;
                Lm[6 * i + i] = std::sqrt(s);
            } else {
                Lm[6 * i + j] = s / Lm[6 * j + j];
            }
        }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = -g[i];
        for (int q = 0; q < i; ++q) s -= Lm[6 * i + q] * y[q];
        y[i] = s / Lm[6 * i + i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int q = i + 1; q < 6; ++q) s -= Lm[6 * q + i] * x[q];
        x[i] = s / Lm[6 * i + i];
    }
    return true;
}

void exp_so3(const double w[3], double E[9])
{
    const double th = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    const double K[9] = {0.0, -w[2], w[1], w[2], 0.0, -w[0], -w[1], w[0], 0.0};
    double K2[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) K2[3 * a + b] = K[3 * a] * K[b] + K[3 * a + 1] * K[3 + b] + K[3 * a + 2] * K[6 + b];
    const double A = th < 1e-12 ? 1.0 : std::sin(th) / th;
    const double B = th < 1e-12 ? 0.0 : (1.0 - std::cos(th)) / (th * th);
    for (int q = 0; q < 9; ++q) E[q] = (q % 4 == 0 ? 1.0 : 0.0) + A * K[q] + B * K2[q];
}

// device buffers of one registration
struct GicpBufs {
    cudaStream_t st;
    float* xyz = nullptr;
    double* Cs = nullptr;
    double* partial = nullptr;
    double* out = nullptr;
    int32_t* vox = nullptr;
    uint8_t* found = nullptr;
    ~GicpBufs()
    {
        for (void* q : {(void*)xyz, (void*)Cs, (void*)partial, (void*)out, (void*)vox, (void*)found})
            if (q) cudaFreeAsync(q, st);
    }
};

struct Params {
    double r, tau, rho, eps, eps_rot, eps_trans;
    int max_iters;
};

}  // namespace
}  // namespace bbs

// the GICP target (opaque to callers)
struct bbs_gicp_target {
    int device;
    float r;
    bbs::GicpSlot* slots;
    double* cov;        // per voxel: the shape of C_t (6 doubles)
    int64_t T;          // slots, a power of two
    int log2T;
    int32_t maxp;       // longest probe of any voxel
    int64_t n_voxels;
};

namespace bbs {
namespace {

TargetView view_of(const bbs_gicp_target* t)
{
    TargetView v;
    v.slots = t->slots;
    v.cov = t->cov;
    v.shift = (uint32_t)(32 - t->log2T);
    v.mask = (uint32_t)(t->T - 1);
    v.maxp = t->maxp;
    v.pad = 0;
    v.r = (double)t->r;
    return v;
}

int params_of(const bbs_gicp_target* t, const bbs_gicp_opts* o, Params* p)
{
    p->r = (double)t->r;
    p->tau = (o && o->tau > 0.0) ? o->tau : p->r;
    p->rho = (o && o->rho > 0.0) ? o->rho : 2.0 * p->r;
    p->eps = (o && o->cov_eps > 0.0) ? o->cov_eps : 1e-3;
    p->eps_rot = (o && o->eps_rot > 0.0) ? o->eps_rot : 1e-6;
    p->eps_trans = (o && o->eps_trans > 0.0) ? o->eps_trans : 1e-6;
    p->max_iters = (o && o->max_iters > 0) ? o->max_iters : 30;
    if (!std::isfinite(p->tau) || !std::isfinite(p->rho) || !std::isfinite(p->eps))
        return set_error(BBS_EINVAL, "gicp: non-finite option");
    return BBS_OK;
}

// scan to the device, its covariances
int prepare(const float* xyz, int64_t k, int is_device, const Params& P, GicpBufs& B)
{
    if (!is_device) {
        BBS_CUDA_TRY(cudaMallocAsync((void**)&B.xyz, sizeof(float) * 3 * (size_t)k, B.st));
        BBS_CUDA_TRY(cudaMemcpyAsync(B.xyz, xyz, sizeof(float) * 3 * (size_t)k, cudaMemcpyHostToDevice, B.st));
    }
    const float* d_xyz = B.xyz ? B.xyz : xyz;
    const int nblk = (int)((k + GT - 1) / GT);
    BBS_CUDA_TRY(cudaMallocAsync((void**)&B.Cs, sizeof(double) * 6 * (size_t)k, B.st));
    BBS_CUDA_TRY(cudaMallocAsync((void**)&B.partial, sizeof(double) * NACC * (size_t)nblk, B.st));
    BBS_CUDA_TRY(cudaMallocAsync((void**)&B.out, sizeof(double) * NACC, B.st));
    const double rho2 = P.rho * P.rho;
    source_cov_kernel<<<(unsigned)((k * 32 + 255) / 256), 256, 0, B.st>>>(d_xyz, k, rho2, (float)(rho2 * (1.0 + 1e-5)),
                                                                       P.r, P.eps, B.Cs);
    BBS_CUDA_TRY(cudaGetLastError());
    return BBS_OK;
}

int linearize_once(const bbs_gicp_target* tg, const float* d_xyz, int64_t k, const Params& P, const Pose& T,
                   GicpBufs& B, double H[36], double g[6], double* cost, int64_t* n, bool want_vox)
{
    const int nblk = (int)((k + GT - 1) / GT);
    linearize_kernel<<<nblk, GT, 0, B.st>>>(view_of(tg), d_xyz, B.Cs, k, T, P.r, P.tau * P.tau, P.eps, B.partial,
                                            want_vox ? B.vox : nullptr, want_vox ? B.found : nullptr);
    reduce_partials_kernel<<<1, NACC * 32, 0, B.st>>>(B.partial, nblk, B.out);
    BBS_CUDA_TRY(cudaGetLastError());
    double acc[NACC];
    BBS_CUDA_TRY(cudaMemcpyAsync(acc, B.out, sizeof(acc), cudaMemcpyDeviceToHost, B.st));
    BBS_CUDA_TRY(cudaStreamSynchronize(B.st));
    int q = 0;
    for (int u = 0; u < 6; ++u)
        for (int v = u; v < 6; ++v, ++q) H[6 * u + v] = H[6 * v + u] = acc[q];
    for (int u = 0; u < 6; ++u) g[u] = acc[21 + u];
    *cost = acc[27];
    *n = (int64_t)acc[28];
    return BBS_OK;
}

int check_args(const bbs_gicp_target* t, const float* xyz, int64_t k)
{
    if (!t) return set_error(BBS_EINVAL, "gicp: NULL target");
    if (k < 1 || !xyz) return set_error(BBS_EINVAL, "gicp: empty scan");
    if (k > ((int64_t)1 << 26)) return set_error(BBS_EINVAL, "gicp: more than 2^26 scan points");
    return BBS_OK;
}

int log2_ceil64(int64_t x)
{
    int l = 0;
    while (((int64_t)1 << l) < x) ++l;
    return l;
}

}  // namespace

int gicp_target_device(const bbs_gicp_target* t) { return t->device; }

void gicp_target_free(bbs_gicp_target* t)
{
    if (t->slots) cudaFree(t->slots);
    if (t->cov) cudaFree(t->cov);
    delete t;
}

int gicp_target_info(const bbs_gicp_target* t, int64_t* n_voxels, int64_t* table_size, int32_t* max_probe)
{
    if (n_voxels) *n_voxels = t->n_voxels;
    if (table_size) *table_size = t->T;
    if (max_probe) *max_probe = t->maxp;
    return BBS_OK;
}

int gicp_target_build(const float* xyz, int64_t n, int is_device, float r, cudaStream_t st, bbs_gicp_target** out)
{
    *out = nullptr;
    if (!(r > 0.0f) || !std::isfinite(r)) return set_error(BBS_EINVAL, "gicp_target: r must be positive and finite");
    if (n < 1 || !xyz) return set_error(BBS_EINVAL, "gicp_target: empty cloud");
    const float* d_xyz = xyz;
    float* owned = nullptr;
    int* d_st = nullptr;
    BBS_CUDA_TRY(cudaMallocAsync((void**)&d_st, sizeof(int) * 4, st));
    if (!is_device) {
        if (cudaMallocAsync((void**)&owned, sizeof(float) * 3 * (size_t)n, st) != cudaSuccess ||
            cudaMemcpyAsync(owned, xyz, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            if (owned) cudaFreeAsync(owned, st);
            cudaFreeAsync(d_st, st);
            return set_error(BBS_ENOMEM, "gicp_target: %lld points", (long long)n);
        }
        d_xyz = owned;
    }
    bbs_gicp_target* t = new bbs_gicp_target;
    std::memset(t, 0, sizeof(*t));
    cudaGetDevice(&t->device);
    t->r = r;
    const float rho = (float)(1.0 / (double)r);
    // half the points' count in slots (maps hold several points per voxel), doubled
    // while a probe runs past 64 slots
    int lt = std::max(10, log2_ceil64((n + 1) / 2));
    int rc = BBS_OK;
    for (;; lt += 1) {
        if (lt > 31) {
            rc = set_error(BBS_ENOMEM, "gicp_target: table beyond 2^31 slots");
            break;
        }
        const int64_t T = (int64_t)1 << lt;
        if (t->slots) cudaFree(t->slots);
        t->slots = nullptr;
        if (cudaMalloc((void**)&t->slots, sizeof(GicpSlot) * (size_t)T) != cudaSuccess) {
            rc = set_error(BBS_ENOMEM, "gicp_target: %lld slots", (long long)T);
            break;
        }
        const int blocks = (int)std::min<int64_t>((T + 255) / 256, 8192);
        target_clear_kernel<<<blocks, 256, 0, st>>>(t->slots, T);
        cudaMemsetAsync(d_st, 0, sizeof(int) * 4, st);
        const int pblocks = (int)std::min<int64_t>((n + 255) / 256, 8192);
        target_insert_kernel<<<pblocks, 256, 0, st>>>(d_xyz, n, rho, (double)r, t->slots, (uint32_t)(32 - lt),
                                                      (uint32_t)(T - 1), 64, d_st);
        int hs[4];
        if (cudaGetLastError() != cudaSuccess || cudaMemcpyAsync(hs, d_st, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = set_error(BBS_ECUDA, "gicp_target: build failed");
            break;
        }
        if (hs[1]) {
            rc = set_error(BBS_EKEYRANGE, "gicp_target: a point is not finite or its key exceeds 2^20 voxels");
            break;
        }
        if (hs[0]) continue;   // a probe ran past 64 slots: a larger table
        target_centroid_kernel<<<blocks, 256, 0, st>>>(t->slots, T, (double)r);
        t->T = T;
        t->log2T = lt;
        t->maxp = hs[2];
        t->n_voxels = hs[3];
        // every voxel's covariance shape, from the final centroids
        const int64_t nv = std::max<int64_t>(t->n_voxels, 1);
        int64_t* row_slot = nullptr;
        if (cudaMalloc((void**)&t->cov, sizeof(double) * 6 * (size_t)nv) != cudaSuccess ||
            cudaMallocAsync((void**)&row_slot, sizeof(int64_t) * (size_t)nv, st) != cudaSuccess) {
            rc = set_error(BBS_ENOMEM, "gicp_target: covariance rows");
            break;
        }
        cudaMemsetAsync(d_st, 0, sizeof(int) * 4, st);
        target_rows_kernel<<<blocks, 256, 0, st>>>(t->slots, T, (unsigned long long*)d_st, row_slot);
        target_cov_kernel<<<(unsigned)std::min<int64_t>((t->n_voxels + 255) / 256 + 1, 65535), 256, 0, st>>>(
            view_of(t), row_slot, t->n_voxels, t->cov);
        cudaFreeAsync(row_slot, st);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
            rc = set_error(BBS_ECUDA, "gicp_target: centroids or covariances failed");
            break;
        }
        break;
    }
    cudaFreeAsync(d_st, st);
    if (owned) cudaFreeAsync(owned, st);
    if (rc < 0) {
        gicp_target_free(t);
        return rc;
    }
    *out = t;
    return BBS_OK;
}

int gicp_linearize(const bbs_gicp_target* tg, const float* xyz, int64_t k, int is_device, const double R[9],
                   const double t[3], const bbs_gicp_opts* o, double H[36], double g[6], double* cost, int64_t* n,
                   int32_t* vox, uint8_t* found)
{
    BBS_TRY(check_args(tg, xyz, k));
    Params P;
    BBS_TRY(params_of(tg, o, &P));
    GicpBufs B;
    B.st = o ? (cudaStream_t)o->cuda_stream : (cudaStream_t)0;
    BBS_TRY(prepare(xyz, k, is_device, P, B));
    const float* d_xyz = B.xyz ? B.xyz : xyz;
    const bool want = vox && found;
    if (want) {
        BBS_CUDA_TRY(cudaMallocAsync((void**)&B.vox, sizeof(int32_t) * 3 * (size_t)k, B.st));
        BBS_CUDA_TRY(cudaMallocAsync((void**)&B.found, (size_t)k, B.st));
    }
    Pose T;
    std::memcpy(T.R, R, sizeof(T.R));
    std::memcpy(T.t, t, sizeof(T.t));
    BBS_TRY(linearize_once(tg, d_xyz, k, P, T, B, H, g, cost, n, want));
    if (want) {
        BBS_CUDA_TRY(cudaMemcpyAsync(vox, B.vox, sizeof(int32_t) * 3 * (size_t)k, cudaMemcpyDeviceToHost, B.st));
        BBS_CUDA_TRY(cudaMemcpyAsync(found, B.found, (size_t)k, cudaMemcpyDeviceToHost, B.st));
        BBS_CUDA_TRY(cudaStreamSynchronize(B.st));
    }
    return BBS_OK;
}

int gicp_run(const bbs_gicp_target* tg, const float* xyz, int64_t k, int is_device, const double R0[9],
             const double t0[3], const bbs_gicp_opts* o, bbs_gicp_result* res)
{
    std::memset(res, 0, sizeof(*res));
    const auto c0 = std::chrono::steady_clock::now();
    BBS_TRY(res->status = check_args(tg, xyz, k));
    Params P;
    BBS_TRY(res->status = params_of(tg, o, &P));
    GicpBufs B;
    B.st = o ? (cudaStream_t)o->cuda_stream : (cudaStream_t)0;
    BBS_TRY(res->status = prepare(xyz, k, is_device, P, B));
    const float* d_xyz = B.xyz ? B.xyz : xyz;
    Pose T;
    std::memcpy(T.R, R0, sizeof(T.R));
    std::memcpy(T.t, t0, sizeof(T.t));
    for (int it = 1; it <= P.max_iters; ++it) {
        double H[36], g[6], cost;
        int64_t n;
        BBS_TRY(res->status = linearize_once(tg, d_xyz, k, P, T, B, H, g, &cost, &n, false));
        res->iterations = it;
        res->cost = cost;
        res->correspondences = (int32_t)n;
        if (n < 6) break;   // too few correspondences to fix six parameters
        double x[6];
        if (!solve6(H, g, x)) break;
        double E[9];
        exp_so3(x, E);
        Pose U;
        for (int a = 0; a < 3; ++a) {
            for (int b = 0; b < 3; ++b)
                U.R[3 * a + b] = E[3 * a] * T.R[b] + E[3 * a + 1] * T.R[3 + b] + E[3 * a + 2] * T.R[6 + b];
            U.t[a] = E[3 * a] * T.t[0] + E[3 * a + 1] * T.t[1] + E[3 * a + 2] * T.t[2] + x[3 + a];
        }
        T = U;
        const double nw = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
        const double nv = std::sqrt(x[3] * x[3] + x[4] * x[4] + x[5] * x[5]);
        if (nw < P.eps_rot && nv < P.eps_trans) {
            res->converged = 1;
            break;
        }
    }
    std::memcpy(res->R, T.R, sizeof(T.R));
    std::memcpy(res->t, T.t, sizeof(T.t));
    res->pose[0] = T.t[0];
    res->pose[1] = T.t[1];
    res->pose[2] = T.t[2];
    res->pose[5] = std::atan2(T.R[3], T.R[0]);
    res->pose[4] = -std::asin(std::fmax(-1.0, std::fmin(1.0, T.R[6])));
    res->pose[3] = std::atan2(T.R[7], T.R[8]);
    res->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - c0).count();
    return res->status = BBS_OK;
}

}  // namespace bbs
