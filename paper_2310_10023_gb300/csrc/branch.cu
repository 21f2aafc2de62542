// branch.cu -- fused branch-and-score kernel (Eq. (13) children, Eq. (11)
// scores) and the survivor pass of the search.
//
// Work unit: (parent, chunk of PCHUNK scan points).  A CTA stages its chunk of
// the scan in shared memory once, then walks the parent's rotational children
// (the "tasks"); for each task every thread rotates its points (FP32, fixed
// order, no FMA), floors them exactly, and makes ONE brick probe per point
// that answers all 8 translational children 2c + j (Sec. III-C layout, see
// bbs_internal.cuh).  The 8 child counts are kept as two byte-packed
// registers (4 counts each), reduced per warp with redux.sync on 16-bit
// fields, summed across warps through double-buffered shared memory (one
// barrier per task), and added to a dense (parent, task, child) score array.
// The survivor pass then keeps children scoring above their search's best.
#include "branch.cuh"

namespace bbs {

namespace {

// bits {0, 1, 5, 6} of w (children jx + 5 jy of one z-plane) into bytes 0..3
__device__ __forceinline__ uint32_t spread4(uint32_t w) { return ((w & 0x63u) * 0x40881u) & 0x01010101u; }

// Paired FP32 arithmetic (sm_100+ f32x2): each lane of a pair is an IEEE
// FP32 operation with its own rounding, exactly the scalar result, two points
// per instruction.
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk2(float a, float b)
{
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void up2(f2 v, int32_t& a, int32_t& b) { asm("mov.b64 {%0, %1}, %2;" : "=r"(a), "=r"(b) : "l"(v)); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b)
{
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b)
{
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 add2rm(f2 a, f2 b)
{
    f2 d;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

struct Row2 {
    f2 x, y, z;
};

// ((a0 x + a1 y) + a2 z) for two points, the scalar order and rounding
__device__ __forceinline__ f2 rot2(const Row2& r, f2 X, f2 Y, f2 Z) { return add2(add2(mul2(r.x, X), mul2(r.y, Y)), mul2(r.z, Z)); }

// the 8 child bits of one point: key block at (kx, ky, kz) + {0,1}^3, where the
// keys are relative to the compact origin (COMPACT) or absolute (wide)
template <bool COMPACT>
__device__ __forceinline__ void child_bits(const LevelView& L, int32_t kx, int32_t ky, int32_t kz, uint32_t& w0,
                                           uint32_t& w1)
{
    w0 = w1 = 0;
    if (COMPACT) {
        const uint32_t rx = (uint32_t)kx, ry = (uint32_t)ky, rz = (uint32_t)kz;
        if (rx > L.rmax[0] || ry > L.rmax[1] || rz > L.rmax[2]) return;
        const uint32_t oz = rz & 3u;
        uint4 w;
        if (!probe_compact(L, cbrick_pack(rx >> 2, ry >> 2, rz >> 2), (int)(oz >> 1), w)) return;
        const uint32_t sh = (rx & 3u) + 5u * (ry & 3u);
        w0 = ((oz & 1u) ? w.z : w.y) >> sh;
        w1 = ((oz & 1u) ? w.w : w.z) >> sh;
    } else {
        if (!(key_in_range(kx) && key_in_range(ky) && key_in_range(kz))) return;
        uint4 blo, bhi;
        if (!probe_brick(L, kx >> 2, ky >> 2, kz >> 2, blo, bhi)) return;
        const int oz = kz & 3, sh = (kx & 3) + 5 * (ky & 3);
        w0 = brick_plane(blo, bhi, oz) >> sh;
        w1 = brick_plane(blo, bhi, oz + 1) >> sh;
    }
}

// One task (rotational child) over the staged points, two points per step.
// The chunk is staged as pairs: sxy[j] = (x_2j, x_2j+1, y_2j, y_2j+1) and
// sz[j] = (z_2j, z_2j+1), so each coordinate pair is one 64-bit register for
// the f32x2 operations.  The exact floor of q is the bit pattern of
// fl_rd(q + 1.5 * 2^23) minus that of 1.5 * 2^23 (valid for |q| < 2^22); that
// offset is a multiple of 2^22, so the level shift applies to the raw bit
// pattern and the offset, the translation and the compact origin fold into
// one per-axis constant.
template <bool COMPACT>
__device__ __forceinline__ void score_task(const ulonglong2* sxy, const f2* sz, int n, const LevelView& L, int m,
                                           const Row2& r0, const Row2& r1, const Row2& r2, int32_t cx, int32_t cy,
                                           int32_t cz, uint32_t& acc0, uint32_t& acc1)
{
    const f2 C = pk2(12582912.0f, 12582912.0f);
    const int np = (n + 1) >> 1;
    for (int j = threadIdx.x; j < np; j += blockDim.x) {
        const ulonglong2 xy = sxy[j];
        const f2 Z = sz[j];
        int32_t bx1, bx2, by1, by2, bz1, bz2;
        up2(add2rm(rot2(r0, xy.x, xy.y, Z), C), bx1, bx2);
        up2(add2rm(rot2(r1, xy.x, xy.y, Z), C), by1, by2);
        up2(add2rm(rot2(r2, xy.x, xy.y, Z), C), bz1, bz2);
        uint32_t w0, w1;
        child_bits<COMPACT>(L, (bx1 >> m) + cx, (by1 >> m) + cy, (bz1 >> m) + cz, w0, w1);
        acc0 += spread4(w0);
        acc1 += spread4(w1);
        if (2 * j + 1 < n) {
            child_bits<COMPACT>(L, (bx2 >> m) + cx, (by2 >> m) + cy, (bz2 >> m) + cz, w0, w1);
            acc0 += spread4(w0);
            acc1 += spread4(w1);
        }
    }
}

__device__ __forceinline__ int find_seg(const Plan* P, int64_t w)
{
    int lo = 0, hi = P->nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P->seg[mid].first_work <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_dense_seg(const Plan* P, int64_t d)
{
    int lo = 0, hi = P->nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P->seg[mid].dense_base <= d) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// rotational-child ranges of a parent at level l (decoded from its rotation index)
__device__ __forceinline__ void parent_ranges(const DevGrid& g, int l, uint32_t prot, int32_t lo[3], int32_t ext[3])
{
    const int32_t ng = g.N[l][2], nb = g.N[l][1];
    const int32_t c[3] = {(int32_t)(prot / ((uint32_t)ng * (uint32_t)nb)), (int32_t)((prot / (uint32_t)ng) % (uint32_t)nb),
                          (int32_t)(prot % (uint32_t)ng)};
    for (int i = 0; i < 3; ++i) {
        int32_t a, b;
        child_range(g, l, i, c[i], a, b);
        lo[i] = a;
        ext[i] = b - a;
    }
}

}  // namespace

constexpr int TB = 64;   // tasks reduced per barrier round

template <int MODE>
__global__ void __launch_bounds__(256, 5) branch2_kernel(const Plan* __restrict__ P, const SearchDev* __restrict__ Sall,
                                                         const NodeRec* __restrict__ parents, int32_t* dense)
{
    if (P->status != PLAN_OK) return;
    const int64_t n_work = P->n_work;
    __shared__ ulonglong2 sxy[PCHUNK / 2];
    __shared__ f2 sz[PCHUNK / 2];
    __shared__ uint32_t red[TB][4];
    const int tid = threadIdx.x, lane = tid & 31;
    float* fxy = reinterpret_cast<float*>(sxy);
    float* fz = reinterpret_cast<float*>(sz);
    for (int64_t w = blockIdx.x; w < n_work; w += gridDim.x) {
        const Seg g = P->seg[find_seg(P, w)];
        const SearchDev& S = Sall[g.sid];
        const int64_t local = w - g.first_work;
        const int64_t pi = local / g.chunks;
        const int32_t k0 = (int32_t)(local - pi * g.chunks) * PCHUNK;
        const int32_t n = min(PCHUNK, S.K - k0);
        __syncthreads();   // the previous item's readers of the staged points are done
        for (int i = tid; i < n; i += blockDim.x) {
            const float4 p = __ldg(S.scan + k0 + i);
            const int j = i >> 1, h = i & 1;
            fxy[4 * j + h] = p.x;
            fxy[4 * j + 2 + h] = p.y;
            fz[2 * j + h] = p.z;
        }
        int m, T;
        int32_t tx, ty, tz;
        int32_t lo[3] = {0, 0, 0}, ext[3] = {1, 1, 1};
        if (MODE == MODE_INITIAL) {
            const int64_t vp = g.first_parent + pi;
            const int32_t pz = (int32_t)(vp % S.pext[2]);
            const int32_t py = (int32_t)((vp / S.pext[2]) % S.pext[1]);
            const int32_t px = (int32_t)(vp / ((int64_t)S.pext[2] * S.pext[1]));
            tx = 2 * (S.pmin[0] + px);
            ty = 2 * (S.pmin[1] + py);
            tz = 2 * (S.pmin[2] + pz);
            m = S.lmax;
            T = S.grid.N[m][0] * S.grid.N[m][1] * S.grid.N[m][2];
        } else {
            const NodeRec par = parents[g.first_parent + pi];
            const int l = rl_level(par.rl);
            m = l - 1;
            parent_ranges(S.grid, l, rl_rot(par.rl), lo, ext);
            T = m >= 0 ? ext[0] * ext[1] * ext[2] : 0;
            tx = 2 * par.cx;
            ty = 2 * par.cy;
            tz = 2 * par.cz;
        }
        if (m < 0) continue;   // uniform: a leaf has no children (staging reads nothing more)
        const LevelView Lv = S.maps[m];
        const int64_t roff = S.grid.rot_off[m];
        const int32_t Nb = S.grid.N[m][1], Ng = S.grid.N[m][2];
        const int32_t off = 0x4B400000 >> m;   // the floor offset after the level shift
        for (int t0 = 0; t0 < T; t0 += TB) {
            const int tb = min(TB, T - t0);
            for (int i = tid; i < 4 * TB; i += blockDim.x) (&red[0][0])[i] = 0u;
            __syncthreads();   // staged points and zeroed partials visible
            for (int tt = 0; tt < tb; ++tt) {
                const int t = t0 + tt;
                uint32_t crot;
                if (MODE == MODE_INITIAL) {
                    crot = (uint32_t)t;
                } else {
                    const int32_t ja = t / (ext[1] * ext[2]), jb = (t / ext[2]) % ext[1], jg = t % ext[2];
                    crot = (uint32_t)(((int64_t)(lo[0] + ja) * Nb + (lo[1] + jb)) * Ng + (lo[2] + jg));
                }
                const float4* A = S.rot + 3 * (roff + (int64_t)crot);
                const float4 a0 = __ldg(A), a1 = __ldg(A + 1), a2 = __ldg(A + 2);
                const Row2 r0{pk2(a0.x, a0.x), pk2(a0.y, a0.y), pk2(a0.z, a0.z)};
                const Row2 r1{pk2(a1.x, a1.x), pk2(a1.y, a1.y), pk2(a1.z, a1.z)};
                const Row2 r2{pk2(a2.x, a2.x), pk2(a2.y, a2.y), pk2(a2.z, a2.z)};
                uint32_t acc0 = 0, acc1 = 0;   // bytes: children (0,4,2,6) and (1,5,3,7)
                if (Lv.compact)
                    score_task<true>(sxy, sz, n, Lv, m, r0, r1, r2, tx - off - Lv.base[0], ty - off - Lv.base[1],
                                     tz - off - Lv.base[2], acc0, acc1);
                else
                    score_task<false>(sxy, sz, n, Lv, m, r0, r1, r2, tx - off, ty - off, tz - off, acc0, acc1);
                // 16-bit fields: at most 8 points per thread x 32 lanes, x 8 warps, per field
                uint32_t e0 = acc0 & 0x00FF00FFu, o0 = (acc0 >> 8) & 0x00FF00FFu;
                uint32_t e1 = acc1 & 0x00FF00FFu, o1 = (acc1 >> 8) & 0x00FF00FFu;
                e0 = __reduce_add_sync(0xffffffffu, e0);
                o0 = __reduce_add_sync(0xffffffffu, o0);
                e1 = __reduce_add_sync(0xffffffffu, e1);
                o1 = __reduce_add_sync(0xffffffffu, o1);
                if (lane == 0) {
                    atomicAdd(&red[tt][0], e0);
                    atomicAdd(&red[tt][1], o0);
                    atomicAdd(&red[tt][2], e1);
                    atomicAdd(&red[tt][3], o1);
                }
            }
            __syncthreads();   // every warp's partial sums are in
            for (int i = tid; i < 8 * tb; i += blockDim.x) {
                // child j = 4 jx + 2 jy + jz of task tt: word (jz ? 2 : 0) + jx, half jy
                const int tt = i >> 3, j = i & 7;
                const int jx = j >> 2, jy = (j >> 1) & 1, jz = j & 1;
                const uint32_t sum = red[tt][(jz ? 2 : 0) + jx];
                const uint32_t cnt = jy ? (sum >> 16) : (sum & 0xFFFFu);
                if (cnt) atomicAdd(&dense[g.dense_base + (pi * g.R + t0 + tt) * 8 + j], (int32_t)cnt);
            }
            __syncthreads();   // the partials are read before the next round zeroes them
        }
    }
}

// survivors: children scoring above their search's best, staged with per-score
// histograms (count, children, leaves) for the frontier insertion
template <int MODE>
__global__ void __launch_bounds__(256) finalize_kernel(const Plan* __restrict__ P, SearchDev* S,
                                                       const NodeRec* __restrict__ parents, int32_t* dense, SurvOut out)
{
    if (P->status != PLAN_OK) return;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_dense = P->n_dense;
    const int64_t n_round = (n_dense + 31) & ~(int64_t)31;
    for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < n_round; d += stride) {
        bool surv = false;
        int32_t score = 0, sid = 0;
        NodeRec nd;
        nd.cx = nd.cy = nd.cz = 0;
        nd.rl = 0;
        int m = 0;
        uint32_t crot = 0;
        if (d < n_dense) {
            const Seg g = P->seg[find_dense_seg(P, d)];
            sid = g.sid;
            const SearchDev& s = S[sid];
            const int64_t local = d - g.dense_base;
            const int64_t per = (int64_t)g.R * 8;
            const int64_t pi = local / per;
            const int32_t rem = (int32_t)(local - pi * per);
            const int32_t t = rem >> 3, j = rem & 7;
            bool valid = pi < g.n_parents;
            int32_t tx = 0, ty = 0, tz = 0;
            if (valid && MODE == MODE_INITIAL) {
                const int64_t vp = g.first_parent + pi;
                const int32_t pz = (int32_t)(vp % s.pext[2]);
                const int32_t py = (int32_t)((vp / s.pext[2]) % s.pext[1]);
                const int32_t px = (int32_t)(vp / ((int64_t)s.pext[2] * s.pext[1]));
                tx = 2 * (s.pmin[0] + px) + (j >> 2);
                ty = 2 * (s.pmin[1] + py) + ((j >> 1) & 1);
                tz = 2 * (s.pmin[2] + pz) + (j & 1);
                valid = tx >= s.wmin[0] && tx <= s.wmax[0] && ty >= s.wmin[1] && ty <= s.wmax[1] && tz >= s.wmin[2] &&
                        tz <= s.wmax[2];
                m = s.lmax;
                crot = (uint32_t)t;
            } else if (valid) {
                const NodeRec par = parents[g.first_parent + pi];
                const int l = rl_level(par.rl);
                m = l - 1;
                int32_t lo[3], ext[3];
                parent_ranges(s.grid, l, rl_rot(par.rl), lo, ext);
                valid = m >= 0 && t < ext[0] * ext[1] * ext[2];
                if (valid) {
                    const int32_t ja = t / (ext[1] * ext[2]), jb = (t / ext[2]) % ext[1], jg = t % ext[2];
                    crot = (uint32_t)(((int64_t)(lo[0] + ja) * s.grid.N[m][1] + (lo[1] + jb)) * s.grid.N[m][2] +
                                      (lo[2] + jg));
                    tx = 2 * par.cx + (j >> 2);
                    ty = 2 * par.cy + ((j >> 1) & 1);
                    tz = 2 * par.cz + (j & 1);
                }
            }
            // the dense array must be zero for the next round: consume it
            const int32_t dv = dense[d];
            if (dv) dense[d] = 0;
            if (valid) {
                score = dv;
                surv = score > s.ctl->best;
                nd.cx = tx;
                nd.cy = ty;
                nd.cz = tz;
                nd.rl = rl_pack(crot, m);
            }
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, surv);
        if (!ball) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(out.count, (unsigned long long)__popc(ball));
        base = __shfl_sync(0xffffffffu, base, 0);
        const uint32_t key = surv ? (((uint32_t)sid << 24) | (uint32_t)score) : 0xFFFFFFFFu;
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        if (surv) {
            const unsigned long long pos = base + __popc(ball & ((1u << lane) - 1u));
            if (pos < (unsigned long long)out.cap) {
                out.nodes[pos] = nd;
                out.scores[pos] = score;
                out.sid[pos] = sid;
            } else {
                atomicOr(out.err, 2);
            }
            SearchDev& s = S[sid];
            if ((__ffs(peers) - 1) == lane) atomicAdd(&s.h_cnt[score], (uint32_t)__popc(peers));
            atomicAdd(&s.h_kids[score], (unsigned long long)node_children(s.grid, m, crot));
            if (m == 0) atomicAdd(&s.h_leaf[score], 1u);
        }
    }
}

cudaError_t launch_branch(int mode, const Plan* P, const SearchDev* S, const NodeRec* parents, int32_t* dense,
                          int blocks, cudaStream_t st)
{
    if (blocks <= 0) return cudaSuccess;
    if (mode == MODE_INITIAL) branch2_kernel<MODE_INITIAL><<<blocks, 256, 0, st>>>(P, S, parents, dense);
    else branch2_kernel<MODE_SEARCH><<<blocks, 256, 0, st>>>(P, S, parents, dense);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int mode, const Plan* P, SearchDev* S, const NodeRec* parents, int32_t* dense,
                            const SurvOut& out, int blocks, cudaStream_t st)
{
    if (blocks <= 0) return cudaSuccess;
    if (mode == MODE_INITIAL) finalize_kernel<MODE_INITIAL><<<blocks, 256, 0, st>>>(P, S, parents, dense, out);
    else finalize_kernel<MODE_SEARCH><<<blocks, 256, 0, st>>>(P, S, parents, dense, out);
    return cudaGetLastError();
}

}  // namespace bbs
