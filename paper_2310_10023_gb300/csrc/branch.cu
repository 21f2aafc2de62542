// branch.cu -- fused branch-and-score kernel (Eq. (13) children, Eq. (11)
// scores) and the survivor pass of the search.
//
// Work: every rotational child ("task") of every parent of a launch, over
// every point of its search's scan.  The launch's work is cut into slices
// (task, block of PBLK points) and each CTA of one resident wave takes an
// equal contiguous range of them, so the SMs finish together whatever the mix
// of parents.  For each task, every thread rotates its points (FP32, fixed
// order, no FMA), floors them exactly, and makes ONE brick probe per point
// that answers all 8 translational children 2c + j (Sec. III-C layout, see
// bbs_internal.cuh).  The 8 child counts are kept as two byte-packed
// registers (4 counts each), reduced per warp with redux.sync on 16-bit
// fields, summed across warps in shared memory, and added to a dense
// (task, child) score array.  The survivor pass then keeps children scoring
// above their search's best.
#include "branch.cuh"

namespace bbs {

namespace {

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
// fl_rd(a * b + c) per lane, one rounding of the exact value
__device__ __forceinline__ f2 fma2rm(f2 a, f2 b, f2 c)
{
    f2 d;
    asm("fma.rm.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

struct Row2 {
    f2 x, y, z;
};

// ((a0 x + a1 y) + a2 z) for two points, the scalar order and rounding
__device__ __forceinline__ f2 rot2(const Row2& r, f2 X, f2 Y, f2 Z) { return add2(add2(mul2(r.x, X), mul2(r.y, Y)), mul2(r.z, Z)); }

// Bit pattern of a floored key: for the per-axis constant C = 1.5 * 2^23 + d
// (d an integer, |d| < 2^21), fl_rd(q * 2^-m + C) rounds the exact value once,
// so while |floor(q / 2^m) + d| < 2^22 its bit pattern is KB + floor(q / 2^m) + d:
// the level-m key of Eq. (11), offset by d, in the low 22 bits.  Outside that
// range the pattern leaves [KB, KB + 2^22) and fails every range check below.
constexpr uint32_t KB = 0x4B400000u;   // bit pattern of 1.5 * 2^23

// the 8 child bits of one point from the bit patterns of its level-m key,
// offset so that the key block (kx, ky, kz) + {0,1}^3 is relative to the
// level's box origin (compact, dense) or absolute (wide)
template <int LAYOUT>
__device__ __forceinline__ void child_bits(const LevelView& L, uint32_t bx, uint32_t by, uint32_t bz, uint32_t& w0,
                                           uint32_t& w1)
{
    w0 = w1 = 0;
    if (LAYOUT == LAYOUT_DENSE) {
        // relative keys: a pattern outside [KB, KB + 2^22) differs from KB above
        // bit 21 and so exceeds every rmax (< 2^22)
        // (branch-free: a query outside the box reads the zero brick past it)
        const uint32_t rx = bx ^ KB, ry = by ^ KB, rz = bz ^ KB;
        const bool in = rx <= L.rmax[0] && ry <= L.rmax[1] && rz <= L.rmax[2];
        const uint32_t idx = in ? ((rx >> 2) * L.nby + (ry >> 2)) * L.nbz + (rz >> 2) : L.mask;
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(L.slots + idx) + ((rz >> 1) & 1u));
        const uint32_t sh = (rx & 3u) + 5u * (ry & 3u);
        w0 = ((rz & 1u) ? w.z : w.y) >> sh;
        w1 = ((rz & 1u) ? w.w : w.z) >> sh;
    } else if (LAYOUT == LAYOUT_COMPACT) {
        // relative keys in [0, 2^13) x [0, 2^13) x [0, 4092): 11 / 11 / 10-bit brick
        // fields that cannot overflow, and never the empty tag (brick z <= 1022);
        // bricks beyond the map's own box are simply absent
        if (((bx ^ KB) | (by ^ KB)) >= (1u << 13) || (bz ^ KB) >= 4092u) return;
        // brick key (rx >> 2) | (ry >> 2) << 11 | (rz >> 2) << 22 straight from the
        // patterns: KB is 0 in every bit that lands in a field
        const uint32_t key = ((bx >> 2) & 0x7FFu) | ((by << 9) & 0x3FF800u) | ((bz << 20) & 0xFFC00000u);
        uint4 w;
        if (!probe_compact(L, key, (int)((bz >> 1) & 1u), w)) return;
        const uint32_t sh = (bx & 3u) + 5u * (by & 3u);
        w0 = ((bz & 1u) ? w.z : w.y) >> sh;
        w1 = ((bz & 1u) ? w.w : w.z) >> sh;
    } else {
        const int32_t kx = (int32_t)(bx - KB), ky = (int32_t)(by - KB), kz = (int32_t)(bz - KB);
        if (!(key_in_range(kx) && key_in_range(ky) && key_in_range(kz))) return;
        uint4 blo, bhi;
        if (!probe_brick(L, kx >> 2, ky >> 2, kz >> 2, blo, bhi)) return;
        const int oz = kz & 3, sh = (kx & 3) + 5 * (ky & 3);
        w0 = brick_plane(blo, bhi, oz) >> sh;
        w1 = brick_plane(blo, bhi, oz + 1) >> sh;
    }
}

// Child counters: one 4-bit counter per translational child in one 32-bit
// word, child i = jx + 2 jy + 4 jz at bit 4 (jx + 2 jz) + 16 jy, so that
// (acc >> 4 k) & 0x000F000F holds the children (jx, jz) = (k & 1, k >> 1)
// with jy = 0 and jy = 1 in its two 16-bit halves.  A point adds
// CHILD_LUT[v] for its 8-bit child mask v (one shared-memory load and one
// add).  A scoring thread counts at most 10 points of a run (a run is at
// most PCHUNK points over 224 threads, two points per pair), so no counter
// passes 15.
__host__ __device__ constexpr uint32_t child_lut_entry(uint32_t v)
{
    return ((v & 1u) << 0) | (((v >> 1) & 1u) << 4) | (((v >> 2) & 1u) << 16) | (((v >> 3) & 1u) << 20) |
           (((v >> 4) & 1u) << 8) | (((v >> 5) & 1u) << 12) | (((v >> 6) & 1u) << 24) | (((v >> 7) & 1u) << 28);
}
// the scoring CTA: warps 0..6 score (NCONS threads), warp 7 describes the rounds
constexpr int NCONS = 224;
static_assert(2 * ((PCHUNK / 2 + NCONS - 1) / NCONS) <= 15, "4-bit child counters hold the points of one run per thread");

// The 8-bit child mask of one point from a byte grid (LAYOUT_BYTES): relative
// keys clamped to the empty key past the box, one byte load.
__device__ __forceinline__ uint32_t bytes_mask(const LevelView& L, uint32_t bx, uint32_t by, uint32_t bz, uint32_t ex,
                                               uint32_t ey, uint32_t ez)
{
    const uint32_t rx = min(bx ^ KB, ex), ry = min(by ^ KB, ey), rz = min(bz ^ KB, ez);
    return __ldg(reinterpret_cast<const uint8_t*>(L.slots) + ((rx * L.nby + ry) * L.nbz + rz));
}
// The same for a run whose every point is known to land inside the grid (the
// chunk-box test of the run): no per-axis clamp, and the -KB of the three
// patterns folded into one constant, cfix = -KB (ny nz + nz + 1) mod 2^32 --
// the index is exact because its true value is below 2^31.  One min against
// the last cell (L.mask) keeps every load inside the grid whatever the test.
__device__ __forceinline__ uint32_t bytes_mask_inside(const LevelView& L, uint32_t bx, uint32_t by, uint32_t bz,
                                                      uint32_t cfix)
{
    const uint32_t idx = min((bx * L.nby + by) * L.nbz + bz + cfix, L.mask);
    return __ldg(reinterpret_cast<const uint8_t*>(L.slots) + idx);
}
// the 8-bit child mask from the two plane words of the brick layouts
// (bits {0, 1, 5, 6}: children jx + 5 jy of the z = 0 and z = 1 planes)
__device__ __forceinline__ uint32_t planes_mask(uint32_t w0, uint32_t w1)
{
    return (w0 & 3u) | ((w0 >> 3) & 0xCu) | ((w1 & 3u) << 4) | ((w1 << 1) & 0xC0u);
}

// One run (a rotational child over blocks of the staged chunk), two points
// per step.  The chunk is staged as pairs: sxy[j] = (x_2j, x_2j+1, y_2j,
// y_2j+1) and sz[j] = (z_2j, z_2j+1), so each coordinate pair is one 64-bit
// register for the f32x2 operations; thread t of the nt scoring threads takes
// pairs jlo + t, jlo + t + nt, ... below jhi.  q = (A_i0 x + A_i1 y) + A_i2 z is rounded to FP32
// after every product and sum (no FMA), as the oracle; the floor, the level
// shift and the key offset are one fma.rm of that q (see KB).
template <int LAYOUT, bool INSIDE = false>
__device__ __forceinline__ void score_run(const ulonglong2* sxy, const f2* sz, int n, int jlo, int jhi,
                                          const LevelView& L, const Row2& r0, const Row2& r1, const Row2& r2, f2 S,
                                          f2 Cx, f2 Cy, f2 Cz, const uint32_t* lut, uint32_t& acc, int t, int nt)
{
    const uint32_t ex = L.rmax[0] + 1u, ey = L.rmax[1] + 1u, ez = L.rmax[2] + 1u;   // bytes: the empty key past the box
    const uint32_t cfix = 0u - KB * (L.nby * L.nbz + L.nbz + 1u);
    auto mask = [&](uint32_t bx, uint32_t by, uint32_t bz) -> uint32_t {
        if (LAYOUT == LAYOUT_BYTES && INSIDE) return bytes_mask_inside(L, bx, by, bz, cfix);
        if (LAYOUT == LAYOUT_BYTES) return bytes_mask(L, bx, by, bz, ex, ey, ez);
        uint32_t w0, w1;
        child_bits<LAYOUT>(L, bx, by, bz, w0, w1);
        return planes_mask(w0, w1);
    };
    auto pair = [&](int j) {
        const ulonglong2 xy = sxy[j];
        const f2 Z = sz[j];
        int32_t bx1, bx2, by1, by2, bz1, bz2;
        up2(fma2rm(rot2(r0, xy.x, xy.y, Z), S, Cx), bx1, bx2);
        up2(fma2rm(rot2(r1, xy.x, xy.y, Z), S, Cy), by1, by2);
        up2(fma2rm(rot2(r2, xy.x, xy.y, Z), S, Cz), bz1, bz2);
        acc += lut[mask((uint32_t)bx1, (uint32_t)by1, (uint32_t)bz1)];
        if (2 * j + 1 < n) acc += lut[mask((uint32_t)bx2, (uint32_t)by2, (uint32_t)bz2)];
    };
    int j = jlo + t;
    if (LAYOUT == LAYOUT_DENSE || LAYOUT == LAYOUT_BYTES)   // two pairs per step: four gathers in flight per thread
        for (; j + nt < jhi; j += 2 * nt) {
            pair(j);
            pair(j + nt);
        }
    for (; j < jhi; j += nt) pair(j);
}

// the segment holding launch-local slice w (segments in slice order)
__device__ __forceinline__ int find_slice_seg(const Plan* P, int64_t w)
{
    int lo = 0, hi = P->nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P->seg[mid].first_slice <= w) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// the segment holding launch-local task u (segments in task order)
__device__ __forceinline__ int find_task_seg(const Plan* P, int64_t u)
{
    int lo = 0, hi = P->nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P->seg[mid].first_task <= u) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// translation of virtual parent vp of the initial set (Eq. (3)-(5) window at l_max)
__device__ __forceinline__ void virtual_parent(const SearchDev& S, int64_t vp, int32_t& px, int32_t& py, int32_t& pz)
{
    pz = S.pmin[2] + (int32_t)(vp % S.pext[2]);
    py = S.pmin[1] + (int32_t)((vp / S.pext[2]) % S.pext[1]);
    px = S.pmin[0] + (int32_t)(vp / ((int64_t)S.pext[2] * S.pext[1]));
}

// Whether every point of run d lands inside its level's byte grid L.  The
// key of axis i is floor(q_i / 2^m) + o_i (o_i = t_i - base_i, the run's key
// offset) with q_i the FP32 value of sum_k A_ik x_k.  Over the chunk's box
// the exact sum lies in [lo, hi] (per term the smaller and larger of the
// corner products).  Here lo and hi are formed in FP32 (three products, two
// sums: within 3u / (1 - 3u) of mag = sum_k |A_ik| max |x_k|, u = 2^-24), and
// each point's FP32 q_i lies within as much again of its exact value, so
// widening by 2e-6 mag (which also covers the rounding of mag and of the
// widening) bounds every q_i.  Inside: every key in [0, rmax_i + 1].  A
// clamped offset (|o| = 2^21) never passes.  FP32 throughout: FP64 runs at a
// small fraction of the FP32 rate on this part.
template <typename RD>
__device__ __forceinline__ bool run_inside(const RD& d, const float4* __restrict__ box, const LevelView& L)
{
    const float4 blo = __ldg(box), bhi = __ldg(box + 1);
    const float lo3[3] = {blo.x, blo.y, blo.z}, hi3[3] = {bhi.x, bhi.y, bhi.z};
    const float s = __int_as_float((127 - d.m) << 23);   // 2^-m
    bool in = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float qlo = 0.0f, qhi = 0.0f, mag = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float a = __int_as_float((int)(uint32_t)d.a[3 * i + k]);
            const float p1 = __fmul_rn(a, lo3[k]), p2 = __fmul_rn(a, hi3[k]);
            qlo = __fadd_rn(qlo, fminf(p1, p2));
            qhi = __fadd_rn(qhi, fmaxf(p1, p2));
            mag = __fadd_rn(mag, __fmul_rn(fabsf(a), fmaxf(fabsf(lo3[k]), fabsf(hi3[k]))));
        }
        const float marg = __fadd_rn(__fmul_rn(2e-6f, mag), 1e-30f);
        const float o = __int_as_float((int)(uint32_t)d.kc[i]) - 12582912.0f;
        in = in && floorf(__fmul_rn(__fsub_rn(qlo, marg), s)) + o >= 0.0f &&
             floorf(__fmul_rn(__fadd_rn(qhi, marg), s)) + o <= (float)L.rmax[i] + 1.0f;
    }
    return in;
}

// A run: one task over blocks [b0, b1) of point chunk c, described in shared
// memory for the whole CTA.
struct __align__(16) RunDesc {
    f2 a[9];          // rotation entries A_ik, each duplicated for the paired lanes
    f2 kc[3];         // per-axis 1.5 * 2^23 + translation (- box origin), paired
    f2 s;             // 2^-m, paired
    int32_t m;        // child level
    int32_t c;        // point chunk
    int32_t b0, b1;   // PBLK-point blocks [b0, b1) of the chunk
    int32_t sid;      // search
    int32_t inside;   // every point of the run lands inside the level's byte grid
    int64_t task;     // launch-local task index
};

constexpr int NRUN = 32;   // runs described per round of a CTA

}  // namespace

// The rotation rows (A = fl32(R / r)) of one run's task, from its rl, into
// the run's descriptor (kept out of line: the scoring loop keeps its
// registers; the describing warp forms one run per lane).  FP32 double-float
// arithmetic gives the rows' exact bits but for rare entries near a rounding
// boundary (or out of its range), which take the FP64 formation.
__device__ __noinline__ void run_rows(RunDesc& d, uint32_t rl, const SearchDev& S)
{
    float A[9];
    search_rows(S.cs, S.grid, rl_level(rl), rl_rot(rl), A);
#pragma unroll
    for (int e = 0; e < 9; ++e) d.a[e] = pk2(A[e], A[e]);
}

// named barriers of the scoring CTA (0 is __syncthreads): the describing
// warp fills round buffer b and arrives on FULL + b; the scoring warps wait
// there, score, and arrive on EMPTY + b when they no longer read the buffer;
// CONS synchronizes the scoring warps alone
constexpr int BAR_FULL = 1, BAR_EMPTY = 3, BAR_CONS = 5;
constexpr int64_t SMALL_LAUNCH = 256;   // slices per CTA below which a launch is split statically
__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void bar_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// The CTA's static range [cur, end) of the launch's slices: the first
// static_pm / 1000 of them in equal shares, the rest handed out later in
// shrinking grabs.  A launch of fewer than SMALL_LAUNCH slices per CTA (about
// one round each) is split statically: there a grab's round costs more than
// the balance it buys (measured, indoor).
__device__ __forceinline__ int64_t static_slices(const Plan* P, int64_t n_slices)
{
    return n_slices < SMALL_LAUNCH * (int64_t)gridDim.x ? n_slices : n_slices * P->static_pm / 1000;
}

// The search and point chunk of slice x (false when its segment is empty):
// the chunk the CTA's first run reads
__device__ __forceinline__ bool slice_chunk(const Plan* P, int64_t x, int32_t& sid, int32_t& c)
{
    const Seg& g = P->seg[find_slice_seg(P, x)];
    if (g.n_tasks <= 0 || x < g.first_slice || x >= g.first_slice + g.n_tasks * g.nblk) return false;
    const int64_t cc = (x - g.first_slice) / (4 * g.n_tasks);
    const int nchunk = (g.nblk + 3) >> 2;
    sid = g.sid;
    c = (int32_t)(cc < nchunk - 1 ? cc : nchunk - 1);
    return true;
}

// The describing warp of a scoring CTA (out of line: its registers and its
// FP64 row formation stay out of the scoring warps' allocation).
template <int MODE>
__device__ __noinline__ void describe_rounds(Plan* __restrict__ P, const SearchDev* __restrict__ Sall,
                                             const TaskRec* __restrict__ tasks, RunDesc (*rd)[NRUN], int32_t* s_nrun,
                                             int64_t n_slices)
{
    const int lane = threadIdx.x & 31;
    // the static range first, then grabs of at least grab_min as CTAs finish
    const int64_t n_static = static_slices(P, n_slices);
    const int64_t grab_min = P->grab_min > 0 ? P->grab_min : 1;
    int64_t cur = n_static * blockIdx.x / gridDim.x, end = n_static * (blockIdx.x + 1) / gridDim.x;
    int gi = -1;
    int round = 0;
    for (;; ++round) {
        const int b = round & 1;
        if (round >= 2) bar_sync(BAR_EMPTY + b, 256);   // the scoring warps are done with buffer b
        if (cur >= end) {   // this range is done: take the next grab
            unsigned long long got = 0, want = 0;
            if (lane == 0) {
                const unsigned long long seen = *(volatile unsigned long long*)&P->next_slice;
                const int64_t left = n_slices - n_static - (int64_t)seen;
                int64_t w = left / (2 * (int64_t)gridDim.x);
                if (w < grab_min) w = grab_min;
                want = (unsigned long long)w;
                got = (unsigned long long)n_static + atomicAdd(&P->next_slice, want);
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            want = __shfl_sync(0xffffffffu, want, 0);
            cur = (int64_t)got;
            end = min((int64_t)(got + want), n_slices);
            gi = -1;
        }
        if (cur >= end) {   // every slice is handed out: the scoring warps stop
            if (lane == 0) s_nrun[b] = 0;
            __syncwarp();
            bar_arrive(BAR_FULL + b, 256);
            if (round >= 1) bar_sync(BAR_EMPTY + (b ^ 1), 256);   // the last round's release
            break;
        }
        if (gi < 0) gi = find_slice_seg(P, cur);
        const Seg* g = &P->seg[gi];
        int64_t seg_end = g->first_slice + g->n_tasks * g->nblk;
        while (cur >= seg_end) {   // the range continues in a later segment
            g = &P->seg[++gi];
            seg_end = g->first_slice + g->n_tasks * g->nblk;
        }
        const int64_t nt = g->n_tasks;
        const int nchunk = (g->nblk + 3) >> 2;
        const int nbl = g->nblk - 4 * (nchunk - 1);   // blocks of the last chunk
        // seg-relative slices: chunk c holds tasks 0..nt-1 of nbc(c) blocks each
        const int64_t x0 = cur - g->first_slice, xh = min(end, seg_end) - g->first_slice;
        auto tc_of = [&](int64_t x) -> int64_t {   // (chunk * nt + task) of slice x
            int64_t c = x / (4 * nt);
            if (c > nchunk - 1) c = nchunk - 1;
            const int nbc = c < nchunk - 1 ? 4 : nbl;
            return c * nt + (x - c * 4 * nt) / nbc;
        };
        auto tc_first = [&](int64_t v) -> int64_t {   // first slice of (chunk * nt + task) v
            const int64_t c = v / nt;
            const int nbc = c < nchunk - 1 ? 4 : nbl;
            return c * 4 * nt + (v - c * nt) * nbc;
        };
        const int64_t v0 = tc_of(x0), vh = tc_of(xh - 1);
        const int nrun = (int)(vh - v0 + 1 < NRUN ? vh - v0 + 1 : NRUN);
        const int64_t xe = v0 + nrun <= vh ? tc_first(v0 + nrun) : xh;   // this round ends at slice xe
        if (lane < nrun) {
            const SearchDev& S = Sall[g->sid];
            const int64_t v = v0 + lane;
            const int64_t c = v / nt, u = v - c * nt;
            const int nbc = c < nchunk - 1 ? 4 : nbl;
            const int64_t rs = c * 4 * nt + u * nbc;
            int m;
            int32_t tx, ty, tz;
            RunDesc& d = rd[b][lane];
            if (MODE == MODE_INITIAL) {
                virtual_parent(S, g->first_parent + u / g->R, tx, ty, tz);
                tx *= 2;
                ty *= 2;
                tz *= 2;
                const float4* At = S.rot + 3 * (u % g->R);   // the top level's table
                const float4 a0 = __ldg(At), a1 = __ldg(At + 1), a2 = __ldg(At + 2);
                d.a[0] = pk2(a0.x, a0.x), d.a[1] = pk2(a0.y, a0.y), d.a[2] = pk2(a0.z, a0.z);
                d.a[3] = pk2(a1.x, a1.x), d.a[4] = pk2(a1.y, a1.y), d.a[5] = pk2(a1.z, a1.z);
                d.a[6] = pk2(a2.x, a2.x), d.a[7] = pk2(a2.y, a2.y), d.a[8] = pk2(a2.z, a2.z);
                m = S.lmax;
            } else {
                const TaskRec tr = tasks[g->first_task + u];
                m = rl_level(tr.rl);
                tx = tr.tx;
                ty = tr.ty;
                tz = tr.tz;
                run_rows(d, tr.rl, S);
            }
            const LevelView& L = S.maps[m];
            const bool cmp = L.layout != LAYOUT_WIDE;
            const int32_t t3[3] = {tx, ty, tz};
            for (int i = 0; i < 3; ++i) {
                // |offset| >= 2^21 puts every point of the run outside the key range
                // (|floor(q / 2^m)| <= 2^18 by the scan bound), as the clamped one does
                int32_t o = t3[i] - (cmp ? L.base[i] : 0);
                o = o > (1 << 21) ? (1 << 21) : (o < -(1 << 21) ? -(1 << 21) : o);
                const float cf = 12582912.0f + (float)o;   // exact: an integer below 2^24
                d.kc[i] = pk2(cf, cf);
            }
            const float sc = __int_as_float((127 - m) << 23);   // 2^-m
            d.s = pk2(sc, sc);
            d.m = m;
            d.c = (int32_t)c;
            d.sid = g->sid;
            d.b0 = (int32_t)(max(rs, x0) - rs);
            d.b1 = (int32_t)(min(rs + nbc, xe) - rs);
            d.task = g->first_task + u;
            d.inside = L.layout == LAYOUT_BYTES ? (int32_t)run_inside(d, S.cbox + 2 * c, L) : 0;
        }
        if (lane == 0) s_nrun[b] = nrun;
        __syncwarp();
        bar_arrive(BAR_FULL + b, 256);   // buffer b holds the round
        cur = g->first_slice + xe;
    }
}

// Fused branch + score.  The launch's slices (task, PBLK-point block) are
// split into equal contiguous ranges, one per CTA, for the first static_pm
// per mille, the rest handed out in shrinking grabs.  Warp 7 of a CTA walks
// its ranges in rounds of at most NRUN runs (maximal pieces of one task over
// one chunk) and describes each round into one of two buffers (task record,
// rotation rows, key offsets, the chunk-box test), one run per lane, while
// warps 0..6 score the round before: staging a chunk of the scan only when
// the chunk changes, and adding each run's 8 child counts to the dense
// scores at the round's end.  Describing overlaps scoring, so a round's
// loads and FP64 row formation no longer stall the scoring warps.
template <int MODE, bool BYTES>
__global__ void __launch_bounds__(256, BRANCH_CTAS_PER_SM)
    branch3_kernel(Plan* __restrict__ P, const SearchDev* __restrict__ Sall, const TaskRec* __restrict__ tasks,
                   int32_t* dense)
{
    __shared__ ulonglong2 sxy[PCHUNK / 2];
    __shared__ f2 sz[PCHUNK / 2];
    __shared__ RunDesc rd[2][NRUN];
    __shared__ uint32_t red[2][NRUN][4];
    __shared__ uint32_t lut[256];   // child counter increments per 8-bit child mask
    __shared__ int32_t s_nrun[2];
    const int tid = threadIdx.x, lane = tid & 31;
    // launch-independent set-up, before waiting on the kernel before
    for (int i = tid; i < 2 * 4 * NRUN; i += blockDim.x) (&red[0][0][0])[i] = 0u;
    for (int i = tid; i < 256; i += blockDim.x) lut[i] = child_lut_entry((uint32_t)i);
    pdl_wait();   // the round's plan and tasks are written by the kernels before
    pdl_trigger();
    __syncthreads();
    if (P->status != PLAN_OK || P->grow) return;
    const int64_t n_slices = P->n_slices;

    if (tid >= NCONS) {   // the describing warp
        describe_rounds<MODE>(P, Sall, tasks, rd, s_nrun, n_slices);
        return;
    }

    // ---- the scoring warps (threads 0 .. NCONS - 1) -------------------------
    float* fxy = reinterpret_cast<float*>(sxy);
    float* fz = reinterpret_cast<float*>(sz);
    int32_t staged_sid = -1, staged_c = -1;   // the chunk in shared memory (the same in every scoring thread)
    auto stage = [&](int32_t sid, int32_t c) {   // chunk c of search sid's scan, as coordinate pairs
        const SearchDev& S = Sall[sid];
        const int32_t k0 = c * PCHUNK;
        const int32_t n = min(PCHUNK, S.K - k0);
        for (int i = tid; i < n; i += NCONS) {
            const float4 p = __ldg(S.scan + k0 + i);
            const int j = i >> 1, h = i & 1;
            fxy[4 * j + h] = p.x;
            fxy[4 * j + 2 + h] = p.y;
            fz[2 * j + h] = p.z;
        }
        staged_sid = sid;
        staged_c = c;
        bar_sync(BAR_CONS, NCONS);   // staged points visible
    };
    {   // the chunk of the CTA's first static slice, staged while warp 7 describes
        const int64_t ns = static_slices(P, n_slices);
        const int64_t cur = ns * blockIdx.x / gridDim.x, end = ns * (blockIdx.x + 1) / gridDim.x;
        int32_t sid, c;
        if (cur < end && slice_chunk(P, cur, sid, c)) stage(sid, c);
    }
    for (int round = 0;; ++round) {
        const int b = round & 1;
        bar_sync(BAR_FULL + b, 256);   // the describing warp filled buffer b
        const int nrun = s_nrun[b];
        if (nrun == 0) break;
        for (int r = 0; r < nrun; ++r) {
            const RunDesc& d = rd[b][r];
            const SearchDev& S = Sall[d.sid];
            if (d.sid != staged_sid || d.c != staged_c) {   // uniform over the scoring threads
                if (staged_sid >= 0) bar_sync(BAR_CONS, NCONS);   // the previous chunk's readers are done
                stage(d.sid, d.c);
            }
            const LevelView Lv = S.maps[d.m];
            const Row2 r0{d.a[0], d.a[1], d.a[2]};
            const Row2 r1{d.a[3], d.a[4], d.a[5]};
            const Row2 r2{d.a[6], d.a[7], d.a[8]};
            const int n = min(PCHUNK, S.K - d.c * PCHUNK);
            const int jlo = d.b0 * (PBLK / 2), jhi = min(d.b1 * (PBLK / 2), (n + 1) >> 1);
            uint32_t acc = 0;   // 4-bit child counters (child_lut_entry)
            if (BYTES) {   // every level of every search is a byte grid: only its path is compiled
                if (d.inside)
                    score_run<LAYOUT_BYTES, true>(sxy, sz, n, jlo, jhi, Lv, r0, r1, r2, d.s, d.kc[0], d.kc[1],
                                                  d.kc[2], lut, acc, tid, NCONS);
                else
                    score_run<LAYOUT_BYTES>(sxy, sz, n, jlo, jhi, Lv, r0, r1, r2, d.s, d.kc[0], d.kc[1], d.kc[2], lut,
                                            acc, tid, NCONS);
            } else if (Lv.layout == LAYOUT_BYTES && d.inside)
                score_run<LAYOUT_BYTES, true>(sxy, sz, n, jlo, jhi, Lv, r0, r1, r2, d.s, d.kc[0], d.kc[1], d.kc[2],
                                              lut, acc, tid, NCONS);
            else if (Lv.layout == LAYOUT_BYTES)
                score_run<LAYOUT_BYTES>(sxy, sz, n, jlo, jhi, Lv, r0, r1, r2, d.s, d.kc[0], d.kc[1], d.kc[2], lut,
                                        acc, tid, NCONS);
            else if (Lv.layout == LAYOUT_DENSE)
                score_run<LAYOUT_DENSE>(sxy, sz, n, jlo, jhi, Lv, r0, r1, r2, d.s, d.kc[0], d.kc[1], d.kc[2], lut,
                                        acc, tid, NCONS);
            else if (Lv.layout == LAYOUT_COMPACT)
                score_run<LAYOUT_COMPACT>(sxy, sz, n, jlo, jhi, Lv, r0, r1, r2, d.s, d.kc[0], d.kc[1], d.kc[2], lut,
                                          acc, tid, NCONS);
            else
                score_run<LAYOUT_WIDE>(sxy, sz, n, jlo, jhi, Lv, r0, r1, r2, d.s, d.kc[0], d.kc[1], d.kc[2], lut,
                                       acc, tid, NCONS);
            // word k: children (jx, jz) = (k & 1, k >> 1), jy = 0 low and jy = 1 high;
            // 16-bit fields: at most 10 points per thread x 32 lanes, x 7 warps, per field
            uint32_t e0 = acc & 0x000F000Fu, o0 = (acc >> 4) & 0x000F000Fu;
            uint32_t e1 = (acc >> 8) & 0x000F000Fu, o1 = (acc >> 12) & 0x000F000Fu;
            e0 = __reduce_add_sync(0xffffffffu, e0);
            o0 = __reduce_add_sync(0xffffffffu, o0);
            e1 = __reduce_add_sync(0xffffffffu, e1);
            o1 = __reduce_add_sync(0xffffffffu, o1);
            if (lane == 0) {
                if (e0) atomicAdd(&red[b][r][0], e0);
                if (o0) atomicAdd(&red[b][r][1], o0);
                if (e1) atomicAdd(&red[b][r][2], e1);
                if (o1) atomicAdd(&red[b][r][3], o1);
            }
        }
        bar_sync(BAR_CONS, NCONS);   // every scoring warp's partial sums are in
        for (int w = tid; w < 4 * nrun; w += NCONS) {
            // word k of a run: children with jx = k & 1, jz = k >> 1; low half jy = 0, high half jy = 1
            const int r = w >> 2, k = w & 3;
            const uint32_t sum = red[b][r][k];
            if (!sum) continue;
            red[b][r][k] = 0u;   // zero again before the buffer's next round
            int32_t* dd = dense + rd[b][r].task * 8 + 4 * (k & 1) + (k >> 1);
            if (sum & 0xFFFFu) atomicAdd(dd, (int32_t)(sum & 0xFFFFu));
            if (sum >> 16) atomicAdd(dd + 2, (int32_t)(sum >> 16));
        }
        bar_arrive(BAR_EMPTY + b, 256);   // buffer b may be refilled
    }
}

// the second pass of the lexmin leaf over the current node array (kept out
// of line: the survivor pass keeps its registers)
__device__ __noinline__ void lex_rotation_pass(SearchDev* S, const FrontDev& F, const LoopState* LS)
{
    const int cur = LS->cur;
    const int64_t n = min((int64_t)LS->fn[cur], LS->cap);   // appends past the capacity were not stored
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t key = F.keys[cur][i];
        Ctl* c = S[key >> 24].ctl;
        if (c->reason != 3 || (int32_t)(key & 0xFFFFFFu) != c->sstar) continue;
        const NodeRec nd = F.nodes[cur][i];
        if (rl_level(nd.rl) != 0) continue;
        if (lex_translation(nd) == c->lex_t) atomicMin(&c->lex_r, rl_rot(nd.rl));
    }
}

// survivors: children scoring above their search's best, appended to the
// frontier array the next iteration reads, with their bucket counts
// (nodes, children, leaves) and the search's size and top bucket.  The
// append position is claimed once per CTA (one atomic on the array's count
// per 256 children instead of one per warp), and when the launch holds one
// search its size and top bucket are raised once per CTA too.
// First, when a search popped a leaf bucket this iteration, the second pass
// of its lexmin leaf: the smallest rotation among the bucket's leaves at the
// smallest translation key (the compaction's first pass found that key);
// with lex_only nothing else.
template <int MODE>
__global__ void __launch_bounds__(256) finalize_kernel(const Plan* __restrict__ P, SearchDev* S,
                                                       const TaskRec* __restrict__ tasks, int32_t* dense, FrontDev F,
                                                       LoopState* LS, int lex_only, const int32_t* __restrict__ tscore)
{
    pdl_wait();   // the scores are written by the scoring kernel before
    pdl_trigger();
    if (P->grow) return;   // the round waits for the host to grow the frontier
    if (MODE == MODE_SEARCH && LS->lex_pass) lex_rotation_pass(S, F, LS);
    if (lex_only || P->status != PLAN_OK) return;
    __shared__ uint32_t s_woff[8];
    __shared__ uint32_t s_total;
    __shared__ unsigned long long s_base;
    __shared__ int32_t s_top;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nxt = 1 - LS->cur;
    const bool one = P->nseg == 1;   // every child of the launch belongs to one search
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_dense = P->n_tasks * 8;
    if (threadIdx.x == 0) s_top = -1;
    __syncthreads();
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < n_dense; b0 += stride) {   // uniform per CTA
        const int64_t d = b0 + threadIdx.x;
        bool surv = false, viol = false;
        double vex = 0.0;
        int32_t score = 0, sid = 0;
        NodeRec nd;
        nd.cx = nd.cy = nd.cz = 0;
        nd.rl = 0;
        int m = 0;
        uint32_t crot = 0;
        if (d < n_dense) {
            const int64_t u = d >> 3;
            const int j = (int)(d & 7);
            const Seg& g = P->seg[find_task_seg(P, u)];
            sid = g.sid;
            bool valid = true;
            int32_t tx, ty, tz;
            if (MODE == MODE_INITIAL) {
                const SearchDev& s = S[sid];
                const int64_t lu = u - g.first_task;
                virtual_parent(s, g.first_parent + lu / g.R, tx, ty, tz);
                tx = 2 * tx + (j >> 2);
                ty = 2 * ty + ((j >> 1) & 1);
                tz = 2 * tz + (j & 1);
                valid = tx >= s.wmin[0] && tx <= s.wmax[0] && ty >= s.wmin[1] && ty <= s.wmax[1] && tz >= s.wmin[2] &&
                        tz <= s.wmax[2];
                m = s.lmax;
                crot = (uint32_t)(lu % g.R);
            } else {
                const TaskRec& tr = tasks[u];
                m = rl_level(tr.rl);
                crot = rl_rot(tr.rl);
                tx = tr.tx + (j >> 2);
                ty = tr.ty + ((j >> 1) & 1);
                tz = tr.tz + (j & 1);
            }
            // the dense array must be zero for the next launch: consume it
            const int32_t dv = dense[d];
            if (dv) dense[d] = 0;
            if (MODE == MODE_SEARCH && tscore) {   // Sec. IV-A: does the child beat its parent's bound?
                const int32_t ps = tscore[u];
                viol = dv > ps;
                if (viol) vex = (double)(dv - ps) / (double)dv;
            }
            if (valid) {
                score = dv;
                surv = score > g.best;
                nd.cx = tx;
                nd.cy = ty;
                nd.cz = tz;
                nd.rl = rl_pack(crot, m);
            }
        }
        if (MODE == MODE_SEARCH && tscore) {   // the bound check's counts
            const uint32_t vb = __ballot_sync(0xffffffffu, viol);
            if (vb && one) {   // one search: one atomic pair per warp
                double x = vex;
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if ((__ffs(vb) - 1) == lane) {
                    Ctl* c = S[sid].ctl;
                    atomicAdd(&c->st_viol, (unsigned long long)__popc(vb));
                    atomicAdd(&c->st_excess, x);
                }
            } else if (viol) {
                Ctl* c = S[sid].ctl;
                atomicAdd(&c->st_viol, 1ull);
                atomicAdd(&c->st_excess, vex);
            }
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, surv);
        if (lane == 0) s_woff[warp] = __popc(ball);
        if (one && ball) {
            const int32_t wtop = __reduce_max_sync(0xffffffffu, surv ? score : -1);
            if (lane == 0) atomicMax(&s_top, wtop);
        }
        __syncthreads();   // the warps' counts and top
        if (threadIdx.x == 0) {
            uint32_t t = 0;
            for (int w = 0; w < 8; ++w) {
                const uint32_t c = s_woff[w];
                s_woff[w] = t;
                t += c;
            }
            s_total = t;
            s_base = t ? atomicAdd(&LS->fn[nxt], (unsigned long long)t) : 0ull;
            if (one && t) {
                Ctl* c = S[P->seg[0].sid].ctl;
                atomicAdd((unsigned long long*)&c->size, (unsigned long long)t);
                atomicMax(&c->top, s_top);
            }
        }
        __syncthreads();   // the CTA's base and the warps' offsets
        if (s_total) {
            const uint32_t key = surv ? (((uint32_t)sid << 24) | (uint32_t)score) : 0xFFFFFFFFu;
            const uint32_t peers = __match_any_sync(0xffffffffu, key);                 // same search and score
            const uint32_t same = __match_any_sync(0xffffffffu, surv ? sid : -1);      // same search
            if (surv) {
                SearchDev& s = S[sid];
                const unsigned long long pos = s_base + s_woff[warp] + __popc(ball & ((1u << lane) - 1u));
                // bucket counts, one atomic per (search, score) group of the warp
                const uint32_t kids = (uint32_t)node_children(s.grid, m, crot);
                const uint32_t gk = __reduce_add_sync(peers, kids);
                const uint32_t gl = __reduce_add_sync(peers, m == 0 ? 1u : 0u);
                if (pos < (unsigned long long)LS->cap) {   // the run's limit (at most the arrays' size)
                    F.nodes[nxt][pos] = nd;
                    F.keys[nxt][pos] = key;
                } else {
                    atomicOr(&s.ctl->err, 1);   // the frontier is full: the search fails
                }
                if ((__ffs(peers) - 1) == lane) {
                    atomicAdd(&s.b_cnt[score], (unsigned long long)__popc(peers));
                    atomicAdd(&s.b_kids[score], (unsigned long long)gk);
                    if (gl) atomicAdd(&s.b_leaf[score], (unsigned long long)gl);
                    if (!one) atomicMax(&s.ctl->top, score);
                }
                if (!one && (__ffs(same) - 1) == lane)
                    atomicAdd((unsigned long long*)&s.ctl->size, (unsigned long long)__popc(same));
            }
        }
        if (threadIdx.x == 0) s_top = -1;
        __syncthreads();   // shared state consumed before the next pass
    }
}

cudaError_t launch_branch(int mode, Plan* P, const SearchDev* S, const TaskRec* tasks, int32_t* dense, int blocks,
                          cudaStream_t st, bool bytes_only, bool pdl)
{
    if (blocks <= 0) return cudaSuccess;
    void (*k)(Plan*, const SearchDev*, const TaskRec*, int32_t*);
    if (mode == MODE_INITIAL) k = bytes_only ? branch3_kernel<MODE_INITIAL, true> : branch3_kernel<MODE_INITIAL, false>;
    else k = bytes_only ? branch3_kernel<MODE_SEARCH, true> : branch3_kernel<MODE_SEARCH, false>;
    return launch_pdl(k, dim3(blocks), dim3(256), st, pdl, P, S, tasks, dense);
}

cudaError_t launch_finalize(int mode, const Plan* P, SearchDev* S, const TaskRec* tasks, int32_t* dense,
                            const FrontDev& F, LoopState* LS, int blocks, cudaStream_t st, bool lex_only,
                            const int32_t* tscore, bool pdl)
{
    if (blocks <= 0) return cudaSuccess;
    if (mode == MODE_INITIAL)
        return launch_pdl(finalize_kernel<MODE_INITIAL>, dim3(blocks), dim3(256), st, pdl, P, S, tasks, dense, F, LS, 0,
                          (const int32_t*)nullptr);
    return launch_pdl(finalize_kernel<MODE_SEARCH>, dim3(blocks), dim3(256), st, pdl, P, S, tasks, dense, F, LS,
                      lex_only ? 1 : 0, tscore);
}

}  // namespace bbs
