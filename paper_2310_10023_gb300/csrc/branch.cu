// branch.cu -- fused branch-and-score kernel (Eq. (13) children, Eq. (11)
// scores) and the survivor pass of the search.
//
// Work: every rotational child ("task") of every parent of a launch, over
// every point of its search's scan.  The launch's work is cut into slices
// (task, chunk of PCHUNK points) and each CTA of one resident wave takes an
// equal contiguous range of them, so the SMs finish together whatever the mix
// of parents.  Consecutive tasks that share their rotation (the engine orders
// a round's tasks by rotation) form runs: every scoring thread rotates its
// points of the chunk once per run (FP32, fixed order, no FMA), floors them
// exactly into level-key patterns, and then makes ONE byte probe per point
// and task that answers all 8 translational children 2c + j (Sec. III-C
// layout, see bbs_internal.cuh), the task's translation being an integer
// offset of the key.  The 8 child counts are kept as 4-bit fields of one
// register, summed per warp with redux.sync on byte fields, then across
// warps in shared memory, and added to a dense (task, child) score array.
// The survivor pass then keeps children scoring above their search's best.
#include "branch.cuh"

namespace bbs {

namespace {

// The rotated coordinate of Eq. (11), q_i = (A_i0 x + A_i1 y) + A_i2 z, with
// every product and sum rounded to FP32 on its own as the oracle does.
// Scalar IEEE operations with explicit rounding: the compiler neither
// contracts nor reorders them.  (Paired f32x2 multiplies and adds are not
// used: measured on this part, the compiler fuses them into FMAs whatever
// their rounding modifier and -fmad=false, which moves about a third of the
// q values by an ulp and, rarely, a floor across an integer.)
__device__ __forceinline__ float rot_q(const float* a, float x, float y, float z)
{
    return __fadd_rn(__fadd_rn(__fmul_rn(a[0], x), __fmul_rn(a[1], y)), __fmul_rn(a[2], z));
}

// Bit pattern of a floored key: for the per-axis constant C = 1.5 * 2^23 + d
// (d an integer, |d| < 2^21), fl_rd(q * 2^-m + C) rounds the exact value once,
// so while |floor(q / 2^m) + d| < 2^22 its bit pattern is KB + floor(q / 2^m) + d:
// the level-m key of Eq. (11), offset by d, in the low 22 bits.  Outside that
// range the pattern leaves [KB, KB + 2^22) and fails every range check below.
constexpr uint32_t KB = 0x4B400000u;   // bit pattern of 1.5 * 2^23
// the bit pattern of fl_rd(q * s + c): with s = 2^-m and c = 1.5 * 2^23 + d,
// KB + floor(q / 2^m) + d
__device__ __forceinline__ uint32_t key_bits(float q, float s, float c) { return __float_as_uint(__fmaf_rd(q, s, c)); }

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
// word, child i = jx + 2 jy + 4 jz (bit i of a byte grid's child mask) at
// bits 4i .. 4i + 3.  A point adds CHILD_LUT[v] for its 8-bit child mask v
// (one shared-memory load and one add).  A scoring thread counts at most
// PPT = 7 points of a task (a chunk is PCHUNK = 7 x 224 points), so no
// counter passes 7, and the even and the odd children's counters, spread to
// bytes, sum over a warp's 32 lanes to at most 224 per byte.
__host__ __device__ constexpr uint32_t child_lut_entry(uint32_t v)
{
    return ((v & 1u) << 0) | (((v >> 1) & 1u) << 4) | (((v >> 2) & 1u) << 8) | (((v >> 3) & 1u) << 12) |
           (((v >> 4) & 1u) << 16) | (((v >> 5) & 1u) << 20) | (((v >> 6) & 1u) << 24) | (((v >> 7) & 1u) << 28);
}
// the scoring CTA: warps 0..6 score (NCONS threads), warp 7 describes the rounds
constexpr int NCONS = 224;

// the 8-bit child mask from the two plane words of the brick layouts
// (bits {0, 1, 5, 6}: children jx + 5 jy of the z = 0 and z = 1 planes)
__device__ __forceinline__ uint32_t planes_mask(uint32_t w0, uint32_t w1)
{
    return (w0 & 3u) | ((w0 >> 3) & 0xCu) | ((w1 & 3u) << 4) | ((w1 << 1) & 0xC0u);
}

// One task of a brick layout over points [plo, phi) of the staged chunk:
// every point rotated and floored with the task's own offsets; thread t of
// the nt scoring threads takes points plo + t, plo + t + nt, ...  The floor,
// the level shift and the key offset are one fma.rm of q (see KB).
template <int LAYOUT>
__device__ __forceinline__ void score_run(const float4* sp, int plo, int phi, const LevelView& L, const float (&A)[9],
                                          float s, float cx, float cy, float cz, const uint32_t* lut, uint32_t& acc,
                                          int t, int nt)
{
    for (int p = plo + t; p < phi; p += nt) {
        const float4 v4 = sp[p];
        const uint32_t bx = key_bits(rot_q(A, v4.x, v4.y, v4.z), s, cx);
        const uint32_t by = key_bits(rot_q(A + 3, v4.x, v4.y, v4.z), s, cy);
        const uint32_t bz = key_bits(rot_q(A + 6, v4.x, v4.y, v4.z), s, cz);
        uint32_t w0, w1;
        child_bits<LAYOUT>(L, bx, by, bz, w0, w1);
        acc += lut[planes_mask(w0, w1)];
    }
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

// The key bounds of a chunk under rotation rows A at level m: for every
// point of the chunk and axis i, klo_i <= floor(q_i / 2^m) <= khi_i, with q_i
// the FP32 value of sum_k A_ik x_k (the translation is added to the key
// afterwards, exactly).  Over the chunk's box the exact sum lies in [lo, hi]
// (per term the smaller and larger of the corner products).  Here lo and hi
// are formed in FP32 (three products, two sums: within 3u / (1 - 3u) of mag =
// sum_k |A_ik| max |x_k|, u = 2^-24), and each point's FP32 q_i lies within
// as much again of its exact value, so widening by 2e-6 mag (which also
// covers the rounding of mag and of the widening) bounds every q_i.  The
// floors are exact integers (|q / 2^m| <= 2^18 by the scan bound).  FP32
// throughout: FP64 runs at a small fraction of the FP32 rate on this part.
__device__ __forceinline__ void chunk_key_bounds(const float A[9], const float4* __restrict__ box, int m,
                                                 float klo[3], float khi[3])
{
    const float4 blo = __ldg(box), bhi = __ldg(box + 1);
    const float lo3[3] = {blo.x, blo.y, blo.z}, hi3[3] = {bhi.x, bhi.y, bhi.z};
    const float s = __int_as_float((127 - m) << 23);   // 2^-m
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float qlo = 0.0f, qhi = 0.0f, mag = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float a = A[3 * i + k];
            const float p1 = __fmul_rn(a, lo3[k]), p2 = __fmul_rn(a, hi3[k]);
            qlo = __fadd_rn(qlo, fminf(p1, p2));
            qhi = __fadd_rn(qhi, fmaxf(p1, p2));
            mag = __fadd_rn(mag, __fmul_rn(fabsf(a), fmaxf(fabsf(lo3[k]), fabsf(hi3[k]))));
        }
        const float marg = __fadd_rn(__fmul_rn(2e-6f, mag), 1e-30f);
        klo[i] = floorf(__fmul_rn(__fsub_rn(qlo, marg), s));
        khi[i] = floorf(__fmul_rn(__fadd_rn(qhi, marg), s));
    }
}

// A run: consecutive slices of one round that score one chunk of one
// search's scan under one rotation (tasks sharing their rotational child,
// translations apart), described in shared memory for the whole CTA.  The
// scoring threads rotate their points of the chunk once per run and probe
// once per point and task.
struct __align__(16) RunDesc {
    float a[9];       // rotation entries A_ik
    float s;          // 2^-m
    int32_t m;        // child level
    int32_t c;        // point chunk
    int32_t sid;      // search
    int32_t first;    // the run's slices: slots [first, first + n) of the round
    int32_t n;
    int32_t pad[2];
};

// One slice of a round: a task over its run's chunk.
struct __align__(16) SlotDesc {
    float kc[3];      // per-axis 1.5 * 2^23 + translation (- box origin) (brick layouts)
    uint32_t pad;
    uint32_t ok[3];   // byte grids near the edge: per-axis translation (- box origin) - KB, mod 2^32
    uint32_t pad2;
    int64_t task;     // launch-local task index
    uint32_t delta;   // byte grids: index offset of the translation, with the folded pattern constant
    int32_t inside;   // every point of the chunk lands inside the level's byte grid
};

constexpr int NSLOT = 32;   // slices per round, one per lane of the describing warp

}  // namespace

// named barriers of the scoring CTA (0 is __syncthreads): the describing
// warp fills round buffer b and arrives on FULL + b; the scoring warps wait
// there, score, and arrive on EMPTY + b when they no longer read the buffer;
// CONS synchronizes the scoring warps alone
constexpr int BAR_FULL = 1, BAR_EMPTY = 3, BAR_CONS = 5;
__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void bar_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// The CTA's static range [cur, end) of the launch's slices: the first
// static_pm / 1000 of them in equal shares, the rest handed out later in
// shrinking grabs.  (Weighing a scan's short last chunk by its points
// measured slower: a slice's description and reduction cost the same
// whatever its points.)
__device__ __forceinline__ void static_range(const Plan* P, int64_t n_slices, int64_t& cur, int64_t& end,
                                             int64_t& n_static)
{
    n_static = n_slices * P->static_pm / 1000;
    cur = n_static * blockIdx.x / gridDim.x;
    end = n_static * (blockIdx.x + 1) / gridDim.x;
}

// The search and point chunk of slice x (false when its segment is empty):
// the chunk the CTA's first run reads
__device__ __forceinline__ bool slice_chunk(const Plan* P, int64_t x, int32_t& sid, int32_t& c)
{
    const Seg& g = P->seg[find_slice_seg(P, x)];
    if (g.n_tasks <= 0 || x < g.first_slice || x >= g.first_slice + g.n_tasks * g.nblk) return false;
    sid = g.sid;
    c = (int32_t)((x - g.first_slice) / g.n_tasks);
    return true;
}

// The describing warp of a scoring CTA (out of line: its registers and its
// row formation stay out of the scoring warps' allocation).  A round is up to
// NSLOT consecutive slices of one segment, one per lane; lanes whose slice
// opens a new chunk or a new rotation lead a run and form its rotation rows
// and its chunk's key bounds, every lane its task's offsets and inside test.
template <int MODE>
__device__ __noinline__ void describe_rounds(Plan* __restrict__ P, const SearchDev* __restrict__ Sall,
                                             const TaskRec* __restrict__ tasks, RunDesc (*rd)[NSLOT],
                                             SlotDesc (*sd)[NSLOT], int32_t (*s_cnt)[2], int64_t n_slices)
{
    const int lane = threadIdx.x & 31;
    // the static range first, then grabs of at least grab_min as CTAs finish
    int64_t cur, end, n_static;
    static_range(P, n_slices, cur, end, n_static);
    const int64_t grab_min = P->grab_min > 0 ? P->grab_min : 1;
    int gi = -1;
    // scan points rotated for the current search (lane 0), added to its control block on a change of search
    // (searches scored outside the engine -- bbs_score_children, the host queue -- have none)
    int rot_sid = -1;
    unsigned long long rot_pts = 0;
    auto flush_rot = [&]() {
        if (lane == 0 && rot_sid >= 0 && rot_pts) {
            Ctl* c = Sall[rot_sid].ctl;
            if (c) atomicAdd(&c->st_rotpts, rot_pts);
        }
        rot_pts = 0;
    };
    for (int round = 0;; ++round) {
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
            if (lane == 0) s_cnt[b][0] = 0;
            __syncwarp();
            bar_arrive(BAR_FULL + b, 256);
            flush_rot();
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
        // seg-relative slices: slice x is task x mod nt over chunk x / nt
        const int64_t x0 = cur - g->first_slice, xh = min(end, seg_end) - g->first_slice;
        const int cnt = (int)(xh - x0 < NSLOT ? xh - x0 : NSLOT);
        const bool valid = lane < cnt;
        const SearchDev& S = Sall[g->sid];
        int64_t c = -1, u = 0;
        uint32_t key = 0;   // the slice's rotation: rl, or the top table's index
        int32_t m = 0, t3[3] = {0, 0, 0};
        if (valid) {
            const int64_t x = x0 + lane;
            c = x / nt;
            u = x - c * nt;
            if (MODE == MODE_INITIAL) {
                // rotation-major: the virtual parents of one rotation are consecutive tasks
                const int64_t take = nt / g->R;
                const int64_t ri = u / take;
                virtual_parent(S, g->first_parent + (u - ri * take), t3[0], t3[1], t3[2]);
                for (int i = 0; i < 3; ++i) t3[i] *= 2;
                key = (uint32_t)ri;
                m = S.lmax;
            } else {
                const TaskRec tr = tasks[g->first_task + u];
                key = tr.rl;
                m = rl_level(tr.rl);
                t3[0] = tr.tx;
                t3[1] = tr.ty;
                t3[2] = tr.tz;
            }
        }
        const int64_t cprev = __shfl_up_sync(0xffffffffu, c, 1);
        const uint32_t kprev = __shfl_up_sync(0xffffffffu, key, 1);
        const bool start = valid && (lane == 0 || c != cprev || key != kprev);
        const uint32_t starts = __ballot_sync(0xffffffffu, start);
        const uint32_t below = starts & (0xFFFFFFFFu >> (31 - lane));   // run starts at lanes <= lane
        const int lead = 31 - __clz(below);                             // lane 0 always starts
        float klo[3] = {0.0f, 0.0f, 0.0f}, khi[3] = {0.0f, 0.0f, 0.0f};
        if (start) {
            RunDesc& d = rd[b][__popc(below) - 1];
            float A[9];
            if (MODE == MODE_INITIAL) {
                const float4* At = S.rot + 3 * key;   // the top level's table
                const float4 a0 = __ldg(At), a1 = __ldg(At + 1), a2 = __ldg(At + 2);
                A[0] = a0.x, A[1] = a0.y, A[2] = a0.z;
                A[3] = a1.x, A[4] = a1.y, A[5] = a1.z;
                A[6] = a2.x, A[7] = a2.y, A[8] = a2.z;
            } else {
                search_rows(S.cs, S.grid, m, rl_rot(key), A);
            }
#pragma unroll
            for (int e = 0; e < 9; ++e) d.a[e] = A[e];
            const float sc = __int_as_float((127 - m) << 23);   // 2^-m
            d.s = sc;
            d.m = m;
            d.c = (int32_t)c;
            d.sid = g->sid;
            d.first = lane;
            const uint32_t above = lane == 31 ? 0u : starts >> (lane + 1);
            d.n = (above ? __ffs(above) + lane : cnt) - lane;
            chunk_key_bounds(A, S.cbox + 2 * c, m, klo, khi);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            klo[i] = __shfl_sync(0xffffffffu, klo[i], lead);
            khi[i] = __shfl_sync(0xffffffffu, khi[i], lead);
        }
        bool own = false;   // the slice rotates the chunk on its own (edge or brick layout)
        if (valid) {
            const LevelView& L = S.maps[m];
            const bool cmp = L.layout != LAYOUT_WIDE;
            SlotDesc& e = sd[b][lane];
            bool in = L.layout == LAYOUT_BYTES;
            int32_t o[3];
            for (int i = 0; i < 3; ++i) {
                // |offset| >= 2^21 puts every point outside the key range
                // (|floor(q / 2^m)| <= 2^18 by the scan bound), as the clamped one does
                int32_t v = t3[i] - (cmp ? L.base[i] : 0);
                v = v > (1 << 21) ? (1 << 21) : (v < -(1 << 21) ? -(1 << 21) : v);
                o[i] = v;
                const float cf = 12582912.0f + (float)v;   // exact: an integer below 2^24
                e.kc[i] = cf;
                e.ok[i] = (uint32_t)v - KB;   // pattern KB + k plus this: the relative key k + v
                // inside: every key of the chunk in [0, rmax_i + 1] (sums of integers below 2^24: exact)
                in = in && klo[i] + (float)v >= 0.0f && khi[i] + (float)v <= (float)L.rmax[i] + 1.0f;
            }
            e.task = g->first_task + u;
            e.inside = in ? 1 : 0;
            own = !in;
            // index of key (k + o) = base pattern index (rotate_keys) + delta, mod 2^32:
            // the offsets' index plus -KB (ny nz + nz + 1), the patterns' constant
            e.delta = ((uint32_t)o[0] * L.nby + (uint32_t)o[1]) * L.nbz + (uint32_t)o[2] -
                      KB * (L.nby * L.nbz + L.nbz + 1u);
        }
        // scan points rotated by this round: a byte-grid run rotates once, and once more for its slices
        // near the grid's edge; a brick-layout run once per slice
        const uint32_t owns = __ballot_sync(0xffffffffu, own);
        uint32_t rp = 0;   // at most NSLOT + 1 rotations of PCHUNK points per round
        if (start) {
            const uint32_t above = lane == 31 ? 0u : starts >> (lane + 1);
            const int nr = (above ? __ffs(above) + lane : cnt) - lane;   // the run's slices
            const uint32_t rmask = (nr >= 32 ? 0xFFFFFFFFu : ((1u << nr) - 1u)) << lane;
            const int npts = min(PCHUNK, S.K - (int32_t)c * PCHUNK);
            const uint32_t nown = (uint32_t)__popc(owns & rmask);
            rp = (uint32_t)npts * (S.maps[m].layout == LAYOUT_BYTES ? 1u + (nown ? 1u : 0u) : nown);
        }
        rp = __reduce_add_sync(0xffffffffu, rp);
        if (g->sid != rot_sid) {
            flush_rot();
            rot_sid = g->sid;
        }
        rot_pts += rp;
        if (lane == 0) {
            s_cnt[b][0] = __popc(starts);
            s_cnt[b][1] = cnt;
        }
        __syncwarp();
        bar_arrive(BAR_FULL + b, 256);   // buffer b holds the round
        cur += cnt;
    }
}

// points per scoring thread of a chunk: tid + i NCONS, i = 0 .. PPT - 1
constexpr int PPT = PCHUNK / NCONS;
static_assert(PPT * NCONS == PCHUNK, "a chunk is PPT points per scoring thread");
static_assert(PPT * 32 <= 255, "a warp's byte-wide child counts hold one chunk");

// The base indices of this thread's points of the staged chunk under run d's
// rotation: the floored level-m key patterns (KB + floor(q / 2^m) per axis,
// see KB) combined as (bx ny + by) nz + bz, mod 2^32.  A task adds its slot's
// delta: for a task inside the grid the sum is the key's byte index.
__device__ __forceinline__ void rotate_keys(const float4* sp, const RunDesc& d, const LevelView& L,
                                            uint32_t (&base)[PPT], int tid)
{
    float A[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) A[e] = d.a[e];
    const float s = d.s, c0 = 12582912.0f;
    const uint32_t ny = L.nby, nz = L.nbz;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const float4 v = sp[tid + i * NCONS];
        const uint32_t bx = key_bits(rot_q(A, v.x, v.y, v.z), s, c0);
        const uint32_t by = key_bits(rot_q(A + 3, v.x, v.y, v.z), s, c0);
        const uint32_t bz = key_bits(rot_q(A + 6, v.x, v.y, v.z), s, c0);
        base[i] = (bx * ny + by) * nz + bz;
    }
}

// One task inside its byte grid: one byte load per point (the 8 child bits)
// and one counter increment.  Points i >= nv of this thread lie past the
// chunk's end (their base indices are stale): their increments are masked
// off.  The min against the last cell keeps every load inside the grid
// whatever the inside test.
template <bool FULL>
__device__ __forceinline__ uint32_t gather_inside(const uint32_t (&base)[PPT], uint32_t delta, const LevelView& L,
                                                  const uint32_t* lut, int nv)
{
    const uint8_t* __restrict__ cell = reinterpret_cast<const uint8_t*>(L.slots);
    const uint32_t last = L.mask;
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const uint32_t inc = lut[__ldg(cell + min(base[i] + delta, last))];
        acc += FULL ? inc : (i < nv ? inc : 0u);
    }
    return acc;
}

// The floored level-m key patterns of this thread's points under run d's
// rotation, per axis (KB + floor(q / 2^m), see KB): the slices of the run
// near the grid's edge clamp each axis on its own.
__device__ __forceinline__ void rotate_keys3(const float4* sp, const RunDesc& d, uint32_t (&kx)[PPT],
                                             uint32_t (&ky)[PPT], uint32_t (&kz)[PPT], int tid)
{
    float A[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) A[e] = d.a[e];
    const float s = d.s, c0 = 12582912.0f;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const float4 v = sp[tid + i * NCONS];
        kx[i] = key_bits(rot_q(A, v.x, v.y, v.z), s, c0);
        ky[i] = key_bits(rot_q(A + 3, v.x, v.y, v.z), s, c0);
        kz[i] = key_bits(rot_q(A + 6, v.x, v.y, v.z), s, c0);
    }
}

// One slice near its byte grid's edge: each point's relative key k + v per
// axis (pattern + ok, mod 2^32: a negative key wraps past every bound) is
// clamped to the empty key past the box (rmax + 1), then one byte load.
// Points i >= nv of this thread lie past the chunk's end: masked off.
__device__ __forceinline__ uint32_t edge_counts(const uint32_t (&kx)[PPT], const uint32_t (&ky)[PPT],
                                                const uint32_t (&kz)[PPT], const SlotDesc& e, const LevelView& L,
                                                const uint32_t* lut, int nv)
{
    const uint8_t* __restrict__ cell = reinterpret_cast<const uint8_t*>(L.slots);
    const uint32_t ex = L.rmax[0] + 1u, ey = L.rmax[1] + 1u, ez = L.rmax[2] + 1u;
    const uint32_t ox = e.ok[0], oy = e.ok[1], oz = e.ok[2], ny = L.nby, nz = L.nbz;
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
        const uint32_t rx = min(kx[i] + ox, ex), ry = min(ky[i] + oy, ey), rz = min(kz[i] + oz, ez);
        const uint32_t inc = lut[__ldg(cell + ((rx * ny + ry) * nz + rz))];
        acc += i < nv ? inc : 0u;
    }
    return acc;
}

// A thread's 4-bit child counters of one task, summed over the warp: the
// even children's counters spread to the four bytes of one word, the odd
// children's to another (at most PPT x 32 = 224 per byte), stored by lane 0
// in the warp's own two words of the slot (no atomics).
__device__ __forceinline__ void reduce_counts(uint32_t acc, uint32_t* red2, int lane)
{
    const uint32_t ev = __reduce_add_sync(0xffffffffu, acc & 0x0F0F0F0Fu);
    const uint32_t od = __reduce_add_sync(0xffffffffu, (acc >> 4) & 0x0F0F0F0Fu);
    if (lane == 0) {
        red2[0] = ev;
        red2[1] = od;
    }
}

// Fused branch + score.  The launch's slices (task, chunk of the scan) are
// split into equal contiguous ranges, one per CTA, for the first static_pm
// per mille, the rest handed out in shrinking grabs.  Warp 7 of a CTA walks
// its ranges in rounds of at most NSLOT slices and describes each round into
// one of two buffers -- runs of slices that share a chunk and a rotation
// (their rows and the chunk's key bounds), and per slice its task's offsets
// and inside test -- while warps 0..6 score the round before: staging a
// chunk of the scan only when the chunk changes, rotating their points once
// per run, probing once per point and slice, and adding each slice's 8 child
// counts to the dense scores at the round's end.
template <int MODE, bool BYTES>
__global__ void __launch_bounds__(256, BRANCH_CTAS_PER_SM)
    branch3_kernel(Plan* __restrict__ P, const SearchDev* __restrict__ Sall, const TaskRec* __restrict__ tasks,
                   int32_t* dense)
{
    __shared__ float4 sp[PCHUNK];        // the staged chunk: (x, y, z, 0) per point
    __shared__ RunDesc rd[2][NSLOT];
    __shared__ SlotDesc sd[2][NSLOT];
    __shared__ uint32_t red[2][NSLOT][NCONS / 32][2];   // per slot and scoring warp: even, odd children's byte counts
    __shared__ uint32_t lut[256];   // child counter increments per 8-bit child mask
    __shared__ int32_t s_cnt[2][2]; // per buffer: runs, slices
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // launch-independent set-up, before waiting on the kernel before
    for (int i = tid; i < 256; i += blockDim.x) lut[i] = child_lut_entry((uint32_t)i);
    pdl_wait();   // the round's plan and tasks are written by the kernels before
    pdl_trigger();
    __syncthreads();
    if (P->status != PLAN_OK || P->grow) return;
    const int64_t n_slices = P->n_slices;

    if (tid >= NCONS) {   // the describing warp
        describe_rounds<MODE>(P, Sall, tasks, rd, sd, s_cnt, n_slices);
        return;
    }

    // ---- the scoring warps (threads 0 .. NCONS - 1) -------------------------
    int32_t staged_sid = -1, staged_c = -1;   // the chunk in shared memory (the same in every scoring thread)
    auto stage = [&](int32_t sid, int32_t c) {   // chunk c of search sid's scan
        const SearchDev& S = Sall[sid];
        const int32_t k0 = c * PCHUNK;
        const int32_t n = min(PCHUNK, S.K - k0);
        for (int i = tid; i < n; i += NCONS) sp[i] = __ldg(S.scan + k0 + i);
        staged_sid = sid;
        staged_c = c;
        bar_sync(BAR_CONS, NCONS);   // staged points visible
    };
    {   // the chunk of the CTA's first static slice, staged while warp 7 describes
        int64_t cur, end, ns;
        static_range(P, n_slices, cur, end, ns);
        int32_t sid, c;
        if (cur < end && slice_chunk(P, cur, sid, c)) stage(sid, c);
    }
    for (int round = 0;; ++round) {
        const int b = round & 1;
        bar_sync(BAR_FULL + b, 256);   // the describing warp filled buffer b
        const int nrun = s_cnt[b][0];
        if (nrun == 0) break;
        for (int r = 0; r < nrun; ++r) {
            const RunDesc& d = rd[b][r];
            const SearchDev& S = Sall[d.sid];
            if (d.sid != staged_sid || d.c != staged_c) {   // uniform over the scoring threads
                if (staged_sid >= 0) bar_sync(BAR_CONS, NCONS);   // the previous chunk's readers are done
                stage(d.sid, d.c);
            }
            const LevelView Lv = S.maps[d.m];
            const int n = min(PCHUNK, S.K - d.c * PCHUNK);
            const int t0 = d.first, t1 = d.first + d.n;
            if (BYTES || Lv.layout == LAYOUT_BYTES) {
                {   // the slices inside the grid: the run's rotated keys once, one probe per point and slice
                    uint32_t base[PPT];
                    rotate_keys(sp, d, Lv, base, tid);
                    if (n == PCHUNK) {
                        for (int t = t0; t < t1; ++t) {
                            const SlotDesc& e = sd[b][t];
                            if (e.inside) reduce_counts(gather_inside<true>(base, e.delta, Lv, lut, PPT), red[b][t][warp], lane);
                        }
                    } else {   // the scan's last chunk: this thread's points below n
                        const int nv = n > tid ? (n - tid + NCONS - 1) / NCONS : 0;
                        for (int t = t0; t < t1; ++t) {
                            const SlotDesc& e = sd[b][t];
                            if (e.inside) reduce_counts(gather_inside<false>(base, e.delta, Lv, lut, nv), red[b][t][warp], lane);
                        }
                    }
                }
                bool edge = false;   // uniform: the slot descriptors are shared
                for (int t = t0; t < t1 && !edge; ++t) edge = !sd[b][t].inside;
                if (edge) {   // near the grid's edge: the run's keys per axis, each clamped
                    uint32_t kx[PPT], ky[PPT], kz[PPT];
                    rotate_keys3(sp, d, kx, ky, kz, tid);
                    const int nv = n > tid ? (n - tid + NCONS - 1) / NCONS : 0;
                    for (int t = t0; t < t1; ++t) {
                        const SlotDesc& e = sd[b][t];
                        if (!e.inside) reduce_counts(edge_counts(kx, ky, kz, e, Lv, lut, nv), red[b][t][warp], lane);
                    }
                }
            } else {   // brick layouts: every slice rotates and probes on its own
                float A[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) A[k] = d.a[k];
                for (int t = t0; t < t1; ++t) {
                    const SlotDesc& e = sd[b][t];
                    uint32_t acc = 0;
                    if (Lv.layout == LAYOUT_DENSE)
                        score_run<LAYOUT_DENSE>(sp, 0, n, Lv, A, d.s, e.kc[0], e.kc[1], e.kc[2], lut, acc, tid, NCONS);
                    else if (Lv.layout == LAYOUT_COMPACT)
                        score_run<LAYOUT_COMPACT>(sp, 0, n, Lv, A, d.s, e.kc[0], e.kc[1], e.kc[2], lut, acc, tid, NCONS);
                    else
                        score_run<LAYOUT_WIDE>(sp, 0, n, Lv, A, d.s, e.kc[0], e.kc[1], e.kc[2], lut, acc, tid, NCONS);
                    reduce_counts(acc, red[b][t][warp], lane);
                }
            }
        }
        bar_sync(BAR_CONS, NCONS);   // every scoring warp's counts are in
        // Each slot's counts summed over the scoring warps: word k holds the
        // children i = 2 q + k (q = 0..3) in its bytes; bytes 0, 2 and 1, 3
        // are summed in 16-bit fields (at most 7 x 224 each).
        const int nsl = s_cnt[b][1];
        for (int w = tid; w < 2 * nsl; w += NCONS) {
            const int t = w >> 1, k = w & 1;
            uint32_t lo = 0, hi = 0;
#pragma unroll
            for (int v = 0; v < NCONS / 32; ++v) {
                const uint32_t x = red[b][t][v][k];
                lo += x & 0x00FF00FFu;
                hi += (x >> 8) & 0x00FF00FFu;
            }
            // child i = jx + 2 jy + 4 jz -> dense 4 jx + 2 jy + jz (jx = k)
            int32_t* dd = dense + sd[b][t].task * 8 + 4 * k;
            const uint32_t c0 = lo & 0xFFFFu, c2 = hi & 0xFFFFu, c4 = lo >> 16, c6 = hi >> 16;   // i = k + 0, 2, 4, 6
            if (c0) atomicAdd(dd, (int32_t)c0);       // jy = 0, jz = 0
            if (c2) atomicAdd(dd + 2, (int32_t)c2);   // jy = 1, jz = 0
            if (c4) atomicAdd(dd + 1, (int32_t)c4);   // jy = 0, jz = 1
            if (c6) atomicAdd(dd + 3, (int32_t)c6);   // jy = 1, jz = 1
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
                // rotation-major, as the scoring kernel reads the initial set
                const int64_t take = g.n_tasks / g.R;
                const int64_t ri = lu / take;
                virtual_parent(s, g.first_parent + (lu - ri * take), tx, ty, tz);
                tx = 2 * tx + (j >> 2);
                ty = 2 * ty + ((j >> 1) & 1);
                tz = 2 * tz + (j & 1);
                valid = tx >= s.wmin[0] && tx <= s.wmax[0] && ty >= s.wmin[1] && ty <= s.wmax[1] && tz >= s.wmin[2] &&
                        tz <= s.wmax[2];
                m = s.lmax;
                crot = (uint32_t)ri;
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
