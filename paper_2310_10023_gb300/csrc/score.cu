// score.cu -- Eq. (11) scoring kernels.
//
// score_nodes_kernel: one warp per caller node; lanes stride over the scan;
//   each point is rotated (FP32, fixed order, no FMA), floored to its fine key,
//   shifted to the node's level and looked up; hits are summed with
//   ballot / popc.
//
// branch_kernel: the fused branch-and-score step of the search (Eq. (13)).
//   One warp per (parent, rotational child): the child rotation is loaded once,
//   every point is rotated once, and the single brick probe of its key block
//   answers all 8 translational children 2c + j.  Per-lane counters are
//   reduced with redux.sync at the end; survivors (score > best) are appended
//   with one atomic per warp and counted into the per-score histograms that
//   feed the frontier insertion.
#include "bbs_internal.cuh"
#include "branch.cuh"

namespace bbs {

__global__ void __launch_bounds__(256) score_nodes_kernel(ScoreArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < a.n; w += nwarps) {
        const int32_t* c = a.nodes + 7 * w;
        const int l = c[6];
        bool ok = l >= 0 && l < a.grid.levels;
        if (ok)
            for (int i = 0; i < 3; ++i) {
                ok = ok && c[3 + i] >= 0 && c[3 + i] < a.grid.N[l][i];
                const int64_t t = (int64_t)c[i] * ((int64_t)1 << l);
                ok = ok && t >= -(int64_t)KEY_LIMIT && t <= (int64_t)KEY_LIMIT;
            }
        if (!ok) {
            if (lane == 0) {
                a.scores[w] = -1;
                atomicOr(a.err, 1);
            }
            continue;
        }
        const int64_t rot = ((int64_t)c[3] * a.grid.N[l][1] + c[4]) * a.grid.N[l][2] + c[5];
        const float4* A = a.rot + 3 * (a.grid.rot_off[l] + rot);
        const float4 r0 = A[0], r1 = A[1], r2 = A[2];
        const LevelView L = a.maps[l];
        uint32_t hits = 0;
        for (int64_t k = lane; k < a.k; k += 32) {
            const float4 s = __ldg(a.scan + k);
            const int32_t kx = (fine_key(r0, s) >> l) + c[0];
            const int32_t ky = (fine_key(r1, s) >> l) + c[1];
            const int32_t kz = (fine_key(r2, s) >> l) + c[2];
            hits += voxel_bit(L, kx, ky, kz);
        }
        hits = __reduce_add_sync(0xffffffffu, hits);
        if (lane == 0) a.scores[w] = (int32_t)hits;
    }
}

int launch_score_nodes(const bbs_maps* m, const ScanState& s, const int32_t* d_nodes, int64_t n, int32_t* d_scores,
                       int* d_err, cudaStream_t st)
{
    if (n <= 0) return BBS_OK;
    ScoreArgs a;
    for (int l = 0; l < MAX_LEVELS; ++l) a.maps[l] = l < m->levels ? level_view(m, l) : LevelView{};
    a.grid = dev_grid(s.grid);
    a.rot = s.rot;
    a.scan = s.scan;
    a.k = s.k;
    a.nodes = d_nodes;
    a.n = n;
    a.scores = d_scores;
    a.err = d_err;
    int64_t blocks = (n + 7) / 8;
    if (blocks > 152 * 64) blocks = 152 * 64;
    score_nodes_kernel<<<(int)blocks, 256, 0, st>>>(a);
    BBS_CUDA_TRY(cudaGetLastError());
    return BBS_OK;
}

// ---------------------------------------------------------------------------

template <int MODE>
__global__ void __launch_bounds__(256) branch_kernel(BranchArgs a)
{
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_items = a.n_items_dev ? *a.n_items_dev * a.items_per : a.n_items;
    const int32_t best = a.best ? *a.best : 0;
    for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < n_items; w += nwarps) {
        int m;            // child level
        uint32_t crot;    // child rotation index at level m
        int32_t tx, ty, tz;   // child translation base 2c (children 2c + j)
        uint32_t valid = 0xFFu;
        if (MODE == MODE_INITIAL) {
            m = a.init_level;
            const int64_t nrot = (int64_t)a.grid.N[m][0] * a.grid.N[m][1] * a.grid.N[m][2];
            const int64_t wi = w + a.item0;
            const int64_t vp = wi / nrot;
            crot = (uint32_t)(wi - vp * nrot);
            const int32_t pz = (int32_t)(vp % a.pext[2]);
            const int32_t py = (int32_t)((vp / a.pext[2]) % a.pext[1]);
            const int32_t px = (int32_t)(vp / ((int64_t)a.pext[2] * a.pext[1]));
            tx = 2 * (a.pmin[0] + px);
            ty = 2 * (a.pmin[1] + py);
            tz = 2 * (a.pmin[2] + pz);
            valid = 0;
            for (int j = 0; j < 8; ++j) {
                const int32_t x = tx + (j >> 2), y = ty + ((j >> 1) & 1), z = tz + (j & 1);
                if (x >= a.wmin[0] && x <= a.wmax[0] && y >= a.wmin[1] && y <= a.wmax[1] && z >= a.wmin[2] &&
                    z <= a.wmax[2])
                    valid |= 1u << j;
            }
        } else {
            const int64_t p = w / a.items_per;
            const int32_t j = (int32_t)(w - p * a.items_per);
            const NodeRec par = a.parents[p];
            const int l = rl_level(par.rl);
            m = l - 1;
            const uint32_t prot = rl_rot(par.rl);
            const int32_t ngp = a.grid.N[l][2], nbp = a.grid.N[l][1];
            const int32_t pg = (int32_t)(prot % (uint32_t)ngp), pb = (int32_t)((prot / (uint32_t)ngp) % (uint32_t)nbp);
            const int32_t pa = (int32_t)(prot / ((uint32_t)ngp * (uint32_t)nbp));
            int32_t la, ha, lb, hb, lg, hg;
            child_range(a.grid, l, 0, pa, la, ha);
            child_range(a.grid, l, 1, pb, lb, hb);
            child_range(a.grid, l, 2, pg, lg, hg);
            const int32_t na = ha - la, nb = hb - lb, ng = hg - lg;
            if (m < 0 || j >= na * nb * ng) {
                if (MODE == MODE_DENSE && lane < 8) a.dense[8 * w + lane] = -1;
                continue;
            }
            const int32_t ja = j / (nb * ng), jb = (j / ng) % nb, jg = j % ng;
            crot = (uint32_t)(((int64_t)(la + ja) * a.grid.N[m][1] + (lb + jb)) * a.grid.N[m][2] + (lg + jg));
            tx = 2 * par.cx;
            ty = 2 * par.cy;
            tz = 2 * par.cz;
        }
        const float4* A = a.rot + 3 * (a.grid.rot_off[m] + (int64_t)crot);
        const float4 r0 = A[0], r1 = A[1], r2 = A[2];
        const LevelView L = a.maps[m];
        uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0, c6 = 0, c7 = 0;
        for (int64_t k = lane; k < a.k; k += 32) {
            const float4 s = __ldg(a.scan + k);
            const int32_t kx = (fine_key(r0, s) >> m) + tx;
            const int32_t ky = (fine_key(r1, s) >> m) + ty;
            const int32_t kz = (fine_key(r2, s) >> m) + tz;
            uint32_t w0 = 0, w1 = 0;
            if (key_in_range(kx) && key_in_range(ky) && key_in_range(kz)) {
                uint4 lo, hi;
                if (probe_brick(L, kx >> 2, ky >> 2, kz >> 2, lo, hi)) {
                    const int oz = kz & 3, sh = (kx & 3) + 5 * (ky & 3);
                    w0 = brick_plane(lo, hi, oz) >> sh;
                    w1 = brick_plane(lo, hi, oz + 1) >> sh;
                }
            }
            // child j = 4 jx + 2 jy + jz: bit jx + 5 jy of plane oz + jz
            c0 += w0 & 1u;
            c1 += w1 & 1u;
            c2 += (w0 >> 5) & 1u;
            c3 += (w1 >> 5) & 1u;
            c4 += (w0 >> 1) & 1u;
            c5 += (w1 >> 1) & 1u;
            c6 += (w0 >> 6) & 1u;
            c7 += (w1 >> 6) & 1u;
        }
        c0 = __reduce_add_sync(0xffffffffu, c0);
        c1 = __reduce_add_sync(0xffffffffu, c1);
        c2 = __reduce_add_sync(0xffffffffu, c2);
        c3 = __reduce_add_sync(0xffffffffu, c3);
        c4 = __reduce_add_sync(0xffffffffu, c4);
        c5 = __reduce_add_sync(0xffffffffu, c5);
        c6 = __reduce_add_sync(0xffffffffu, c6);
        c7 = __reduce_add_sync(0xffffffffu, c7);
        uint32_t mine = c0;
        mine = lane == 1 ? c1 : mine;
        mine = lane == 2 ? c2 : mine;
        mine = lane == 3 ? c3 : mine;
        mine = lane == 4 ? c4 : mine;
        mine = lane == 5 ? c5 : mine;
        mine = lane == 6 ? c6 : mine;
        mine = lane == 7 ? c7 : mine;
        const bool is_child = lane < 8 && ((valid >> lane) & 1u);
        if (MODE == MODE_DENSE) {
            if (lane < 8) a.dense[8 * w + lane] = is_child ? (int32_t)mine : -1;
            continue;
        }
        const bool surv = is_child && (int32_t)mine > best;
        const uint32_t ball = __ballot_sync(0xffffffffu, surv);
        if (!ball) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.surv_count, (unsigned long long)__popc(ball));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (surv) {
            const unsigned long long pos = base + __popc(ball & ((1u << lane) - 1u));
            if (pos < (unsigned long long)a.surv_cap) {
                NodeRec nd;
                nd.cx = tx + (lane >> 2);
                nd.cy = ty + ((lane >> 1) & 1);
                nd.cz = tz + (lane & 1);
                nd.rl = rl_pack(crot, m);
                a.surv_nodes[pos] = nd;
                a.surv_scores[pos] = (int32_t)mine;
                atomicAdd(&a.h_cnt[mine], 1u);
                atomicAdd(&a.h_kids[mine], (unsigned long long)node_children(a.grid, m, crot));
                if (m == 0) atomicAdd(&a.h_leaf[mine], 1u);
            } else {
                atomicOr(a.err, 2);
            }
        }
    }
}


void fill_branch_common(const bbs_maps* m, const ScanState& s, BranchArgs* a)
{
    std::memset(a, 0, sizeof(*a));
    for (int l = 0; l < MAX_LEVELS; ++l) a->maps[l] = l < m->levels ? level_view(m, l) : LevelView{};
    a->grid = dev_grid(s.grid);
    a->rot = s.rot;
    a->scan = s.scan;
    a->k = s.k;
}

int branch_blocks(int64_t items)
{
    int64_t b = (items + 7) / 8;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

cudaError_t launch_branch(int mode, const BranchArgs& a, cudaStream_t st)
{
    const int blocks = branch_blocks(a.n_items);
    if (mode == MODE_INITIAL) branch_kernel<MODE_INITIAL><<<blocks, 256, 0, st>>>(a);
    else if (mode == MODE_SEARCH) branch_kernel<MODE_SEARCH><<<blocks, 256, 0, st>>>(a);
    else branch_kernel<MODE_DENSE><<<blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

int launch_branch_dense(const bbs_maps* m, const ScanState& s, const NodeRec* d_parents, int64_t n_parents, int rmax,
                        int32_t* d_scores, cudaStream_t st)
{
    if (n_parents <= 0) return BBS_OK;
    BranchArgs a;
    fill_branch_common(m, s, &a);
    a.parents = d_parents;
    a.items_per = rmax;
    a.n_items = n_parents * rmax;
    a.dense = d_scores;
    BBS_CUDA_TRY(launch_branch(MODE_DENSE, a, st));
    return BBS_OK;
}

}  // namespace bbs
