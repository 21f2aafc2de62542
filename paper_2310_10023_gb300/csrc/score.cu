// score.cu -- Eq. (11) scores of caller nodes (the bbs_score_batch parity
// surface): one warp per node; lanes stride over the scan; each point is
// rotated (FP32, fixed order, no FMA), floored to its fine key, shifted to the
// node's level and looked up in that level's map; hits are summed per warp.
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
        float A[9];
        rotation_rows(a.cs, a.grid, l, (uint32_t)rot, A);
        const float4 r0 = make_float4(A[0], A[1], A[2], 0.0f), r1 = make_float4(A[3], A[4], A[5], 0.0f),
                     r2 = make_float4(A[6], A[7], A[8], 0.0f);
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
    a.cs = s.cs;
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

}  // namespace bbs
