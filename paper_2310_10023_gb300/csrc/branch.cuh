// branch.cuh -- argument blocks of the scoring kernels.
#pragma once

#include <cstring>

#include "bbs_internal.cuh"

namespace bbs {

struct ScoreArgs {
    LevelView maps[MAX_LEVELS];
    DevGrid grid;
    const float4* rot;
    const float4* scan;
    int64_t k;
    const int32_t* nodes;
    int64_t n;
    int32_t* scores;
    int* err;
};

enum { MODE_INITIAL = 0, MODE_SEARCH = 1, MODE_DENSE = 2 };

struct BranchArgs {
    LevelView maps[MAX_LEVELS];
    DevGrid grid;
    const float4* rot;
    const float4* scan;
    int64_t k;
    // work items: parents x items_per (MODE_SEARCH / MODE_DENSE) or virtual
    // parents x rotations at init_level (MODE_INITIAL)
    const NodeRec* parents;
    int64_t n_items;              // used when n_items_dev is NULL
    const int64_t* n_items_dev;   // device parent count; items = count * items_per
    int64_t items_per;
    // MODE_INITIAL: virtual parents p in pmin + [0, pext), children 2p + j kept
    // when inside [wmin, wmax] (the initial set of Eq. (3)-(5))
    int64_t item0;                // MODE_INITIAL: first item of this launch
    int32_t init_level;
    int32_t pmin[3], pext[3];
    int32_t wmin[3], wmax[3];
    // MODE_DENSE output: 8 scores per item (-1 where no child)
    int32_t* dense;
    // MODE_SEARCH / MODE_INITIAL output: survivors with score > *best
    const int32_t* best;
    NodeRec* surv_nodes;
    int32_t* surv_scores;
    unsigned long long* surv_count;
    int64_t surv_cap;
    uint32_t* h_cnt;              // per score: survivors
    unsigned long long* h_kids;   // per score: their children
    uint32_t* h_leaf;             // per score: leaves among them
    int* err;
};

// launch the fused branch-and-score kernel in one of the modes above
cudaError_t launch_branch(int mode, const BranchArgs& a, cudaStream_t st);

void fill_branch_common(const bbs_maps* m, const ScanState& s, BranchArgs* a);
int branch_blocks(int64_t items);

}  // namespace bbs
