// branch.cuh -- the fused branch-and-score kernel and the search engine's
// device structures.
#pragma once

#include <cstring>

#include "bbs_internal.cuh"

namespace bbs {

constexpr int CH = 256;        // nodes per frontier chunk
constexpr int PCHUNK = 2048;   // scan points staged in shared memory per CTA
constexpr int MAXSEG = 256;    // parent runs per scoring launch

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

// Control block of one search (device).
struct Ctl {
    int32_t best;          // provisional best score (threshold - 1 at start)
    int32_t top;           // every bucket above top is empty
    int32_t found;
    int32_t done;
    NodeRec match;
    int64_t size;          // nodes in F
    int64_t peak;          // largest size after an insertion
    int64_t n_parents;     // parents popped by the last select
    int64_t n_pop;         // chunks popped by the last select
    int64_t n_act;         // chunks in use
    int64_t popped_kids;   // children of the parents popped by the last select
    int32_t err;           // 1 pool exhausted
    int32_t reason;        // last select: 1 batch full, 2 below best, 3 leaf, 4 F emptied, 0 F was empty
    int32_t match_changed;
    int32_t active;        // slot in use
    // statistics kept on the device (the search loop may run without the host)
    int64_t st_iters, st_parents, st_nodes, st_gathers;
    unsigned long long t_start_ns, t_match_ns, t_end_ns;   // %globaltimer
};

// One search slot (device).  Frontier arrays have K + 1 buckets.
struct SearchDev {
    const float4* scan;
    const float4* rot;
    int32_t K;
    int32_t lmax;
    int64_t batch;
    int32_t rmax;               // dense task slots per parent (most rotational children)
    int32_t chunks;             // point chunks per parent
    int32_t pmin[3], pext[3];   // virtual parents of the initial set
    int32_t wmin[3], wmax[3];   // initial translation window, Eq. (3)-(5)
    DevGrid grid;
    LevelView maps[MAX_LEVELS];
    int64_t* b_cnt;
    int64_t* b_kids;
    int64_t* b_leaf;
    int32_t* b_tail;
    uint32_t* h_cnt;
    unsigned long long* h_kids;
    uint32_t* h_leaf;
    uint32_t* w_pos;
    int32_t* w_space;
    int64_t* w_choff;
    int32_t* w_tail;
    int32_t* w_fill0;
    int32_t* act;
    int32_t* pop_ids;
    int64_t* pop_start;
    Ctl* ctl;                   // this search's control block (contiguous across searches)
};

// The shared chunk pool (device).
struct PoolDev {
    NodeRec* nodes;
    int32_t* chunk_bucket;
    int32_t* chunk_fill;
    int32_t* free_ids;
    unsigned long long* free_top;
    int64_t nchunks;
};

enum { MODE_INITIAL = 0, MODE_SEARCH = 1, MODE_DENSE = 2 };

// A run of parents of one search inside a scoring launch.
struct Seg {
    int64_t first_parent;   // into the parent array, or the first virtual parent (initial set)
    int64_t first_work;     // first (parent, point chunk) work item
    int64_t n_parents;
    int64_t dense_base;     // first dense child-score slot of the run
    int32_t chunks;         // point chunks per parent
    int32_t sid;
    int32_t R;              // dense task slots per parent
    int32_t pad;
};

enum { PLAN_OK = 0, PLAN_EMPTY = 1, PLAN_OVERFLOW = 2 };

// The plan of one scoring round, in device memory: written by the host (host
// path) or by plan_kernel (device-driven iterations).
struct Plan {
    int64_t n_work;          // (parent, point chunk) work items
    int64_t n_dense;         // dense (parent, task, child) score slots, at most the dense capacity
    int32_t nseg;
    int32_t mode;
    int32_t status;          // PLAN_*: the kernels of a round run only when PLAN_OK
    int32_t iters;           // iterations of the current device-driven loop
    int32_t max_iters;       // the device-driven loop stops after this many
    int32_t pad;
    Seg seg[MAXSEG];
};

// survivors of a finalize pass
struct SurvOut {
    NodeRec* nodes;
    int32_t* scores;
    int32_t* sid;
    unsigned long long* count;
    int64_t cap;
    int* err;
};

// scoring and survivor kernels of one round; `blocks` is the grid (the
// kernels stride over the plan's work), each skips unless the plan is PLAN_OK
cudaError_t launch_branch(int mode, const Plan* P, const SearchDev* S, const NodeRec* parents, int32_t* dense,
                          int blocks, cudaStream_t st);
cudaError_t launch_finalize(int mode, const Plan* P, SearchDev* S, const NodeRec* parents, int32_t* dense,
                            const SurvOut& out, int blocks, cudaStream_t st);

}  // namespace bbs
