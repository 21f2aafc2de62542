// branch.cuh -- the fused branch-and-score kernel and the search engine's
// device structures.
#pragma once

#include <cstring>

#include "bbs_internal.cuh"

namespace bbs {

constexpr int CH = 256;        // nodes per frontier chunk
constexpr int PCHUNK = 1568;   // scan points staged in shared memory per CTA (7 per scoring thread)
static_assert(PCHUNK == SCAN_CHUNK, "chunk boxes are kept per staged chunk");
constexpr int PBLK = PCHUNK;   // scan points per slice: a slice is one task over one chunk
constexpr int MAXSEG = 256;    // task runs per scoring launch
constexpr int64_t TASK_CAP = (int64_t)1 << 19;   // rotational-child tasks per scoring launch

struct ScoreArgs {
    LevelView maps[MAX_LEVELS];
    DevGrid grid;
    const double2* cs;
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
    int32_t sstar;         // last select: buckets above sstar popped
    int32_t clear;         // last select: every other node dropped
    unsigned long long lex_t;   // lexmin leaf of a popped leaf bucket: translation key,
    uint32_t lex_r;             // then rotation (Algorithm 2's tie rule)
    int32_t err;           // 1 frontier full, 4 inconsistent counts
    int64_t size;          // nodes in F
    int64_t peak;          // largest size seen by a select
    int64_t n_parents;     // parents popped by the last select
    int64_t n_tasks;       // their rotational children (tasks)
    int64_t popped_kids;   // their children (8 per task)
    int32_t reason;        // last select: 1 batch full, 2 below best, 3 leaf, 4 F emptied, 0 F was empty
    int32_t match_changed;
    int32_t active;        // slot in use
    int32_t pad;
    // statistics kept on the device (the search loop may run without the host)
    int64_t st_iters, st_parents, st_nodes, st_gathers;
    unsigned long long st_viol;   // children scoring above their parent (Sec. IV-A's bound check)
    double st_excess;             // sum over them of (child - parent) / child
    unsigned long long st_rotpts; // scan points the scoring kernel rotated (once per run of a shared rotation)
    unsigned long long t_start_ns, t_match_ns, t_end_ns;   // %globaltimer
};

// One search slot (device).  Bucket arrays have K + 1 entries (scores 0..K).
struct SearchDev {
    const float4* scan;
    const float4* cbox;         // per PCHUNK-point chunk of the scan: min, max corner
    const float4* rot;          // rows of the top level's rotations
    const double2* cs;          // (cos, sin) of every segment angle
    int32_t K;
    int32_t lmax;
    int64_t batch;
    int32_t nblk;               // PCHUNK-point chunks of the scan
    int32_t pad0;
    int32_t pmin[3], pext[3];   // virtual parents of the initial set
    int32_t wmin[3], wmax[3];   // initial translation window, Eq. (3)-(5)
    DevGrid grid;
    LevelView maps[MAX_LEVELS];
    unsigned long long* b_cnt;  // nodes per score bucket
    unsigned long long* b_kids; // their children
    unsigned long long* b_leaf; // their leaves
    Ctl* ctl;                   // this search's control block (contiguous across searches)
};

// The frontier of every search: nodes with key score | search << 24, in two
// arrays that swap roles each iteration (the current nodes are read, kept and
// new ones are appended to the other).
struct FrontDev {
    NodeRec* nodes[2];
    uint32_t* keys[2];
    int64_t cap;
};

// Rotation groups of a round that scores in one launch (engine.cu): an
// open-addressing table over (search, rl) keys whose entry index names the
// group, per-entry arrays (GROUP_TABLE entries each), and per-search lists
// of the entries in use and per-parent arrays (TASK_CAP entries each).
constexpr int64_t GROUP_TABLE = 2 * TASK_CAP;
constexpr unsigned long long GROUP_EMPTY = ~0ull;
struct GroupDev {
    unsigned long long* tab;   // GROUP_TABLE entries: the key (search << 32 | rl), or GROUP_EMPTY
    uint32_t* cnt;             // per entry: parents joined (zero between rounds)
    uint32_t* ntask;           // per entry: rotational children of each of its parents
    int64_t* off;              // per entry: the group's first task
    uint32_t* np;              // per entry: the group's parents
    uint32_t* ngrp;            // per search slot: groups created this round
    uint32_t* list;            // the entries of search s's groups, at poff[s] .. poff[s] + ngrp[s]
    uint32_t* pslot;           // per parent: its group's entry
    uint32_t* pidx;            // per parent: its index in the group
};

// Device state of the iteration loop.
struct LoopState {
    unsigned long long fn[2];   // nodes in each frontier array
    int32_t cur;                // the array holding the current nodes
    int32_t lex_pass;           // a search popped a leaf bucket this iteration
    uint32_t select_done;       // select CTAs finished this iteration (the last one plans)
    int32_t exit_on_finish;     // the device loop also ends when a search finishes or fails
    int64_t cap;                // nodes each frontier array holds
    int64_t grow_need;          // a round that asked to grow: nodes the arrays must hold
};

enum { MODE_INITIAL = 0, MODE_SEARCH = 1, MODE_DENSE = 2 };

// One rotational child of a scoring round: its parent's translation and
// rl_pack(child rotation, child level); the scoring kernel forms the
// rotation's rows (rotation_entry) when it describes the task's runs.  Its 8
// translational children are the dense scores 8 * task .. 8 * task + 7.
struct __align__(16) TaskRec {
    int32_t tx, ty, tz;     // 2 x the parent's translation indices (the children add {0,1}^3)
    uint32_t rl;
};

// A segment: the tasks of one search inside a scoring launch.  Its work is
// split into slices (task, PCHUNK-point chunk of the scan), ordered by chunk,
// then task, so that consecutive slices reuse the staged chunk and tasks
// that share a rotation stay next to each other; each CTA of the launch takes
// an equal contiguous range of slices.
struct Seg {
    int64_t first_parent;   // initial set: first virtual parent of the run
    int64_t first_task;     // launch-local index of the run's first task
    int64_t n_tasks;
    int64_t first_slice;    // launch-local index of the run's first slice
    int32_t sid;
    int32_t nblk;           // PCHUNK-point chunks of the search's scan
    int32_t R;              // initial set: rotations per virtual parent
    int32_t best;           // the search's best when the launch was planned: survivors score above it
};

enum { PLAN_OK = 0, PLAN_EMPTY = 1, PLAN_OVERFLOW = 2, PLAN_SPLIT = 3 };

// The plan of one scoring launch, in device memory: written by the host (host
// path) or by plan_kernel (device-driven iterations).  PLAN_SPLIT marks a
// round gathered whole but scored in several host-planned launches.
struct Plan {
    int64_t n_slices;
    int64_t n_tasks;         // dense child scores: 8 per task, at most 8 * TASK_CAP
    int64_t n_parents;       // device-planned rounds: the popped parents of every search
    unsigned long long next_slice;   // dynamic share: the next slice not yet handed out (0 at launch)
    int32_t static_pm;       // per-mille of the slices split statically over the CTAs
    int32_t grab_min;        // smallest dynamic grab (slices)
    int32_t nseg;
    int32_t mode;
    int32_t status;          // PLAN_*: the scoring kernels of a round run only when PLAN_OK
    int32_t iters;           // iterations of the current device-driven loop
    int32_t max_iters;       // the device-driven loop stops after this many
    int32_t grow;            // the round's survivors may not fit the frontier arrays: the host grows
                             // them before the round goes on (compact, score and survivors wait)

    Seg seg[MAXSEG];
};

// rotational children of a node at level l with rotation index rot, Eq. (13):
// first child and count per axis at level l - 1; their number (0 at the leaf level)
__host__ __device__ __forceinline__ int32_t rot_children(const DevGrid& g, int l, uint32_t rot, int32_t lo[3],
                                                         int32_t ext[3])
{
    if (l <= 0) {
        for (int i = 0; i < 3; ++i) lo[i] = ext[i] = 0;
        return 0;
    }
    const uint32_t ng = (uint32_t)g.N[l][2], nb = (uint32_t)g.N[l][1];
    const int32_t c[3] = {(int32_t)(rot / (ng * nb)), (int32_t)((rot / ng) % nb), (int32_t)(rot % ng)};
    int32_t n = 1;
    for (int i = 0; i < 3; ++i) {
        int32_t a, b;
        child_range(g, l, i, c[i], a, b);
        lo[i] = a;
        ext[i] = b - a;
        n *= b - a;
    }
    return n;
}

// launch shape (bbs_tuning), resolved: every field in range
struct Tuning {
    int64_t launch_tasks = TASK_CAP;
    int32_t static_pm = 750;
    int32_t grab_min = 16;
    int32_t ctas_per_sm = 4;
    int32_t frontier_log2 = 0;   // 0: the default starting capacity
    bool operator==(const Tuning& o) const
    {
        return launch_tasks == o.launch_tasks && static_pm == o.static_pm && grab_min == o.grab_min &&
               ctas_per_sm == o.ctas_per_sm && frontier_log2 == o.frontier_log2;
    }
};
Tuning current_tuning();
int set_tuning(const bbs_tuning* t);   // validates; NULL restores the defaults
// the search with its frontier on the host (hostqueue.cu)
int hostqueue_run(const bbs_maps* m, const float* xyz, int64_t k, int is_device, const bbs_ranges* rg,
                  const bbs_opts* opts, cudaStream_t st, bbs_result* res);

// CTAs of a scoring launch: one resident wave (4 CTAs of 256 threads per SM, 64 registers a thread)
constexpr int BRANCH_CTAS_PER_SM = 4;

// scoring and survivor kernels of one launch; `blocks` is the grid (the
// scoring kernel splits the plan's slices evenly over it, the survivor kernel
// strides), each returns at once unless the plan is PLAN_OK; bytes_only picks
// the scoring kernel compiled for byte-grid levels alone (every level of
// every search of the launch must be one: maps_all_bytes)
cudaError_t launch_branch(int mode, Plan* P, const SearchDev* S, const TaskRec* tasks, int32_t* dense, int blocks,
                          cudaStream_t st, bool bytes_only, bool pdl = false);
// survivors (score above their search's best) are appended to the frontier
// array the next iteration reads, with their bucket counts; in search mode
// first the second lexmin pass of a popped leaf bucket (lex_only: that alone)
cudaError_t launch_finalize(int mode, const Plan* P, SearchDev* S, const TaskRec* tasks, int32_t* dense,
                            const FrontDev& F, LoopState* LS, int blocks, cudaStream_t st, bool lex_only = false,
                            const int32_t* tscore = nullptr, bool pdl = false);

}  // namespace bbs
