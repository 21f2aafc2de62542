// engine.cuh -- host side of the batched best-first search engine (engine.cu).
//
// An Engine owns the shared frontier arrays and up to max_slots search slots.  A
// search is added into a free slot (scan uploaded, grid and rotation tables
// built, frontier arrays allocated), its initial set is scored by start(),
// and every step() advances every live search by one canonical batch.  A
// search that finishes is reported by step() and released by finalize(),
// which also writes its bbs_result.  Slots can be added between steps, so the
// same engine serves one call (bbs_localize), a batch (bbs_localize_many) or
// a stream of requests (the server).  A search's trajectory depends only on
// its own batches, never on which other searches share the launches.
#pragma once

#include <cstdint>
#include <vector>

#include "branch.cuh"

namespace bbs {

struct SearchHost {
    bool used = false;     // the slot holds a search
    bool live = false;     // the search is still iterating
    bool fresh = false;    // its initial set is not scored yet
    ScanState scan{};
    const bbs_maps* maps = nullptr;
    bbs_result res{};
    int32_t thr = 0;
    int rmax = 1;
    int chunks = 1;
    int status = 0;        // error status when the search failed on its own
    double t0 = 0, t_match = -1, t_init = 0, t_end = 0;
    SearchDev dev{};
    Ctl ctl0{};
    std::vector<void*> bufs;
    size_t bytes = 0;      // device bytes held by the search
    uint64_t tag = 0;
};

// search slots of one engine: a frontier key holds its search in the top byte
constexpr int MAX_SLOTS = 256;

// the scoring launches of the last timed call on this thread: units (tasks x
// scan points) and device milliseconds of each (bbs_launch_log)
struct LaunchLog {
    std::vector<int64_t> units;
    std::vector<double> ms;
};
LaunchLog& launch_log();

class Engine {
  public:
    Engine(cudaStream_t st, int max_slots, int64_t pool_nodes, bool timed);
    ~Engine();
    Engine(const Engine&) = delete;
    Engine& operator=(const Engine&) = delete;

    int init();
    // reuse for a new run on `st` (the previous run has completed)
    int begin_run(cudaStream_t st, bool timed);
    // a new search in a free slot; *slot receives its index
    int add(const bbs_maps* m, const float* xyz, int64_t k, int is_device, const bbs_ranges* rg, const bbs_opts* opts,
            uint64_t tag, int* slot);
    // score the initial sets of every search added since the last call
    int start();
    // one host-driven iteration of every live search (one synchronization);
    // searches that finished are appended to *finished
    int step(std::vector<int>* finished);
    // advance every live search: by default a captured CUDA graph loops over
    // up to max_iters iterations on the device without the host (a while
    // node whose condition the planning select clears); with BBS_HOST_DRIVEN
    // one host-driven step.  Results are identical either way.
    int iterate(int max_iters, std::vector<int>* finished);
    void set_host_driven(bool v) { host_driven_ = v; }
    // the device loop of iterate() also ends at the first iteration in which a
    // search finishes or fails (the server reports each result at once)
    int set_exit_on_finish(bool v);
    // host-written flag the device loop polls every iteration: nonzero ends
    // it after the current iteration (the server sets it when a request
    // arrives or is cancelled, so the new work joins without waiting)
    volatile int* wake_flag() { return h_wake_; }
    // the frontier of this run holds at most n nodes: the arrays grow
    // (doubling) up to n when a round's survivors might not fit, and a larger
    // pool left by an earlier run is used only up to n
    int set_max_nodes(int64_t n);
    // the search's result; the slot and its memory are released
    int finalize(int slot, bbs_result* out);
    // stop a search early and release it (its result reports status `code`)
    int cancel(int slot, int code, bbs_result* out);

    int live_count() const;
    int used_count() const;
    int free_slot() const;
    size_t fixed_bytes() const { return fixed_bytes_; }
    size_t slot_bytes(int slot) const { return hosts_[(size_t)slot].bytes; }
    uint64_t tag(int slot) const { return hosts_[(size_t)slot].tag; }
    int64_t pool_nodes() const { return fcap_; }
    // device bytes a search of k points with this grid would hold
    size_t estimate_bytes(int64_t k, const HostGrid& g) const;

  private:
    static constexpr int64_t DENSE_CAP = 8 * TASK_CAP;   // child scores per scoring launch
    int score_launch(int mode, const std::vector<Seg>* segs, int64_t n_slices, int64_t n_tasks);
    int score_overflow();
    cudaError_t launch_select(cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond);
    cudaError_t launch_compact(cudaStream_t s, bool pdl = false);
    cudaError_t launch_group(cudaStream_t s, bool pdl = false);
    int read_ctl();
    int upload_cap();
    int grow_frontier();
    int grow_to(int64_t need, int live, int64_t n);
    int resume_grown(std::vector<int>* finished);
    void finish_never_live(std::vector<int>* finished);
    void mark_finished(std::vector<int>* finished);
    int build_graph();
    cudaError_t capture_body(cudaGraph_t body, cudaGraphConditionalHandle cond, bool pdl);
    int upload_slot(int slot);
    int release(int slot);
    template <class T>
    int slot_get(SearchHost& h, T** p, size_t n);

    cudaStream_t st_;
    int max_slots_;
    bool timed_;
    int64_t fcap_;                 // frontier capacity (nodes, all searches)
    int64_t max_nodes_ = 0;        // the run's frontier limit: the capacity may grow to this
    int64_t cap_eff_ = 0;          // nodes the run may hold: min(fcap_, max_nodes_)
    Tuning tune_;                  // launch shape of this run
    size_t fixed_bytes_ = 0;
    FrontDev front_{};
    LoopState* d_ls_ = nullptr;
    SearchDev* d_S_ = nullptr;
    Ctl* d_ctl_ = nullptr;
    NodeRec* parents_ = nullptr;   // popped nodes of a round (per search at poff)
    int64_t* pfirst_ = nullptr;    // first task of each popped node
    TaskRec* tasks_ = nullptr;     // the launch's tasks
    int32_t* tscore_ = nullptr;    // each task's parent score (the bound check of finalize)
    int32_t* pscore_ = nullptr;    // each popped node's score (tasks expanded in windows)
    GroupDev grp_{};               // rotation groups of a round scored in one launch
    uint32_t* cdone_ = nullptr;    // the compaction's finished CTAs (its last one scans a one-slot round's groups)
    int64_t* d_poff_ = nullptr;
    int64_t* d_toff_ = nullptr;
    unsigned long long* d_pcnt_ = nullptr;
    unsigned long long* d_tcnt_ = nullptr;
    int32_t* d_slots_ = nullptr;
    int32_t* dense_ = nullptr;
    Ctl* h_ctl_ = nullptr;         // pinned
    int64_t* h_off_ = nullptr;     // pinned: parent and task offsets of an overflowing round
    int32_t* h_misc_ = nullptr;    // pinned: plan status, loop iterations
    Ctl* h_zero_ = nullptr;        // pinned, all zero
    int* h_wake_ = nullptr;        // pinned and mapped: the device loop's wake-up flag
    int* d_wake_ = nullptr;        // its device address
    bool exit_on_finish_ = false;
    Plan* d_plan_ = nullptr;
    Plan h_plan_{};
    int nsm_ = 152;
    cudaGraphExec_t exec_ = nullptr;
    bool graph_bytes_ = false;     // the graph's scoring kernel is the byte-grid-only variant
    bool graph_pdl_ = true;        // capture the loop body with programmatic dependent launches
    bool bytes_only() const;
    bool host_driven_ = false;
    std::vector<void*> fixed_;
    std::vector<SearchHost> hosts_;
    std::vector<cudaEvent_t> evs_;
    std::vector<int64_t> ev_units_;   // units (tasks x scan points) of each timed scoring launch
    double score_ms_ = 0.0;
    int64_t launches_ = 0, score_launches_ = 0;
    int64_t grown_ = 0;            // times the frontier arrays grew
};

}  // namespace bbs
