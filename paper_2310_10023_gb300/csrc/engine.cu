// engine.cu -- device-resident batched best-first BnB (Sec. III-E,
// Algorithm 2) for one or many searches at once.
//
// Every search keeps its frontier F as per-score bucket counts (nodes,
// children, leaves per integer score, K + 1 buckets) over node records that
// all searches share: two arrays of (node, score | search << 24) that swap
// roles every iteration.
//
// One iteration advances every live search by one canonical batch:
//   select   (1 CTA per search) walk the buckets from the top with a block-wide
//            prefix of their children counts: the first bucket s* reached with
//            children >= b stops; one at or below best clears F; one holding a
//            leaf sets best = s* and clears F (its lexmin leaf is the match);
//            buckets above s* pop.  The last CTA to finish plans the round: the
//            parent and task ranges of every search and the scoring launch's
//            slice map; it ends the device loop when the round is empty or too
//            large for one launch, or after the iteration cap.
//   compact  the current node array: popped nodes become parents and join
//            their rotation group (parents of one level and rotation share
//            their rotational children), kept ones move to the other array,
//            cleared ones go; a popped leaf bucket's leaves give the lexmin key
//   groups   each group its task range, then the task records (the
//            rotational children) written so that one child rotation's tasks
//            are consecutive
//   score    (branch.cu) every child of every task (the kernel forms a run's
//            rotation rows once for the tasks that share them); then the
//            lexmin rotation of a popped leaf bucket, and survivors above best
//            appended to the other array with their bucket counts
// Only popping a leaf changes a search's best, so how its batch is split into
// launches, and which other searches share them, cannot change its result;
// node order inside F is free.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "engine.cuh"

namespace bbs {

// ---- block helpers (blocks of whole warps) ----------------------------------

// Exclusive block prefix sums of N values at once (two barriers); totals in
// `total`.  sh holds 32 * N values; the caller synchronizes before reusing it.
template <int N>
__device__ __forceinline__ void block_excl_scan_n(const int64_t (&v)[N], int64_t (&before)[N], int64_t (&total)[N],
                                                  int64_t* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (int)(blockDim.x >> 5);
    int64_t x[N];
#pragma unroll
    for (int k = 0; k < N; ++k) x[k] = v[k];
    for (int o = 1; o < 32; o <<= 1)
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x[k], o);
            if (lane >= o) x[k] += y;
        }
    if (lane == 31)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[32 * k + wid] = x[k];
    __syncthreads();
    if (wid == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) {
            int64_t t = lane < nw ? sh[32 * k + lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            sh[32 * k + lane] = t;
        }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) {
        before[k] = (wid > 0 ? sh[32 * k + wid - 1] : 0) + x[k] - v[k];
        total[k] = sh[32 * k + nw - 1];
    }
}

// ---- launch shape ---------------------------------------------------------------

namespace {
std::mutex g_tuning_mu;
Tuning g_tuning;
thread_local LaunchLog g_launch_log;
}  // namespace

LaunchLog& launch_log() { return g_launch_log; }

Tuning current_tuning()
{
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    return g_tuning;
}

int set_tuning(const bbs_tuning* t)
{
    Tuning v;
    if (t) {
        if (t->launch_tasks) v.launch_tasks = t->launch_tasks;
        if (t->static_pm) v.static_pm = t->static_pm;
        if (t->grab_min) v.grab_min = t->grab_min;
        if (t->ctas_per_sm) v.ctas_per_sm = t->ctas_per_sm;
        if (t->frontier_log2) v.frontier_log2 = t->frontier_log2;
        if (v.frontier_log2 && (v.frontier_log2 < 10 || v.frontier_log2 > 30))
            return set_error(BBS_EINVAL, "tuning: frontier_log2 %d outside 10..30", v.frontier_log2);
        if (v.launch_tasks < 1 || v.launch_tasks > TASK_CAP)
            return set_error(BBS_EINVAL, "tuning: launch_tasks %lld outside 1..%lld", (long long)v.launch_tasks,
                             (long long)TASK_CAP);
        if (v.static_pm < 1 || v.static_pm > 1000) return set_error(BBS_EINVAL, "tuning: static_pm %d outside 1..1000", v.static_pm);
        if (v.grab_min < 1 || v.grab_min > (1 << 20)) return set_error(BBS_EINVAL, "tuning: grab_min %d outside 1..2^20", v.grab_min);
        if (v.ctas_per_sm < 1 || v.ctas_per_sm > BRANCH_CTAS_PER_SM)
            return set_error(BBS_EINVAL, "tuning: ctas_per_sm %d outside 1..%d", v.ctas_per_sm, BRANCH_CTAS_PER_SM);
    }
    std::lock_guard<std::mutex> lock(g_tuning_mu);
    g_tuning = v;
    return BBS_OK;
}

// ---- kernels -----------------------------------------------------------------

__device__ __forceinline__ unsigned long long gtimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Holds the stream until the host has enqueued a timed scoring launch behind
// it, so that the launch's opening event fires right before the kernel starts
// instead of while the host is still submitting it.  The wait is bounded (at
// most about 20 ms): past it the gate records the overrun in *err and lets the
// stream go, which only lengthens that launch's measured time.
__global__ void timing_gate_kernel(const volatile int* open, int* err)
{
    for (int i = 0; i < 200000; ++i) {
        if (*open) return;
        __nanosleep(100);
    }
    *err = 1;
}

// reset the bucket arrays of one search (blockIdx.x = slot in `slots`)
__global__ void slot_init_kernel(SearchDev* S, const int32_t* slots)
{
    SearchDev& s = S[slots[blockIdx.x]];
    if (threadIdx.x == 0) s.ctl->t_start_ns = gtimer_ns();
    for (int i = threadIdx.x; i <= s.K; i += blockDim.x) {
        s.b_cnt[i] = 0;
        s.b_kids[i] = 0;
        s.b_leaf[i] = 0;
    }
}

// Selection (1 CTA per slot) and, in the last CTA to finish, the plan of the
// round: per-search parent / task offsets and one task run per search.
__global__ void __launch_bounds__(1024) select_kernel(SearchDev* S, int nslots, Plan* P, LoopState* LS,
                                                      int64_t* poff, int64_t* toff, unsigned long long* pcnt,
                                                      unsigned long long* tcnt, cudaGraphConditionalHandle cond,
                                                      int use_cond, Tuning tune, const volatile int* wake)
{
    pdl_wait();   // the previous iteration's survivors and bucket counts are in
    pdl_trigger();
    __shared__ int64_t sh[32 * 4];
    __shared__ int s_first;
    __shared__ int32_t s_star, s_reason;
    __shared__ int64_t s_cnt, s_kids;
    __shared__ int s_last;
    const int tid = threadIdx.x;
    for (int si = blockIdx.x; si < nslots; si += gridDim.x) {
        SearchDev& f = S[si];
        Ctl* c = f.ctl;
        if (!c->active || c->err) continue;   // uniform
        if (c->done) {   // finished earlier: nothing of it takes part in this round
            if (tid == 0) c->match_changed = 0;
            continue;
        }
        const int32_t best = c->best;
        if (tid == 0) {
            s_star = -1;
            s_reason = c->size > 0 ? 4 : 0;
        }
        __syncthreads();
        // 1. the bucket where popping stops, walking down from the top: the
        // buckets passed are the popped ones, emptied on the way
        int64_t carry = 0, ncarry = 0;
        const int32_t top = c->top;
        for (int base = top; base >= 0; base -= blockDim.x) {
            const int s = base - tid;
            int64_t cnt = 0, kids = 0, leaf = 0;
            if (s >= 0) {   // three independent loads
                cnt = (int64_t)f.b_cnt[s];
                kids = (int64_t)f.b_kids[s];
                leaf = (int64_t)f.b_leaf[s];
            }
            const bool have = cnt > 0;
            if (!have) kids = 0;
            if (tid == 0) s_first = (int)blockDim.x;
            // prefixes of the children and node counts from the top
            const int64_t v2[2] = {kids, cnt};
            int64_t ex[2], tot[2];
            block_excl_scan_n<2>(v2, ex, tot, sh);
            const int64_t cum = carry + ex[0];
            const bool stop = have && (cum >= f.batch || s <= best || leaf > 0);
            if (stop) atomicMin(&s_first, tid);
            __syncthreads();
            const int first = s_first;
            if (first < (int)blockDim.x) {
                if (tid == first) {
                    s_star = s;
                    s_reason = cum >= f.batch ? 1 : (s <= best ? 2 : 3);
                    s_kids = cum;               // children of the buckets above s*
                    s_cnt = ncarry + ex[1];     // and their nodes
                }
                if (have && tid < first) {
                    f.b_cnt[s] = 0;
                    f.b_kids[s] = 0;
                    f.b_leaf[s] = 0;
                }
                __syncthreads();
                break;
            }
            if (have) {   // the whole pass is above the stop bucket: popped
                f.b_cnt[s] = 0;
                f.b_kids[s] = 0;
                f.b_leaf[s] = 0;
            }
            carry += tot[0];
            ncarry += tot[1];
            __syncthreads();   // s_first and sh read before the next pass
        }
        if (tid == 0 && s_star < 0) {   // no stop: every bucket popped
            s_kids = carry;
            s_cnt = ncarry;
        }
        __syncthreads();
        const int32_t sstar = s_star;
        const int reason = s_reason;
        const bool clear = reason == 2 || reason == 3;
        // 2. when clearing, every bucket at or below s* empties as well
        if (clear)
            for (int s = tid; s <= sstar; s += blockDim.x) {
                f.b_cnt[s] = 0;
                f.b_kids[s] = 0;
                f.b_leaf[s] = 0;
            }
        const int64_t tnp = s_cnt, tpk = s_kids;

        if (tid == 0) {
            const int64_t size = c->size;
            if (size > c->peak) c->peak = size;
            c->sstar = sstar;
            c->clear = clear ? 1 : 0;
            c->reason = reason;
            c->n_parents = tnp;
            c->n_tasks = tpk / 8;
            c->popped_kids = tpk;
            c->size = clear ? 0 : size - tnp;
            c->top = reason == 1 ? sstar : -1;
            c->match_changed = 0;
            const unsigned long long now = gtimer_ns();
            if (reason == 3) {
                c->best = sstar;
                c->found = 1;
                c->match_changed = 1;
                c->lex_t = ~0ull;
                c->lex_r = ~0u;
                c->t_match_ns = now;
            }
            c->done = tnp == 0;
            if (tnp > 0) {
                c->st_iters += 1;
                c->st_parents += tnp;
                c->st_nodes += tpk;
                c->st_gathers += (tpk / 8) * (int64_t)f.K;
            }
            if (c->done) c->t_end_ns = now;
        }
        __syncthreads();
    }
    // the last CTA to finish plans the round (a single CTA plans at once)
    if (gridDim.x > 1) {
        __threadfence();
        if (tid == 0) s_last = atomicAdd(&LS->select_done, 1u) == gridDim.x - 1;
        __syncthreads();
        if (!s_last) return;
        __threadfence();
    }
    int64_t cp = 0, ct = 0, cs = 0, cn = 0;
    int any3 = 0, anyfin = 0;
    for (int base = 0; base < nslots; base += blockDim.x) {
        const int s = base + tid;
        int64_t np = 0, nt = 0, sl = 0, has = 0;
        int32_t best = 0;
        if (s < nslots) {
            const Ctl* c = S[s].ctl;
            best = c->best;
            if (c->active && !c->done && !c->err) {
                np = c->n_parents;
                nt = c->n_tasks;
            }
            // a leaf bucket popped in this round (the search may have finished with it)
            if (c->active && !c->err && c->match_changed) any3 = 1;
            if (c->active && (c->done || c->err)) anyfin = 1;
            sl = nt * S[s].nblk;
            has = nt > 0;
            pcnt[s] = 0;
            tcnt[s] = 0;
        }
        const int64_t v4[4] = {np, nt, sl, has};
        int64_t ex4[4], tot4[4];
        block_excl_scan_n<4>(v4, ex4, tot4, sh);
        const int64_t ep = ex4[0], et = ex4[1], es = ex4[2], en = ex4[3];
        const int64_t tp = tot4[0], tt = tot4[1], ts = tot4[2], tn = tot4[3];
        if (s < nslots) {
            poff[s] = cp + ep;
            toff[s] = ct + et;
            const int64_t si = cn + en;
            if (has && si < MAXSEG) {
                Seg& g = P->seg[si];
                g.first_parent = cp + ep;
                g.first_task = ct + et;
                g.n_tasks = nt;
                g.first_slice = cs + es;
                g.sid = s;
                g.nblk = S[s].nblk;
                g.R = 0;
                g.best = best;
            }
        }
        cp += tp;
        ct += tt;
        cs += ts;
        cn += tn;
        __syncthreads();   // sh read before the next pass
    }
    any3 = __syncthreads_or(any3);
    anyfin = __syncthreads_or(anyfin);
    if (tid == 0) {
        P->nseg = (int32_t)(cn < MAXSEG ? cn : MAXSEG);
        P->n_slices = cs;
        P->n_tasks = ct;
        P->n_parents = cp;
        P->next_slice = 0;
        P->static_pm = tune.static_pm;
        P->grab_min = tune.grab_min;
        P->mode = MODE_SEARCH;
        int st = PLAN_OK;
        if (cp == 0) st = PLAN_EMPTY;
        else if (cn > MAXSEG || ct > tune.launch_tasks) st = PLAN_OVERFLOW;
        P->status = st;
        // the other array receives the kept nodes (at most the current ones)
        // and the survivors (at most 8 per task): grow first when that may not fit
        const int64_t need = (int64_t)min(LS->fn[1 - LS->cur], (unsigned long long)LS->cap) + 8 * ct;
        P->grow = (st != PLAN_EMPTY && need > LS->cap) ? 1 : 0;
        LS->grow_need = need;
        P->iters += 1;
        // the nodes the last round appended become current; the other array
        // receives the kept and the new nodes
        const int cur = 1 - LS->cur;
        LS->cur = cur;
        LS->fn[1 - cur] = 0;
        LS->lex_pass = any3;
        LS->select_done = 0;
        // the device loop ends with an empty or oversized round, after its
        // iteration cap, when the host asks (wake), or, for the server, when a
        // search finished or failed (its result is reported at once)
        const bool stop = st != PLAN_OK || P->grow || P->iters >= P->max_iters || (LS->exit_on_finish && anyfin) ||
                          *wake != 0;
        if (use_cond && stop) cudaGraphSetConditional(cond, 0);
    }
}

// the tasks (rotational children, Eq. (13)) of parent nd for t in [t0, t1),
// written at tasks[dst + t * stride]: translation and rl (the scoring kernel
// forms the rows)
__device__ __forceinline__ void write_tasks(const DevGrid& g, const NodeRec& nd, const int32_t lo[3],
                                            const int32_t ext[3], int32_t t0, int32_t t1, TaskRec* tasks, int64_t dst,
                                            int32_t* tscore, int32_t pscore, int64_t stride = 1)
{
    const int l = rl_level(nd.rl);
    const int64_t nb = g.N[l - 1][1], ng = g.N[l - 1][2];
    int32_t t = 0;
    for (int32_t ja = 0; ja < ext[0]; ++ja)
        for (int32_t jb = 0; jb < ext[1]; ++jb)
            for (int32_t jg = 0; jg < ext[2]; ++jg, ++t) {
                if (t < t0 || t >= t1) continue;
                const uint32_t crot = (uint32_t)(((int64_t)(lo[0] + ja) * nb + (lo[1] + jb)) * ng + (lo[2] + jg));
                const int64_t at = dst + t * stride;
                TaskRec& r = tasks[at];
                r.tx = 2 * nd.cx;
                r.ty = 2 * nd.cy;
                r.tz = 2 * nd.cz;
                r.rl = rl_pack(crot, l - 1);
                tscore[at] = pscore;
            }
}

// ---- rotation groups of a round -------------------------------------------
//
// The parents a round pops that share their level and rotation have the
// same rotational children (Eq. (13)): their tasks share rotations and
// differ in translation only.  A round that scores in one launch lays its
// tasks out by group so that the scoring kernel rotates a chunk of the scan
// once for all tasks of one rotation: group G of a search (P_G parents,
// T_G rotational children each) holds tasks goff[G] + j P_G + i for child
// rotation j and the group's parent i.  Groups are found by open addressing
// over (search, rl) keys, the entry naming the group: compact_kernel joins
// each parent to its group (one insert and one count per group and warp);
// group_scan_search gives each search's groups their task ranges (in the
// search's range at toff) and empties their entries -- in the compaction's
// last CTA for a one-slot engine, else in group_scan_kernel;
// emit_tasks_kernel writes the task records.

__device__ __forceinline__ uint32_t group_hash(unsigned long long key)
{
    key ^= key >> 29;
    key *= 0xBF58476D1CE4E5B9ull;
    key ^= key >> 32;
    return (uint32_t)key;
}

// The table entry of key (search sid, rl) with T rotational children per
// parent, inserted if absent; the thread that inserts it lists it among the
// search's groups (list at g0 + ngrp[sid]).  The table has twice the
// launch's task capacity in entries, a round at most that many parents: an
// empty entry is always found.  GROUP_TABLE on failure (cannot happen).
__device__ uint32_t group_entry(const GroupDev& G, int sid, uint32_t rl, int32_t T, int64_t g0)
{
    const unsigned long long key = ((unsigned long long)sid << 32) | rl;
    uint32_t h = group_hash(key) & (uint32_t)(GROUP_TABLE - 1);
    for (int64_t probe = 0; probe < GROUP_TABLE; ++probe) {
        unsigned long long v = *(volatile unsigned long long*)&G.tab[h];
        if (v == GROUP_EMPTY) {
            v = atomicCAS(&G.tab[h], GROUP_EMPTY, key);
            if (v == GROUP_EMPTY) {   // this thread created the group
                G.ntask[h] = (uint32_t)T;
                const uint32_t k = atomicAdd(&G.ngrp[sid], 1u);
                if (g0 + k >= TASK_CAP) return (uint32_t)GROUP_TABLE;
                G.list[g0 + k] = h;
                return h;
            }
        }
        if (v == key) return h;
        h = (h + 1) & (uint32_t)(GROUP_TABLE - 1);
    }
    return (uint32_t)GROUP_TABLE;
}

// One search's groups (by the calling CTA): their task ranges in the
// search's range at toff (exclusive scan of P_G T_G in group-id order), their
// parent counts for the emission, and their entries emptied for the next
// round; the sum is checked against the search's task count.
__device__ void group_scan_search(SearchDev* S, int si, const int64_t* __restrict__ poff,
                                  const int64_t* __restrict__ toff, const GroupDev& G, int64_t* sh)
{
    const int tid = threadIdx.x;
    const uint32_t ng = G.ngrp[si];   // uniform
    if (ng == 0) return;
    const int64_t g0 = poff[si];
    int64_t run = toff[si];
    for (uint32_t base = 0; base < ng; base += blockDim.x) {
        const uint32_t g = base + tid;
        int64_t v[1] = {0}, ex[1], tot[1];
        uint32_t h = 0, cnt = 0;
        const bool have = g < ng && g0 + g < TASK_CAP;   // ids past the list's end were never listed
        if (have) {
            h = G.list[g0 + g];
            cnt = G.cnt[h];
            v[0] = (int64_t)cnt * G.ntask[h];
        }
        block_excl_scan_n<1>(v, ex, tot, sh);
        if (have) {
            G.off[h] = run + ex[0];
            G.np[h] = cnt;
            G.cnt[h] = 0;
            G.tab[h] = GROUP_EMPTY;
        }
        run += tot[0];
        __syncthreads();   // sh read before the next pass
    }
    if (tid == 0) {
        G.ngrp[si] = 0;
        Ctl* c = S[si].ctl;
        if (run != toff[si] + c->n_tasks) atomicOr(&c->err, 4);   // groups disagree with the round
    }
}

// One CTA per search slot: group_scan_search of each (engines with several
// slots; a one-slot engine's compaction does it in its last CTA).
__global__ void __launch_bounds__(1024) group_scan_kernel(SearchDev* S, int nslots, const Plan* P,
                                                          const int64_t* __restrict__ poff,
                                                          const int64_t* __restrict__ toff, GroupDev G)
{
    pdl_wait();   // the compaction's groups are in
    pdl_trigger();
    if (P->status != PLAN_OK || P->grow) return;
    __shared__ int64_t sh[32];
    for (int si = blockIdx.x; si < nslots; si += gridDim.x) group_scan_search(S, si, poff, toff, G, sh);
}

// the segment holding parent pi of a device-planned round (segments in parent order)
__device__ __forceinline__ int find_parent_seg(const Plan* P, int64_t pi)
{
    int lo = 0, hi = P->nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P->seg[mid].first_parent <= pi) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The task records of a round that scores in one launch, by group: parent i
// of group G writes its child rotation j at goff[G] + j P_G + i.
__global__ void __launch_bounds__(256) emit_tasks_kernel(SearchDev* S, const Plan* P,
                                                         const NodeRec* __restrict__ parents,
                                                         const int32_t* __restrict__ pscore, GroupDev G,
                                                         TaskRec* __restrict__ tasks, int32_t* __restrict__ tscore)
{
    pdl_wait();   // the groups' task ranges are in
    pdl_trigger();
    if (P->status != PLAN_OK || P->grow) return;
    const int64_t np = min(P->n_parents, TASK_CAP);
    for (int64_t pi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; pi < np; pi += (int64_t)gridDim.x * blockDim.x) {
        const Seg& g = P->seg[find_parent_seg(P, pi)];
        const NodeRec nd = parents[pi];
        const DevGrid& dg = S[g.sid].grid;
        int32_t lo[3], ext[3];
        const int32_t T = rot_children(dg, rl_level(nd.rl), rl_rot(nd.rl), lo, ext);
        const uint32_t h = G.pslot[pi];
        if (T <= 0 || h >= (uint32_t)GROUP_TABLE) continue;
        const int64_t first = G.off[h] + G.pidx[pi], stride = (int64_t)G.np[h];
        if (first < 0 || first + (int64_t)(T - 1) * stride >= P->n_tasks) {   // groups disagree with the round
            atomicOr(&S[g.sid].ctl->err, 4);
            continue;
        }
        write_tasks(dg, nd, lo, ext, 0, T, tasks, first, tscore, pscore[pi], stride);
    }
}

// The current node array after select: popped nodes become the round's
// parents (their first task in pfirst) and, when the round scores in one
// launch, join their rotation's group (group_entry; emit_tasks_kernel
// writes the task records); kept nodes move to the other array; cleared
// nodes, and those of failed or released searches, go.  Leaves of a popped
// leaf bucket take part in the first lexmin pass (smallest translation key).
__global__ void __launch_bounds__(256) compact_kernel(SearchDev* S, FrontDev F, LoopState* LS, const Plan* P,
                                                      NodeRec* __restrict__ parents, int64_t* __restrict__ pfirst,
                                                      int32_t* __restrict__ pscore, const int64_t* __restrict__ poff,
                                                      const int64_t* __restrict__ toff, unsigned long long* pcnt,
                                                      unsigned long long* tcnt, GroupDev G, int nslots,
                                                      int scan_here, uint32_t* done)
{
    pdl_wait();   // select's round plan is in
    pdl_trigger();
    if (P->grow) return;   // the round waits for the host to grow the frontier
    const int cur = LS->cur, nxt = 1 - cur;
    // appends past the capacity were not stored (their searches failed): the
    // count is clamped wherever it is read
    const int64_t n = min((int64_t)LS->fn[cur], LS->cap);
    const bool emit = P->status == PLAN_OK;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_round = (n + 31) & ~(int64_t)31;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
        bool keep = false, popped = false;
        uint32_t key = 0;
        int32_t score = 0;
        int sid = 0;
        int32_t T = 0, lo[3], ext[3];
        NodeRec nd;
        nd.cx = nd.cy = nd.cz = 0;
        nd.rl = 0;
        Ctl* c = nullptr;
        if (i < n) {
            key = F.keys[cur][i];
            nd = F.nodes[cur][i];
            sid = (int)(key >> 24);
            score = (int32_t)(key & 0xFFFFFFu);
            SearchDev& f = S[sid];
            c = f.ctl;
            if (c->active && !c->err) {
                const int32_t sstar = c->sstar;
                if (score > sstar) {
                    popped = true;
                    T = rot_children(f.grid, rl_level(nd.rl), rl_rot(nd.rl), lo, ext);
                } else {
                    keep = !c->clear;
                    if (c->reason == 3 && score == sstar && rl_level(nd.rl) == 0)
                        atomicMin(&c->lex_t, lex_translation(nd));
                }
            }
        }
        // popped nodes: a parent index and a task range each, from the search's
        // counters; one atomic per warp when the warp's popped nodes share a search
        const uint32_t pball = __ballot_sync(0xffffffffu, popped);
        if (pball) {
            int32_t incl = popped ? T : 0;   // inclusive warp scan of the task counts
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int lead = __ffs(pball) - 1;
            const int lead_sid = __shfl_sync(0xffffffffu, sid, lead);
            const bool one = __all_sync(0xffffffffu, !popped || sid == lead_sid);
            unsigned long long p = 0, t0 = 0;
            if (one) {   // warp-uniform
                const int32_t tsum = __shfl_sync(0xffffffffu, incl, 31);
                unsigned long long pb = 0, tb = 0;
                if (lane == lead) {
                    pb = atomicAdd(&pcnt[sid], (unsigned long long)__popc(pball));
                    tb = atomicAdd(&tcnt[sid], (unsigned long long)tsum);
                }
                pb = __shfl_sync(0xffffffffu, pb, lead);
                tb = __shfl_sync(0xffffffffu, tb, lead);
                p = pb + __popc(pball & ((1u << lane) - 1u));
                t0 = tb + (unsigned long long)(incl - (popped ? T : 0));
            } else if (popped) {
                p = atomicAdd(&pcnt[sid], 1ull);
                t0 = T ? atomicAdd(&tcnt[sid], (unsigned long long)T) : 0ull;
            }
            bool grouping = false;
            int64_t pi = 0;
            if (popped) {
                if ((int64_t)p < c->n_parents && (int64_t)(t0 + T) <= c->n_tasks) {
                    pi = poff[sid] + (int64_t)p;
                    parents[pi] = nd;
                    pfirst[pi] = toff[sid] + (int64_t)t0;
                    pscore[pi] = score;
                    grouping = emit && T > 0 && pi < TASK_CAP;
                } else {
                    atomicOr(&c->err, 4);   // bucket counts disagree with the nodes: fail the search
                }
            }
            // rotation groups: the warp's parents of one key join with one insert and one count
            const unsigned long long gkey = grouping ? (((unsigned long long)sid << 32) | nd.rl) : GROUP_EMPTY;
            const uint32_t peers = __match_any_sync(0xffffffffu, gkey);
            const int gl = __ffs(peers) - 1;
            uint32_t h = 0, gbase = 0;
            if (grouping && lane == gl) {
                h = group_entry(G, sid, nd.rl, T, poff[sid]);
                if (h < (uint32_t)GROUP_TABLE) gbase = atomicAdd(&G.cnt[h], (uint32_t)__popc(peers));
            }
            h = __shfl_sync(0xffffffffu, h, gl);
            gbase = __shfl_sync(0xffffffffu, gbase, gl);
            if (grouping) {
                if (h < (uint32_t)GROUP_TABLE) {
                    G.pslot[pi] = h;
                    G.pidx[pi] = gbase + __popc(peers & ((1u << lane) - 1u));
                } else {
                    atomicOr(&c->err, 4);   // more groups than parents: cannot happen
                }
            }
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, keep);
        if (!ball) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&LS->fn[nxt], (unsigned long long)__popc(ball));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) {
            const unsigned long long pos = base + __popc(ball & ((1u << lane) - 1u));
            F.nodes[nxt][pos] = nd;
            F.keys[nxt][pos] = key;
        }
    }
    // a one-slot engine: the last CTA to finish gives the groups their task
    // ranges (the launch the group scan kernel would take is saved)
    if (scan_here && emit) {   // uniform
        __shared__ int s_last;
        __shared__ int64_t sh[32];
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(done, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (int si = 0; si < nslots; ++si) group_scan_search(S, si, poff, toff, G, sh);
            if (threadIdx.x == 0) *done = 0u;
        }
    }
}

// the tasks [ga, gb) of one search's round (gathered parents [p0, p1), their
// first tasks in pfirst) -> tasks[la ..]: a round scored in several launches
__global__ void expand_kernel(const SearchDev* S, int sid, const NodeRec* __restrict__ parents,
                              const int64_t* __restrict__ pfirst, const int32_t* __restrict__ pscore, int64_t p0,
                              int64_t p1, int64_t ga, int64_t gb, int64_t la, TaskRec* __restrict__ tasks,
                              int32_t* __restrict__ tscore)
{
    const DevGrid& g = S[sid].grid;
    for (int64_t p = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < p1; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = pfirst[p];
        if (b >= gb) continue;
        const NodeRec nd = parents[p];
        int32_t lo[3], ext[3];
        const int32_t T = rot_children(g, rl_level(nd.rl), rl_rot(nd.rl), lo, ext);
        if (b + T <= ga) continue;
        const int32_t t0 = (int32_t)(ga > b ? ga - b : 0), t1 = (int32_t)(gb < b + T ? gb - b : T);
        write_tasks(g, nd, lo, ext, t0, t1, tasks, la + b - ga, tscore, pscore[p]);
    }
}

// Removing the nodes of one slot (a search stopped early): the incoming array
// 1 - cur is copied, without them, into array cur, which then becomes the
// incoming one.  Three launches: reset the target, copy, swap.
__global__ void purge_reset_kernel(LoopState* LS) { LS->fn[LS->cur] = 0; }

__global__ void purge_kernel(FrontDev F, LoopState* LS, int slot)
{
    const int in = 1 - LS->cur, out = LS->cur;
    const int64_t n = min((int64_t)LS->fn[in], LS->cap);   // appends past the capacity were not stored
    const int lane = threadIdx.x & 31;
    const int64_t n_round = (n + 31) & ~(int64_t)31;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_round; i += (int64_t)gridDim.x * blockDim.x) {
        bool keep = false;
        uint32_t key = 0;
        NodeRec nd;
        if (i < n) {
            key = F.keys[in][i];
            nd = F.nodes[in][i];
            keep = (int)(key >> 24) != slot;
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, keep);
        if (!ball) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&LS->fn[out], (unsigned long long)__popc(ball));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (keep) {
            const unsigned long long pos = base + __popc(ball & ((1u << lane) - 1u));
            F.nodes[out][pos] = nd;
            F.keys[out][pos] = key;
        }
    }
}

__global__ void purge_swap_kernel(LoopState* LS) { LS->cur = 1 - LS->cur; }

// ---- host engine ---------------------------------------------------------------

namespace {

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int64_t floor_div2(int64_t x) { return x >= 0 ? x / 2 : -((-x + 1) / 2); }

}  // namespace

Engine::Engine(cudaStream_t st, int max_slots, int64_t pool_nodes, bool timed)
    : st_(st), max_slots_(max_slots), timed_(timed), fcap_(pool_nodes), tune_(current_tuning())
{
    hosts_.resize((size_t)max_slots);
}

Engine::~Engine()
{
    for (size_t i = 0; i < hosts_.size(); ++i)
        if (hosts_[i].used) release((int)i);
    if (exec_) cudaGraphExecDestroy(exec_);
    for (void* p : fixed_) cudaFreeAsync(p, st_);
    for (cudaEvent_t e : evs_) cudaEventDestroy(e);
    if (h_ctl_) cudaFreeHost(h_ctl_);
    if (h_off_) cudaFreeHost(h_off_);
    if (h_misc_) cudaFreeHost(h_misc_);
    if (h_zero_) cudaFreeHost(h_zero_);
    if (h_wake_) cudaFreeHost(h_wake_);
}

int Engine::init()
{
    auto get = [&](auto** p, size_t n) -> int {
        using T = typename std::remove_pointer<typename std::remove_reference<decltype(p)>::type>::type;
        void* q = nullptr;
        const size_t bytes = n * sizeof(**p) + 16;
        cudaError_t e = cudaMallocAsync(&q, bytes, st_);
        if (e != cudaSuccess)
            return set_error(BBS_ENOMEM, "engine: cudaMallocAsync(%zu bytes): %s", bytes, cudaGetErrorString(e));
        fixed_.push_back(q);
        fixed_bytes_ += bytes;
        *p = (T)q;
        return BBS_OK;
    };
    if (max_slots_ < 1 || max_slots_ > MAX_SLOTS)
        return set_error(BBS_EINVAL, "engine: %d slots (1..%d)", max_slots_, MAX_SLOTS);
    for (int b = 0; b < 2; ++b) {
        BBS_TRY(get(&front_.nodes[b], (size_t)fcap_));
        BBS_TRY(get(&front_.keys[b], (size_t)fcap_));
    }
    front_.cap = fcap_;
    BBS_TRY(get(&d_ls_, 1));
    BBS_TRY(get(&d_S_, (size_t)max_slots_));
    BBS_TRY(get(&d_ctl_, (size_t)max_slots_));
    BBS_TRY(get(&parents_, (size_t)fcap_));
    BBS_TRY(get(&pfirst_, (size_t)fcap_));
    BBS_TRY(get(&tasks_, (size_t)TASK_CAP));
    BBS_TRY(get(&tscore_, (size_t)TASK_CAP));
    BBS_TRY(get(&pscore_, (size_t)fcap_));
    BBS_TRY(get(&d_poff_, (size_t)max_slots_));
    BBS_TRY(get(&d_toff_, (size_t)max_slots_));
    BBS_TRY(get(&d_pcnt_, (size_t)max_slots_));
    BBS_TRY(get(&d_tcnt_, (size_t)max_slots_));
    BBS_TRY(get(&d_plan_, 1));
    BBS_TRY(get(&d_slots_, (size_t)max_slots_));
    BBS_TRY(get(&dense_, (size_t)DENSE_CAP));
    BBS_TRY(get(&grp_.tab, (size_t)GROUP_TABLE));
    BBS_TRY(get(&grp_.cnt, (size_t)GROUP_TABLE));
    BBS_TRY(get(&grp_.ntask, (size_t)GROUP_TABLE));
    BBS_TRY(get(&grp_.off, (size_t)GROUP_TABLE));
    BBS_TRY(get(&grp_.np, (size_t)GROUP_TABLE));
    BBS_TRY(get(&grp_.ngrp, (size_t)max_slots_));
    BBS_TRY(get(&grp_.list, (size_t)TASK_CAP));
    BBS_TRY(get(&grp_.pslot, (size_t)TASK_CAP));
    BBS_TRY(get(&grp_.pidx, (size_t)TASK_CAP));
    BBS_TRY(get(&cdone_, 1));
    BBS_CUDA_TRY(cudaMemsetAsync(d_ctl_, 0, sizeof(Ctl) * (size_t)max_slots_, st_));
    BBS_CUDA_TRY(cudaMemsetAsync(d_S_, 0, sizeof(SearchDev) * (size_t)max_slots_, st_));
    BBS_CUDA_TRY(cudaMemsetAsync(d_ls_, 0, sizeof(LoopState), st_));
    BBS_CUDA_TRY(cudaMemsetAsync(d_pcnt_, 0, sizeof(unsigned long long) * (size_t)max_slots_, st_));
    BBS_CUDA_TRY(cudaMemsetAsync(d_tcnt_, 0, sizeof(unsigned long long) * (size_t)max_slots_, st_));
    BBS_CUDA_TRY(cudaMemsetAsync(d_plan_, 0, sizeof(Plan), st_));

    BBS_CUDA_TRY(cudaMemsetAsync(dense_, 0, sizeof(int32_t) * (size_t)DENSE_CAP, st_));
    BBS_CUDA_TRY(cudaMemsetAsync(grp_.tab, 0xFF, sizeof(unsigned long long) * (size_t)GROUP_TABLE, st_));
    BBS_CUDA_TRY(cudaMemsetAsync(grp_.ngrp, 0, sizeof(uint32_t) * (size_t)max_slots_, st_));
    BBS_CUDA_TRY(cudaMemsetAsync(grp_.cnt, 0, sizeof(uint32_t) * (size_t)GROUP_TABLE, st_));
    BBS_CUDA_TRY(cudaMemsetAsync(cdone_, 0, sizeof(uint32_t), st_));
    BBS_CUDA_TRY(cudaMallocHost((void**)&h_ctl_, sizeof(Ctl) * (size_t)max_slots_));
    BBS_CUDA_TRY(cudaMallocHost((void**)&h_off_, 2 * sizeof(int64_t) * (size_t)max_slots_));
    BBS_CUDA_TRY(cudaMallocHost((void**)&h_misc_, 4 * sizeof(int32_t)));
    BBS_CUDA_TRY(cudaMallocHost((void**)&h_zero_, sizeof(Ctl)));
    BBS_CUDA_TRY(cudaHostAlloc((void**)&h_wake_, 4 * sizeof(int), cudaHostAllocMapped));
    h_wake_[0] = h_wake_[1] = h_wake_[2] = h_wake_[3] = 0;
    BBS_CUDA_TRY(cudaHostGetDevicePointer((void**)&d_wake_, h_wake_, 0));
    std::memset(h_ctl_, 0, sizeof(Ctl) * (size_t)max_slots_);
    std::memset(h_misc_, 0, 4 * sizeof(int32_t));
    std::memset(h_zero_, 0, sizeof(Ctl));
    {
        int dev = 0, nsm = 0;
        BBS_CUDA_TRY(cudaGetDevice(&dev));
        BBS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        if (nsm > 0) nsm_ = nsm;
    }
    // every slot's record points at its control block even while unused
    std::vector<SearchDev> blank((size_t)max_slots_);
    for (int i = 0; i < max_slots_; ++i) {
        std::memset(&blank[(size_t)i], 0, sizeof(SearchDev));
        blank[(size_t)i].ctl = d_ctl_ + i;
    }
    BBS_CUDA_TRY(cudaMemcpyAsync(d_S_, blank.data(), sizeof(SearchDev) * blank.size(), cudaMemcpyHostToDevice, st_));
    max_nodes_ = fcap_;
    BBS_TRY(upload_cap());
    BBS_CUDA_TRY(cudaStreamSynchronize(st_));   // the host copy above must outlive its transfer
    return BBS_OK;
}

int Engine::upload_cap()
{
    cap_eff_ = std::min(fcap_, max_nodes_);
    // pageable source: staged before the call returns
    BBS_CUDA_TRY(cudaMemcpyAsync(&d_ls_->cap, &cap_eff_, sizeof(int64_t), cudaMemcpyHostToDevice, st_));
    return BBS_OK;
}

int Engine::set_max_nodes(int64_t n)
{
    max_nodes_ = n;
    return upload_cap();
}

// A round whose survivors might not fit asked to grow the frontier arrays
// (select planned it; compaction, scoring and survivors waited).  The
// arrays double until they hold the round's need, within max_nodes_; the
// current nodes move over; the graph, captured with the old arrays, is
// rebuilt on the next iterate.  When the need is beyond max_nodes_ the round
// goes on as it is and the searches whose survivors do not fit fail alone.
// The round planned by the last select asked to grow the frontier arrays
// (compaction, scoring and survivors waited): grow to its need, then let
// the round go on.  The live nodes are in the array select made current.
int Engine::grow_frontier()
{
    LoopState ls;
    BBS_CUDA_TRY(cudaMemcpyAsync(&ls, d_ls_, sizeof(ls), cudaMemcpyDeviceToHost, st_));
    BBS_CUDA_TRY(cudaStreamSynchronize(st_));
    BBS_TRY(grow_to(ls.grow_need, ls.cur, (int64_t)ls.fn[ls.cur]));
    const int32_t zero = 0;
    BBS_CUDA_TRY(cudaMemcpyAsync(&d_plan_->grow, &zero, sizeof(zero), cudaMemcpyHostToDevice, st_));
    return BBS_OK;
}

// The frontier arrays double until they hold `need` nodes, within
// max_nodes_; the n live nodes of array `live` move over; the graph,
// captured with the old arrays, is rebuilt on the next iterate.  When the
// need is beyond max_nodes_ nothing changes: the searches whose survivors do
// not fit fail alone, as without growth.
int Engine::grow_to(int64_t need, int live, int64_t n)
{
    if (need <= cap_eff_ || need > max_nodes_) return BBS_OK;
    int64_t ncap = fcap_;
    while (ncap < need) ncap *= 2;
    if (ncap > max_nodes_) ncap = max_nodes_;
    std::vector<void*> fresh;
    size_t fresh_bytes = 0;
    auto get = [&](auto** p, size_t cnt) -> int {
        void* q = nullptr;
        const size_t bytes = cnt * sizeof(**p) + 16;
        const cudaError_t e = cudaMallocAsync(&q, bytes, st_);
        if (e != cudaSuccess) return set_error(BBS_ENOMEM, "engine: growing the frontier: %s", cudaGetErrorString(e));
        fresh.push_back(q);
        fresh_bytes += bytes;
        *p = (typename std::remove_reference<decltype(*p)>::type)q;
        return BBS_OK;
    };
    FrontDev nf = front_;
    NodeRec* np = nullptr;
    int64_t* nfirst = nullptr;
    int32_t* nscore = nullptr;
    int rc = BBS_OK;
    for (int b = 0; b < 2 && rc == BBS_OK; ++b) {
        rc = get(&nf.nodes[b], (size_t)ncap);
        if (rc == BBS_OK) rc = get(&nf.keys[b], (size_t)ncap);
    }
    if (rc == BBS_OK) rc = get(&np, (size_t)ncap);
    if (rc == BBS_OK) rc = get(&nfirst, (size_t)ncap);
    if (rc == BBS_OK) rc = get(&nscore, (size_t)ncap);
    if (rc != BBS_OK) {
        for (void* q : fresh) cudaFreeAsync(q, st_);
        return rc;
    }
    nf.cap = ncap;
    n = std::min<int64_t>(n, cap_eff_);   // appends past the run's cap were not stored
    BBS_CUDA_TRY(cudaMemcpyAsync(nf.nodes[live], front_.nodes[live], sizeof(NodeRec) * (size_t)n,
                                 cudaMemcpyDeviceToDevice, st_));
    BBS_CUDA_TRY(cudaMemcpyAsync(nf.keys[live], front_.keys[live], sizeof(uint32_t) * (size_t)n,
                                 cudaMemcpyDeviceToDevice, st_));
    // retire the old arrays (stream-ordered, after the copies)
    const void* old[7] = {front_.nodes[0], front_.keys[0], front_.nodes[1], front_.keys[1], parents_, pfirst_, pscore_};
    for (const void* q : old)
        for (size_t i = 0; i < fixed_.size(); ++i)
            if (fixed_[i] == q) {
                cudaFreeAsync(fixed_[i], st_);
                fixed_.erase(fixed_.begin() + (long)i);
                break;
            }
    for (void* q : fresh) fixed_.push_back(q);
    // each array was allocated with 16 bytes to spare (see init)
    const size_t per_node = 2 * (sizeof(NodeRec) + sizeof(uint32_t)) + sizeof(NodeRec) + sizeof(int64_t) + sizeof(int32_t);
    fixed_bytes_ = fixed_bytes_ + fresh_bytes - ((size_t)fcap_ * per_node + 7 * 16);
    front_ = nf;
    parents_ = np;
    pfirst_ = nfirst;
    pscore_ = nscore;
    fcap_ = ncap;
    BBS_TRY(upload_cap());
    if (exec_) {   // the captured graph holds the old arrays
        cudaGraphExecDestroy(exec_);
        exec_ = nullptr;
    }
    grown_ += 1;
    return BBS_OK;
}

// the rest of a round that waited for growth: compaction and the lexmin
// leaf, then the control blocks (the caller scores the round)
int Engine::resume_grown(std::vector<int>* finished)
{
    BBS_TRY(grow_frontier());
    BBS_CUDA_TRY(launch_compact(st_));
    BBS_CUDA_TRY(launch_group(st_));
    BBS_CUDA_TRY(launch_finalize(MODE_SEARCH, d_plan_, d_S_, tasks_, dense_, front_, d_ls_, nsm_ * 8, st_, true));
    launches_ += max_slots_ > 1 ? 4 : 3;
    BBS_CUDA_TRY(cudaGetLastError());
    BBS_TRY(read_ctl());
    mark_finished(finished);
    return BBS_OK;
}

// every search in use scores against byte-grid levels only
bool Engine::bytes_only() const
{
    bool any = false;
    for (const SearchHost& h : hosts_) {
        if (!(h.live || h.fresh) || !h.maps) continue;
        if (!maps_all_bytes(h.maps)) return false;
        any = true;
    }
    return any;
}

int Engine::begin_run(cudaStream_t st, bool timed)
{
    st_ = st;
    timed_ = timed;
    const Tuning t = current_tuning();
    if (!(t == tune_) && exec_) {   // the graph holds the launch shape it was captured with
        cudaGraphExecDestroy(exec_);
        exec_ = nullptr;
    }
    tune_ = t;
    score_ms_ = 0.0;
    launches_ = 0;
    score_launches_ = 0;
    for (cudaEvent_t e : evs_) cudaEventDestroy(e);
    evs_.clear();
    // a finished run leaves no nodes; start from empty arrays all the same
    BBS_CUDA_TRY(cudaMemsetAsync(d_ls_, 0, sizeof(LoopState), st_));
    exit_on_finish_ = false;
    max_nodes_ = fcap_;
    BBS_TRY(upload_cap());
    *h_wake_ = 0;
    h_misc_[2] = 0;
    return BBS_OK;
}

template <class T>
int Engine::slot_get(SearchHost& h, T** p, size_t n)
{
    void* q = nullptr;
    const size_t bytes = n * sizeof(T) + 16;
    cudaError_t e = cudaMallocAsync(&q, bytes, st_);
    if (e != cudaSuccess) return set_error(BBS_ENOMEM, "engine: cudaMallocAsync(%zu bytes): %s", bytes, cudaGetErrorString(e));
    h.bufs.push_back(q);
    h.bytes += bytes;
    *p = (T*)q;
    return BBS_OK;
}

size_t Engine::estimate_bytes(int64_t k, const HostGrid& g) const
{
    const size_t K1 = (size_t)k + 1;
    return sizeof(float4) * (size_t)(k > 0 ? k : 1) + sizeof(float4) * 3 * (size_t)g.nrot[g.levels - 1] +
           sizeof(double2) * (size_t)g.n_cs + 3 * sizeof(unsigned long long) * K1 + 1024;
}

int Engine::free_slot() const
{
    for (size_t i = 0; i < hosts_.size(); ++i)
        if (!hosts_[i].used) return (int)i;
    return -1;
}

int Engine::live_count() const
{
    int n = 0;
    for (const auto& h : hosts_) n += h.live ? 1 : 0;
    return n;
}

int Engine::used_count() const
{
    int n = 0;
    for (const auto& h : hosts_) n += h.used ? 1 : 0;
    return n;
}

int Engine::upload_slot(int i)
{
    SearchHost& h = hosts_[(size_t)i];
    h.dev.ctl = d_ctl_ + i;
    h_ctl_[i] = h.ctl0;
    BBS_CUDA_TRY(cudaMemcpyAsync(d_S_ + i, &h.dev, sizeof(SearchDev), cudaMemcpyHostToDevice, st_));
    BBS_CUDA_TRY(cudaMemcpyAsync(d_ctl_ + i, &h_ctl_[i], sizeof(Ctl), cudaMemcpyHostToDevice, st_));
    return BBS_OK;
}

int Engine::add(const bbs_maps* m, const float* xyz, int64_t k, int is_device, const bbs_ranges* rg,
                const bbs_opts* opts, uint64_t tag, int* slot)
{
    const int i = free_slot();
    if (i < 0) return set_error(BBS_EINVAL, "engine: all %d search slots are in use", max_slots_);
    SearchHost& h = hosts_[(size_t)i];
    h = SearchHost();
    h.used = true;
    h.tag = tag;
    h.t0 = now_ms();
    h.res.num_points = (int32_t)k;
    h.maps = m;
    *slot = i;
    const double frac = (opts && opts->score_frac > 0.0) ? opts->score_frac : 0.95;
    const uint32_t flags = opts ? opts->flags : 0u;
    int rc = BBS_OK;
    if (!(frac > 0.0 && frac <= 1.0)) rc = set_error(BBS_EINVAL, "localize: score_frac %g outside (0, 1]", frac);
    else if (flags & BBS_PRUNE_GE) rc = set_error(BBS_EINVAL, "localize: BBS_PRUNE_GE is not supported");
    else if (flags & BBS_SEARCH_DFS)
        rc = set_error(BBS_EINVAL, "localize: the depth-first order runs in bbs_localize_hostqueue");
    else if (k > (1 << 24) - 2) rc = set_error(BBS_EINVAL, "localize: more than 2^24 - 2 scan points");
    if (rc == BBS_OK) rc = scan_prepare(m, xyz, k, is_device, rg, opts, st_, &h.scan, true);
    if (rc < 0) {
        release(i);
        return rc;
    }
    const HostGrid& g = h.scan.grid;
    if ((m->flags & BBS_EXACT_BOUND) && k > 0) {   // the maps' widening must cover this scan's grid
        const int need = exact_dilation_needed(g, h.scan.norm_max);
        const int have = (int)((m->flags >> 12) & 15u);
        if (need < 0 || need > have) {
            rc = need < 0 ? set_error(BBS_EINVAL, "localize: the exact bound does not hold for BBS_CHILD_LITERAL")
                          : set_error(BBS_EINVAL, "localize: exact-bound maps widened by %d, this scan needs %d", have, need);
            release(i);
            return rc;
        }
    }
    h.bytes += estimate_bytes(k, g) - (3 * sizeof(unsigned long long) * ((size_t)k + 1) + 1024);
    h.thr = (int32_t)std::ceil(frac * (double)k);
    h.res.phase_ms[0] = now_ms() - h.t0;
    h.res.h2d_bytes += h.scan.h2d;
    h.res.d2h_bytes += h.scan.d2h;
    h.res.launches += 2;
    if (k == 0) return BBS_OK;   // never live: reported as not found
    SearchDev& d = h.dev;
    std::memset(&d, 0, sizeof(d));
    d.scan = h.scan.scan;
    d.cbox = h.scan.cbox;
    d.rot = h.scan.rot;
    d.cs = h.scan.cs;
    d.K = (int32_t)k;
    d.lmax = g.levels - 1;
    d.batch = (opts && opts->batch > 0) ? opts->batch : 10000;
    d.nblk = (int32_t)((k + PBLK - 1) / PBLK);
    for (int a = 0; a < 3; ++a) {
        const int64_t pmin = floor_div2(g.wmin[a]), pmax = floor_div2(g.wmax[a]);
        d.pmin[a] = (int32_t)pmin;
        d.pext[a] = (int32_t)(pmax - pmin + 1);
        d.wmin[a] = (int32_t)g.wmin[a];
        d.wmax[a] = (int32_t)g.wmax[a];
    }
    d.grid = dev_grid(g);
    for (int l = 0; l < MAX_LEVELS; ++l) d.maps[l] = l < m->levels ? level_view(m, l) : LevelView{};
    const size_t K1 = (size_t)k + 1;
    rc = BBS_OK;
    if (rc == BBS_OK) rc = slot_get(h, &d.b_cnt, K1);
    if (rc == BBS_OK) rc = slot_get(h, &d.b_kids, K1);
    if (rc == BBS_OK) rc = slot_get(h, &d.b_leaf, K1);
    if (rc < 0) {
        release(i);
        return rc;
    }
    h.ctl0 = Ctl();
    h.ctl0.best = h.thr - 1;
    h.ctl0.top = -1;
    h.ctl0.sstar = -1;
    h.ctl0.active = 1;
    h.live = true;
    h.fresh = true;
    int64_t n0 = 1;
    for (int a = 0; a < 3; ++a) n0 *= (g.wmax[a] - g.wmin[a] + 1);
    h.res.nodes_scored = n0 * g.nrot[g.levels - 1];
    rc = upload_slot(i);
    if (rc < 0) {
        release(i);
        return rc;
    }
    return BBS_OK;
}

int Engine::start()
{
    std::vector<int32_t> slots;
    bool others = false;   // searches already iterating keep nodes in the frontier
    for (int i = 0; i < max_slots_; ++i) {
        if (hosts_[(size_t)i].fresh) slots.push_back(i);
        else if (hosts_[(size_t)i].live) others = true;
    }
    if (slots.empty()) return BBS_OK;
    // the initial sets' survivors (at most 8 per task) join the incoming array:
    // grow first when they may not fit
    if (max_nodes_ > cap_eff_) {
        int64_t extra = 0;
        for (int i : slots) {
            const SearchHost& h = hosts_[(size_t)i];
            extra += 8 * (int64_t)h.dev.pext[0] * h.dev.pext[1] * h.dev.pext[2] * h.scan.grid.nrot[h.scan.grid.levels - 1];
        }
        int64_t held = 0;
        int incoming = 1;
        if (others || extra > cap_eff_) {
            LoopState ls;
            BBS_CUDA_TRY(cudaMemcpyAsync(&ls, d_ls_, sizeof(ls), cudaMemcpyDeviceToHost, st_));
            BBS_CUDA_TRY(cudaStreamSynchronize(st_));
            incoming = 1 - ls.cur;
            held = others ? (int64_t)ls.fn[incoming] : 0;
        }
        if (held + extra > cap_eff_) BBS_TRY(grow_to(held + extra, incoming, held));
    }
    BBS_CUDA_TRY(cudaMemcpyAsync(d_slots_, slots.data(), sizeof(int32_t) * slots.size(), cudaMemcpyHostToDevice, st_));
    slot_init_kernel<<<(int)slots.size(), 1024, 0, st_>>>(d_S_, d_slots_);
    launches_ += 1;
    BBS_CUDA_TRY(cudaGetLastError());
    // the initial sets: virtual parents x rotations at l_max, in launches
    // bounded by the task capacity
    std::vector<Seg> segs;
    int64_t nsl = 0, ntk = 0;
    auto flush = [&]() -> int {
        if (segs.empty()) return BBS_OK;
        BBS_TRY(score_launch(MODE_INITIAL, &segs, nsl, ntk));
        segs.clear();
        nsl = ntk = 0;
        return BBS_OK;
    };
    for (int i : slots) {
        SearchHost& h = hosts_[(size_t)i];
        const HostGrid& g = h.scan.grid;
        const int64_t R = g.nrot[g.levels - 1];
        const int64_t vpn = (int64_t)h.dev.pext[0] * h.dev.pext[1] * h.dev.pext[2];
        if (R > TASK_CAP) return set_error(BBS_EINVAL, "localize: %lld initial rotations", (long long)R);
        const int64_t cap = std::max<int64_t>(tune_.launch_tasks, R);
        for (int64_t v0 = 0; v0 < vpn;) {
            const int64_t take = std::min<int64_t>(vpn - v0, (cap - ntk) / R);
            if (take <= 0 || (int)segs.size() == MAXSEG) {
                BBS_TRY(flush());
                continue;
            }
            Seg sg;
            std::memset(&sg, 0, sizeof(sg));
            sg.first_parent = v0;
            sg.first_task = ntk;
            sg.n_tasks = take * R;
            sg.first_slice = nsl;
            sg.sid = i;
            sg.nblk = h.dev.nblk;
            sg.R = (int32_t)R;
            sg.best = h.thr - 1;
            segs.push_back(sg);
            ntk += take * R;
            nsl += take * R * h.dev.nblk;
            h.res.gathers += take * R * h.scan.k;
            v0 += take;
        }
    }
    BBS_TRY(flush());
    // the (cos, sin) entries of the levels below the top, formed on the host
    // while the GPU scores the initial sets; stream order puts them before
    // the first branching
    for (int i : slots) {
        SearchHost& h = hosts_[(size_t)i];
        const int64_t before = h.scan.h2d;
        BBS_TRY(scan_finish_angles(&h.scan, st_));
        h.res.h2d_bytes += h.scan.h2d - before;
    }
    const double t = now_ms();
    for (int i : slots) {
        SearchHost& h = hosts_[(size_t)i];
        h.res.phase_ms[1] = t - h.t0 - h.res.phase_ms[0];
        h.t_init = t;
        h.fresh = false;
    }
    return BBS_OK;
}

void Engine::finish_never_live(std::vector<int>* finished)
{
    // searches that never went live (no points, or failed) finish at once
    for (int i = 0; i < max_slots_; ++i) {
        SearchHost& h = hosts_[(size_t)i];
        if (h.used && !h.live && h.t_end == 0) {
            h.t_end = now_ms();
            finished->push_back(i);
        }
    }
}

int Engine::read_ctl()
{
    BBS_CUDA_TRY(cudaMemcpyAsync(h_ctl_, d_ctl_, sizeof(Ctl) * (size_t)max_slots_, cudaMemcpyDeviceToHost, st_));
    BBS_CUDA_TRY(cudaStreamSynchronize(st_));
    for (int i = 0; i < max_slots_; ++i)
        if (hosts_[(size_t)i].live) hosts_[(size_t)i].res.d2h_bytes += (int64_t)sizeof(Ctl);
    return BBS_OK;
}

void Engine::mark_finished(std::vector<int>* finished)
{
    const double t = now_ms();
    for (int i = 0; i < max_slots_; ++i) {
        SearchHost& h = hosts_[(size_t)i];
        if (!h.live) continue;
        const Ctl& c = h_ctl_[i];
        if (c.err) {
            // the frontier filled while this search inserted, or its counts
            // failed a check: it fails alone
            if (c.err & 4) h.status = set_error(BBS_ECORRUPT, "localize: frontier counts are inconsistent");
            else h.status = set_error(BBS_ENOMEM, "localize: the frontier (%lld nodes) is full", (long long)fcap_);
            h.live = false;
            h.t_end = t;
            finished->push_back(i);
        } else if (c.done) {
            h.live = false;
            h.t_end = t;
            finished->push_back(i);
        }
    }
}

cudaError_t Engine::launch_select(cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond)
{
    select_kernel<<<max_slots_, 1024, 0, s>>>(d_S_, max_slots_, d_plan_, d_ls_, d_poff_, d_toff_, d_pcnt_, d_tcnt_, cond,
                                             use_cond, tune_, d_wake_);
    return cudaGetLastError();
}

cudaError_t Engine::launch_compact(cudaStream_t s, bool pdl)
{
    return launch_pdl(compact_kernel, dim3(nsm_ * 4), dim3(256), s, pdl, d_S_, front_, d_ls_, (const Plan*)d_plan_,
                      parents_, pfirst_, pscore_, (const int64_t*)d_poff_, (const int64_t*)d_toff_, d_pcnt_, d_tcnt_,
                      grp_, max_slots_, max_slots_ == 1 ? 1 : 0, cdone_);
}

// the round's rotation groups: task ranges, then the task records (both
// return at once unless the round scores in one launch)
cudaError_t Engine::launch_group(cudaStream_t s, bool pdl)
{
    if (max_slots_ > 1) {   // a one-slot engine's compaction scans its groups itself
        cudaError_t e = launch_pdl(group_scan_kernel, dim3(max_slots_), dim3(1024), s, pdl, d_S_, max_slots_,
                                   (const Plan*)d_plan_, (const int64_t*)d_poff_, (const int64_t*)d_toff_, grp_);
        if (e != cudaSuccess) return e;
    }
    return launch_pdl(emit_tasks_kernel, dim3(nsm_ * 4), dim3(256), s, pdl, d_S_, (const Plan*)d_plan_,
                      (const NodeRec*)parents_, (const int32_t*)pscore_, grp_, tasks_, tscore_);
}

// one host-driven iteration: select (+ plan), compaction and the second
// lexmin pass on the device, then one synchronization; the scoring launch
// follows the plan
int Engine::step(std::vector<int>* finished)
{
    finish_never_live(finished);
    if (live_count() == 0) return BBS_OK;
    h_plan_.iters = 0;
    h_plan_.max_iters = 1 << 30;
    BBS_CUDA_TRY(cudaMemcpyAsync(&d_plan_->iters, &h_plan_.iters, 2 * sizeof(int32_t), cudaMemcpyHostToDevice, st_));
    BBS_CUDA_TRY(launch_select(st_, 0, 0));
    BBS_CUDA_TRY(launch_compact(st_));
    BBS_CUDA_TRY(launch_group(st_));
    // the lexmin leaf must be complete when the control blocks are read below
    BBS_CUDA_TRY(launch_finalize(MODE_SEARCH, d_plan_, d_S_, tasks_, dense_, front_, d_ls_, nsm_ * 8, st_, true));
    launches_ += max_slots_ > 1 ? 5 : 4;
    BBS_CUDA_TRY(cudaGetLastError());
    // status, iterations, cap and the grow request of the plan
    BBS_CUDA_TRY(cudaMemcpyAsync(h_misc_, &d_plan_->status, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st_));
    BBS_TRY(read_ctl());
    const int32_t status = h_misc_[0];
    if (h_misc_[3]) BBS_TRY(resume_grown(finished));
    else mark_finished(finished);
    if (status == PLAN_OK) return score_launch(MODE_SEARCH, nullptr, 0, 0);
    if (status == PLAN_OVERFLOW) return score_overflow();
    return BBS_OK;
}

// a round too large for one launch: its parents were gathered by the
// compaction; tasks are expanded and scored in windows
int Engine::score_overflow()
{
    const int n = max_slots_;
    BBS_CUDA_TRY(cudaMemcpyAsync(h_off_, d_poff_, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, st_));
    BBS_CUDA_TRY(cudaMemcpyAsync(h_off_ + n, d_toff_, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToHost, st_));
    BBS_CUDA_TRY(cudaStreamSynchronize(st_));
    std::vector<Seg> segs;
    int64_t nsl = 0, ntk = 0;
    auto flush = [&]() -> int {
        if (segs.empty()) return BBS_OK;
        BBS_TRY(score_launch(MODE_SEARCH, &segs, nsl, ntk));
        segs.clear();
        nsl = ntk = 0;
        return BBS_OK;
    };
    for (int i = 0; i < n; ++i) {
        SearchHost& h = hosts_[(size_t)i];
        if (!h.live) continue;
        const int64_t nt = h_ctl_[i].n_tasks, np = h_ctl_[i].n_parents;
        for (int64_t t0 = 0; t0 < nt;) {
            const int64_t take = std::min<int64_t>(nt - t0, tune_.launch_tasks - ntk);
            if (take <= 0 || (int)segs.size() == MAXSEG) {
                BBS_TRY(flush());
                continue;
            }
            const int blocks = (int)std::min<int64_t>((np + 255) / 256, 4096);
            expand_kernel<<<std::max(blocks, 1), 256, 0, st_>>>(d_S_, i, parents_, pfirst_, pscore_, h_off_[i],
                                                                 h_off_[i] + np, h_off_[n + i] + t0,
                                                                 h_off_[n + i] + t0 + take, ntk, tasks_, tscore_);
            launches_ += 1;
            BBS_CUDA_TRY(cudaGetLastError());
            Seg sg;
            std::memset(&sg, 0, sizeof(sg));
            sg.first_task = ntk;
            sg.n_tasks = take;
            sg.first_slice = nsl;
            sg.sid = i;
            sg.nblk = h.dev.nblk;
            sg.best = h_ctl_[i].best;
            segs.push_back(sg);
            ntk += take;
            nsl += take * h.dev.nblk;
            t0 += take;
        }
    }
    return flush();
}

// One iteration of the device loop: select (+ plan), compaction, the
// rotation groups' task ranges and records, scoring (+ lexmin, survivors).  With pdl, each kernel after the first is a
// programmatic dependent launch: its CTAs are scheduled while its predecessor
// drains and wait (pdl_wait) for it to complete, hiding the launch gaps.
cudaError_t Engine::capture_body(cudaGraph_t body, cudaGraphConditionalHandle cond, bool pdl)
{
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = launch_select(cs, cond, 1);
        if (le == cudaSuccess) le = launch_compact(cs, pdl);
        if (le == cudaSuccess) le = launch_group(cs, pdl);
        if (le == cudaSuccess)
            le = launch_branch(MODE_SEARCH, d_plan_, d_S_, tasks_, dense_, nsm_ * tune_.ctas_per_sm, cs, graph_bytes_,
                               pdl);
        if (le == cudaSuccess)
            le = launch_finalize(MODE_SEARCH, d_plan_, d_S_, tasks_, dense_, front_, d_ls_, nsm_ * 8, cs, false, tscore_,
                                 pdl);
        cudaGraph_t out = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &out);
        e = le != cudaSuccess ? le : e2;
    }
    cudaStreamDestroy(cs);
    return e;
}

int Engine::build_graph()
{
    // with programmatic dependent launches first; a driver that refuses them
    // inside the loop body gets the plain launches
    for (int attempt = 0; attempt < 2; ++attempt) {
        const bool pdl = graph_pdl_ && attempt == 0;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaGraphCreate(&g, 0);
        cudaGraphConditionalHandle cond = 0;
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
        alignas(cudaGraphNodeParams) unsigned char np_buf[sizeof(cudaGraphNodeParams)];
        std::memset(np_buf, 0, sizeof(np_buf));
        cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_buf);
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = cond;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
        if (e == cudaSuccess) e = capture_body(np.conditional.phGraph_out[0], cond, pdl);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec_, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) {
            graph_pdl_ = pdl;
            return BBS_OK;
        }
        exec_ = nullptr;
        cudaGetLastError();   // a refused capture leaves no sticky error
        if (!pdl) return set_error(BBS_ECUDA, "engine: building the iteration graph: %s", cudaGetErrorString(e));
    }
    return set_error(BBS_ECUDA, "engine: building the iteration graph");
}

int Engine::set_exit_on_finish(bool v)
{
    exit_on_finish_ = v;
    const int32_t x = v ? 1 : 0;
    // pageable source: staged before the call returns
    BBS_CUDA_TRY(cudaMemcpyAsync(&d_ls_->exit_on_finish, &x, sizeof(x), cudaMemcpyHostToDevice, st_));
    return BBS_OK;
}

int Engine::iterate(int max_iters, std::vector<int>* finished)
{
    // CUDA events cannot sit inside the graph's loop body: timed runs take
    // the host-driven path, whose scoring launches are the same kernels
    if (host_driven_ || timed_) return step(finished);
    finish_never_live(finished);
    if (live_count() == 0) return BBS_OK;
    const bool bo = bytes_only();
    if (exec_ && bo != graph_bytes_) {   // the graph holds the scoring kernel variant it was captured with
        cudaGraphExecDestroy(exec_);
        exec_ = nullptr;
    }
    if (!exec_) {
        graph_bytes_ = bo;
        BBS_TRY(build_graph());
    }
    h_plan_.iters = 0;
    h_plan_.max_iters = max_iters > 0 ? max_iters : 1;
    BBS_CUDA_TRY(cudaMemcpyAsync(&d_plan_->iters, &h_plan_.iters, 2 * sizeof(int32_t), cudaMemcpyHostToDevice, st_));
    BBS_CUDA_TRY(cudaGraphLaunch(exec_, st_));
    // status and the iterations the device loop ran, with the control blocks
    BBS_CUDA_TRY(cudaMemcpyAsync(h_misc_, &d_plan_->status, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st_));
    BBS_TRY(read_ctl());
    const int32_t status = h_misc_[0];
    launches_ += (max_slots_ > 1 ? 6 : 5) * (int64_t)h_misc_[1];   // the loop body's kernels per iteration
    if (h_misc_[3]) {   // the last round waits for the frontier to grow; then it is scored from the host
        BBS_TRY(resume_grown(finished));
        if (status == PLAN_OK) return score_launch(MODE_SEARCH, nullptr, 0, 0);
        if (status == PLAN_OVERFLOW) return score_overflow();
        return BBS_OK;
    }
    mark_finished(finished);
    if (status == PLAN_OVERFLOW) return score_overflow();   // the selected round did not fit one launch
    return BBS_OK;
}

int Engine::finalize(int i, bbs_result* out)
{
    SearchHost& h = hosts_[(size_t)i];
    // the control block as the last read_ctl saw it: a finished search's
    // block no longer changes
    Ctl c;
    std::memset(&c, 0, sizeof(c));
    if (h.scan.k > 0) c = h_ctl_[i];
    if (!evs_.empty()) {
        BBS_CUDA_TRY(cudaEventSynchronize(evs_.back()));
        g_launch_log.units.clear();
        g_launch_log.ms.clear();
    }
    for (size_t e = 0; e + 1 < evs_.size(); e += 2) {
        float ms = 0.0f;
        BBS_CUDA_TRY(cudaEventElapsedTime(&ms, evs_[e], evs_[e + 1]));
        score_ms_ += ms;
        g_launch_log.units.push_back(e / 2 < ev_units_.size() ? ev_units_[e / 2] : 0);
        g_launch_log.ms.push_back(ms);
    }
    for (cudaEvent_t e : evs_) cudaEventDestroy(e);
    evs_.clear();
    ev_units_.clear();
    bbs_result* r = &h.res;
    const double t_fin = now_ms();
    if (h.t_end == 0) h.t_end = t_fin;
    r->launches += launches_;
    r->score_launches = score_launches_;
    r->score_ms = score_ms_;
    int status;
    if (h.status < 0) {
        status = h.status;
    } else if (h.scan.k == 0) {
        r->best_score = h.thr - 1;
        status = BBS_NOT_FOUND;
    } else {
        const HostGrid& g = h.scan.grid;
        r->iterations = c.st_iters;
        r->parents_branched = c.st_parents;
        r->nodes_scored += c.st_nodes;
        r->children_scored = c.st_nodes;
        r->bound_violations = (int64_t)c.st_viol;
        r->bound_excess = c.st_excess;
        r->rotations = (int64_t)c.st_rotpts;
        r->gathers += c.st_gathers;
        r->probes = r->nodes_scored * h.scan.k;
        r->best_score = c.best;
        r->peak_frontier = c.peak;
        // device timestamps: the initial set starts at t_start_ns
        const double dev_end = c.t_end_ns > c.t_start_ns ? (double)(c.t_end_ns - c.t_start_ns) / 1e6 : 0.0;
        const double dev_match = c.found && c.t_match_ns > c.t_start_ns ? (double)(c.t_match_ns - c.t_start_ns) / 1e6 : -1.0;
        const double init_ms = r->phase_ms[1];
        r->phase_ms[2] = (dev_match >= 0 ? dev_match : dev_end) - init_ms;
        r->phase_ms[3] = dev_match >= 0 ? dev_end - dev_match : 0.0;
        if (r->phase_ms[2] < 0) r->phase_ms[2] = 0;
        r->d2h_bytes += (int64_t)sizeof(Ctl);
        if (c.found && c.lex_t != ~0ull) {
            // the lexmin leaf: biased 21-bit translation fields, then the rotation
            const uint32_t rot = c.lex_r;
            const int64_t ng = g.N[0][2], nb = g.N[0][1];
            r->found = 1;
            r->node[0] = (int32_t)((c.lex_t >> 42) & 0x1FFFFF) - KEY_LIMIT;
            r->node[1] = (int32_t)((c.lex_t >> 21) & 0x1FFFFF) - KEY_LIMIT;
            r->node[2] = (int32_t)(c.lex_t & 0x1FFFFF) - KEY_LIMIT;
            r->node[3] = (int32_t)(rot / (ng * nb));
            r->node[4] = (int32_t)((rot / ng) % nb);
            r->node[5] = (int32_t)(rot % ng);
            r->node[6] = 0;
            for (int a = 0; a < 3; ++a) r->pose[a] = (double)r->node[a] * g.r;
            for (int a = 0; a < 3; ++a) r->pose[3 + a] = grid_angle(g, 0, a, r->node[3 + a]);
            r->ms_to_optimum = r->phase_ms[0] + dev_match;
            status = BBS_OK;
        } else if (c.found) {
            status = set_error(BBS_ECORRUPT, "localize: a leaf bucket was popped without a leaf");
        } else {
            r->ms_to_optimum = r->phase_ms[0] + dev_end;
            status = BBS_NOT_FOUND;
        }
    }
    r->status = status;
    r->ms_total = t_fin - h.t0;
    r->phase_ms[4] = t_fin - h.t_end;
    if (out) *out = *r;
    BBS_TRY(release(i));
    return status;
}

int Engine::cancel(int i, int code, bbs_result* out)
{
    SearchHost& h = hosts_[(size_t)i];
    if (h.live) {
        h.live = false;
        h.status = code;
        h.t_end = now_ms();
    }
    return finalize(i, out);
}

int Engine::release(int i)
{
    SearchHost& h = hosts_[(size_t)i];
    if (!h.used) return BBS_OK;
    // a search stopped before it finished may still have nodes: remove them
    // before the slot can be reused
    const bool may_hold = h.dev.K > 0 && h_ctl_[i].active && !h_ctl_[i].done;
    if (may_hold && d_ls_) {
        purge_reset_kernel<<<1, 1, 0, st_>>>(d_ls_);
        purge_kernel<<<nsm_ * 4, 256, 0, st_>>>(front_, d_ls_, i);
        purge_swap_kernel<<<1, 1, 0, st_>>>(d_ls_);
        launches_ += 3;
    }
    // the zeroed control block comes from a pinned block the host never rewrites
    if (d_ctl_) cudaMemcpyAsync(d_ctl_ + i, h_zero_, sizeof(Ctl), cudaMemcpyHostToDevice, st_);
    std::memset(&h_ctl_[i], 0, sizeof(Ctl));
    for (void* p : h.bufs) cudaFreeAsync(p, st_);
    scan_release(&h.scan, st_);
    h = SearchHost();
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(BBS_ECUDA, "engine: %s", cudaGetErrorString(e));
    return BBS_OK;
}

// One scoring launch.  With segs: a host plan (the initial set, or a window of
// a large round) is uploaded; without: the device plan of the last select.
int Engine::score_launch(int mode, const std::vector<Seg>* segs, int64_t n_slices, int64_t n_tasks)
{
    if (segs) {
        h_plan_.n_slices = n_slices;
        h_plan_.n_tasks = n_tasks;
        h_plan_.next_slice = 0;
        h_plan_.static_pm = tune_.static_pm;
        h_plan_.grab_min = tune_.grab_min;
        h_plan_.nseg = (int32_t)segs->size();
        h_plan_.mode = mode;
        h_plan_.status = PLAN_OK;
        for (size_t i = 0; i < segs->size(); ++i) h_plan_.seg[i] = (*segs)[i];
        // pageable source: staged before cudaMemcpyAsync returns, so h_plan_ may be rewritten
        BBS_CUDA_TRY(cudaMemcpyAsync(d_plan_, &h_plan_, offsetof(Plan, seg) + sizeof(Seg) * segs->size(),
                                     cudaMemcpyHostToDevice, st_));
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    volatile int* gate = h_wake_ + 1;   // h_wake_[1]: the timing gate, h_wake_[2]: its overrun flag
    if (timed_) {
        BBS_CUDA_TRY(cudaEventCreate(&e0));
        evs_.push_back(e0);
        BBS_CUDA_TRY(cudaEventCreate(&e1));
        evs_.push_back(e1);
        *gate = 0;
        timing_gate_kernel<<<1, 1, 0, st_>>>(d_wake_ + 1, d_wake_ + 2);
        // the launch's units: a host plan's segments, else the tasks the
        // control blocks (read before every device-planned launch) report
        int64_t u = 0;
        if (segs) {
            for (const Seg& g : *segs) u += g.n_tasks * (int64_t)hosts_[(size_t)g.sid].scan.k;
        } else {
            for (int i = 0; i < max_slots_; ++i)
                if (hosts_[(size_t)i].live && h_ctl_[i].active && !h_ctl_[i].done && !h_ctl_[i].err)
                    u += h_ctl_[i].n_tasks * hosts_[(size_t)i].scan.k;
        }
        ev_units_.push_back(u);
        BBS_CUDA_TRY(cudaEventRecord(e0, st_));
    }
    const cudaError_t le = launch_branch(mode, d_plan_, d_S_, tasks_, dense_, nsm_ * tune_.ctas_per_sm, st_, bytes_only());
    if (timed_) {
        const cudaError_t re = cudaEventRecord(e1, st_);
        *gate = 1;   // everything is enqueued: the stream may run the launch
        BBS_CUDA_TRY(le);
        BBS_CUDA_TRY(re);
    }
    BBS_CUDA_TRY(le);
    BBS_CUDA_TRY(launch_finalize(mode, d_plan_, d_S_, tasks_, dense_, front_, d_ls_, nsm_ * 8, st_, false,
                                 mode == MODE_SEARCH ? tscore_ : nullptr));
    BBS_CUDA_TRY(cudaGetLastError());
    launches_ += 2;
    score_launches_ += 1;
    return BBS_OK;
}

// ---- the one-shot entry points ------------------------------------------------------
//
// Engines (their chunk pool and staging buffers, hundreds of MB) are kept per
// device and reused by later calls: a finished run leaves the pool full and
// every slot released.  A call takes an idle engine with enough slots and pool
// or builds one; at most four idle engines per device are kept.

namespace {

struct CachedEngine {
    int device;
    int slots;
    int64_t pool_nodes;
    Engine* e;
    bool busy;
};

std::mutex g_engine_mu;
std::vector<CachedEngine> g_engines;

Engine* acquire_engine(int slots, int64_t pool_nodes, cudaStream_t st, bool timed, int* rc)
{
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(g_engine_mu);
        for (auto& c : g_engines)
            if (!c.busy && c.device == dev && c.slots >= slots && c.pool_nodes >= pool_nodes &&
                c.pool_nodes <= 4 * pool_nodes + ((int64_t)1 << 22) && c.slots <= 4 * slots + 16) {
                c.busy = true;
                *rc = c.e->begin_run(st, timed);
                return c.e;
            }
    }
    Engine* e = new Engine(st, slots, pool_nodes, timed);
    *rc = e->init();
    if (*rc < 0) {
        delete e;
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_engine_mu);
    g_engines.push_back(CachedEngine{dev, slots, pool_nodes, e, true});
    return e;
}

void release_engine(Engine* e, bool healthy)
{
    std::lock_guard<std::mutex> lock(g_engine_mu);
    for (size_t i = 0; i < g_engines.size(); ++i)
        if (g_engines[i].e == e) {
            int idle = 0;
            for (auto& c : g_engines) idle += (!c.busy && c.device == g_engines[i].device) ? 1 : 0;
            if (!healthy || idle >= 4) {
                delete e;
                g_engines.erase(g_engines.begin() + (long)i);
            } else {
                g_engines[i].busy = false;
            }
            return;
        }
}

}  // namespace

int search_run(const bbs_maps* m, const float* xyz, int64_t k, int is_device, const bbs_ranges* rg,
               const bbs_opts* opts, cudaStream_t st, bbs_result* res)
{
    // the frontier starts at up to 2^24 nodes and doubles as a search needs, up to max_frontier
    const int64_t max_frontier = (opts && opts->max_frontier > 0) ? opts->max_frontier : ((int64_t)1 << 30);
    const bool timed = opts && (opts->flags & BBS_TIME_KERNELS);
    const int64_t slack = (int64_t)CH * std::min<int64_t>(k + 1, 8192);
    const int32_t f2 = current_tuning().frontier_log2;
    const int64_t pool_nodes = f2 ? std::min<int64_t>(max_frontier, (int64_t)1 << f2)
                                  : std::min<int64_t>(max_frontier, (int64_t)1 << 24) + slack;
    std::memset(res, 0, sizeof(*res));
    int rc = BBS_OK;
    Engine* E = acquire_engine(1, pool_nodes, st, timed, &rc);
    if (!E) return rc;
    int slot = -1;
    if (rc == BBS_OK) rc = E->set_max_nodes(std::max(pool_nodes, max_frontier));
    if (rc == BBS_OK) rc = E->add(m, xyz, k, is_device, rg, opts, 0, &slot);
    if (rc == BBS_OK) rc = E->start();
    E->set_host_driven(opts && (opts->flags & BBS_HOST_DRIVEN));
    std::vector<int> fin;
    while (rc == BBS_OK && E->used_count() > 0) {
        fin.clear();
        rc = E->iterate(1 << 20, &fin);
        for (int i : fin) E->finalize(i, res);
    }
    release_engine(E, rc == BBS_OK);
    return rc == BBS_OK ? res->status : rc;
}

int search_run_many(const bbs_maps* m, int n, const float* const* scans, const int64_t* ks, int is_device,
                    const bbs_ranges* rg, const bbs_opts* opts, cudaStream_t st, bbs_result* res)
{
    const int64_t max_frontier = (opts && opts->max_frontier > 0) ? opts->max_frontier : ((int64_t)1 << 30);
    const bool timed = opts && (opts->flags & BBS_TIME_KERNELS);
    int64_t kmax = 1;
    for (int i = 0; i < n; ++i) kmax = std::max(kmax, ks[i]);
    // at most MAX_SLOTS searches advance together; the others take slots as
    // searches finish (each result is the same either way)
    const int slots = std::min(n, MAX_SLOTS);
    const int64_t slack = (int64_t)CH * std::min<int64_t>((kmax + 1) * slots, 8192 * (int64_t)slots);
    const int32_t f2 = current_tuning().frontier_log2;
    const int64_t pool_nodes = f2 ? std::min<int64_t>(max_frontier, (int64_t)1 << f2)
                                  : std::min<int64_t>(max_frontier, (int64_t)1 << 24) + slack;
    int rc = BBS_OK;
    Engine* E = acquire_engine(slots, pool_nodes, st, timed, &rc);
    if (!E) return rc;
    if (rc == BBS_OK) rc = E->set_max_nodes(std::max(pool_nodes, max_frontier));
    int next = 0;
    auto admit = [&]() {
        for (int slot = -1; rc == BBS_OK && next < n && E->used_count() < slots; ++next) {
            std::memset(&res[next], 0, sizeof(res[next]));
            rc = E->add(m, scans[next], ks[next], is_device, rg, opts, (uint64_t)next, &slot);
        }
        if (rc == BBS_OK) rc = E->start();
    };
    admit();
    E->set_host_driven(opts && (opts->flags & BBS_HOST_DRIVEN));
    std::vector<int> fin;
    while (rc == BBS_OK && E->used_count() > 0) {
        fin.clear();
        // with scans still waiting, return to the host every few iterations to refill freed slots
        rc = E->iterate(next < n ? 4 : 1 << 20, &fin);
        for (int s_ : fin) E->finalize(s_, &res[E->tag(s_)]);
        if (rc == BBS_OK && next < n) admit();
    }
    release_engine(E, rc == BBS_OK);
    return rc;
}

}  // namespace bbs
