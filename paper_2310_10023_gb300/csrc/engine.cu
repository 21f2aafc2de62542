// engine.cu -- device-resident batched best-first BnB (Sec. III-E,
// Algorithm 2) for one or many searches at once.
//
// Every search owns a frontier F of scored nodes bucketed by integer score;
// node records live in chunks of CH from one shared free-chunk stack.  A
// search's non-empty bucket owns its chunks (all full but its tail) and every
// chunk in use is listed in the search's active list, tagged by bucket.
//
// One iteration advances every live search by one canonical batch:
//   select  (1 CTA per search) walk buckets from the top with a block-wide
//           prefix of their children counts; the first bucket reached with
//           children(P) >= b stops, one at or below best clears F, one holding
//           a leaf sets (best, lexmin leaf) and clears F; buckets above it pop.
//   gather  popped chunks -> one dense parent array (all searches), chunks freed
//   score   (branch.cu) every child of every parent; finalize keeps > best
//   alloc   (1 CTA per search) chunks for each bucket's survivors
//   scatter survivors into their buckets' chunks
// Only popping a leaf changes a search's best, so how its batch is split into
// launches, and which other searches share them, cannot change its result.
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

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* total, int64_t* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    const int nw = (int)(blockDim.x >> 5);
    if (wid == 0) {
        int64_t s = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const int64_t before = (wid > 0 ? sh[wid - 1] : 0) + x - v;
    *total = sh[nw - 1];
    __syncthreads();
    return before;
}

__device__ __forceinline__ int block_min_int(int v, int* sh)
{
    v = __reduce_min_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int x = sh[threadIdx.x];
        x = __reduce_min_sync(0xffffffffu, x);
        if (threadIdx.x == 0) sh[32] = x;
    }
    __syncthreads();
    const int r = sh[32];
    __syncthreads();
    return r;
}

// lexicographic order of (c_x, c_y, c_z, rotation index); rotation index order
// equals (c_alpha, c_beta, c_gamma) order
struct LexKey {
    unsigned long long t;
    uint32_t r;
};

__device__ __forceinline__ LexKey lex_of(const NodeRec& n)
{
    LexKey k;
    k.t = ((unsigned long long)(uint32_t)(n.cx + KEY_LIMIT) << 42) | ((unsigned long long)(uint32_t)(n.cy + KEY_LIMIT) << 21) |
          (unsigned long long)(uint32_t)(n.cz + KEY_LIMIT);
    k.r = rl_rot(n.rl);
    return k;
}

__device__ __forceinline__ bool lex_lt(const LexKey& a, const LexKey& b) { return a.t < b.t || (a.t == b.t && a.r < b.r); }

// ---- kernels -----------------------------------------------------------------

__device__ __forceinline__ unsigned long long gtimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void pool_init_kernel(PoolDev p)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p.nchunks; i += (int64_t)gridDim.x * blockDim.x) {
        p.free_ids[i] = (int32_t)(p.nchunks - 1 - i);
        p.chunk_bucket[i] = -1;
        p.chunk_fill[i] = 0;
        p.chunk_tasks[i] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *p.free_top = (unsigned long long)p.nchunks;
}

// reset the frontier arrays of one search (blockIdx.x = slot in `slots`)
__global__ void slot_init_kernel(SearchDev* S, const int32_t* slots)
{
    SearchDev& s = S[slots[blockIdx.x]];
    if (threadIdx.x == 0) s.ctl->t_start_ns = gtimer_ns();
    for (int i = threadIdx.x; i <= s.K; i += blockDim.x) {
        s.b_cnt[i] = 0;
        s.b_kids[i] = 0;
        s.b_leaf[i] = 0;
        s.b_tail[i] = -1;
        s.h_cnt[i] = 0;
        s.h_kids[i] = 0;
        s.h_leaf[i] = 0;
        s.w_pos[i] = 0;
    }
}

__global__ void __launch_bounds__(1024) alloc_kernel(SearchDev* S, int nslots, PoolDev pool, const Plan* P)
{
    if (P->status != PLAN_OK) return;
    __shared__ int64_t sh[32];
    __shared__ int64_t s_base;
    __shared__ int s_min[33];
    for (int si = blockIdx.x; si < nslots; si += gridDim.x) {
        SearchDev& f = S[si];
        Ctl* c = f.ctl;
        if (!c->active || c->err) continue;
        // survivors score above best: only those buckets can have new nodes
        const int lo = c->best + 1 > 0 ? c->best + 1 : 0;
        // pass 1: chunks needed by this search, claimed from the shared stack
        int64_t need_sum = 0;
        for (int s = lo + (int)threadIdx.x; s <= f.K; s += blockDim.x) {
            const uint32_t h = f.h_cnt[s];
            if (!h) continue;
            const int32_t tail = f.b_tail[s];
            const int32_t space = tail >= 0 ? CH - pool.chunk_fill[tail] : 0;
            if ((int64_t)h > space) need_sum += ((int64_t)h - space + CH - 1) / CH;
        }
        int64_t tot;
        block_excl_scan(need_sum, &tot, sh);
        if (threadIdx.x == 0) {
            s_base = -1;
            if (tot > 0) {
                const unsigned long long old = atomicAdd(pool.free_top, (unsigned long long)(-(long long)tot));
                if ((long long)old - tot < 0) {
                    atomicAdd(pool.free_top, (unsigned long long)tot);   // give the claim back
                    c->err |= 1;
                } else {
                    s_base = (int64_t)old - tot;   // claimed stack entries [old - tot, old)
                }
            }
        }
        __syncthreads();
        if (c->err) continue;
        const int64_t claim_top = s_base + tot;   // stack index just above the claim
        const int64_t act0 = c->n_act;
        // pass 2: hand out the claimed chunks bucket by bucket
        int64_t carry = 0, added = 0;
        int top = -1;
        for (int base = lo; base <= f.K; base += blockDim.x) {
            const int s = base + threadIdx.x;
            uint32_t h = 0;
            int32_t tail = -1, fill0 = CH, space = 0;
            int64_t need = 0;
            if (s <= f.K) {
                h = f.h_cnt[s];
                if (h) {
                    tail = f.b_tail[s];
                    fill0 = tail >= 0 ? pool.chunk_fill[tail] : CH;
                    space = CH - fill0;
                    need = (int64_t)h > space ? ((int64_t)h - space + CH - 1) / CH : 0;
                }
            }
            int64_t total;
            const int64_t off = carry + block_excl_scan(need, &total, sh);
            if (h) {
                int32_t last = tail;
                for (int64_t i = 0; i < need; ++i) {
                    const int32_t id = pool.free_ids[claim_top - 1 - (off + i)];
                    pool.chunk_bucket[id] = s;
                    pool.chunk_fill[id] = (int32_t)(i < need - 1 ? CH : ((int64_t)h - space) - (need - 1) * CH);
                    pool.chunk_tasks[id] = 0;
                    f.act[act0 + off + i] = id;
                    last = id;
                }
                if (tail >= 0) pool.chunk_fill[tail] = fill0 + (int32_t)((int64_t)h < space ? h : space);
                f.w_space[s] = space;
                f.w_choff[s] = claim_top - 1 - off;   // stack index of the bucket's first new chunk (counting down)
                f.w_tail[s] = tail;
                f.w_fill0[s] = fill0;
                f.w_pos[s] = 0;
                f.b_tail[s] = last;
                f.b_cnt[s] += h;
                f.b_kids[s] += (int64_t)f.h_kids[s];
                f.b_leaf[s] += f.h_leaf[s];
                f.h_cnt[s] = 0;
                f.h_kids[s] = 0;
                f.h_leaf[s] = 0;
                added += h;
                top = s > top ? s : top;
            }
            carry += total;
        }
        int64_t all_added;
        block_excl_scan(added, &all_added, sh);
        const int maxtop = -block_min_int(-top, s_min);
        if (threadIdx.x == 0) {
            c->n_act = act0 + carry;
            c->size += all_added;
            if (c->size > c->peak) c->peak = c->size;
            if (maxtop > c->top) c->top = maxtop;
        }
        __syncthreads();
    }
}

__global__ void scatter_kernel(SearchDev* S, PoolDev pool, const NodeRec* __restrict__ nodes,
                               const int32_t* __restrict__ scores, const int32_t* __restrict__ sids,
                               const int32_t* __restrict__ ntask, const unsigned long long* count, int64_t cap)
{
    int64_t n = (int64_t)*count;
    if (n > cap) n = cap;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        SearchDev& f = S[sids[i]];
        if (f.ctl->err) continue;
        const int32_t s = scores[i];
        const uint32_t rank = atomicAdd(&f.w_pos[s], 1u);
        int32_t chunk, slot;
        if ((int32_t)rank < f.w_space[s]) {
            chunk = f.w_tail[s];
            slot = f.w_fill0[s] + (int32_t)rank;
        } else {
            const int64_t idx = (int64_t)rank - f.w_space[s];
            chunk = pool.free_ids[f.w_choff[s] - idx / CH];
            slot = (int32_t)(idx % CH);
        }
        pool.nodes[(int64_t)chunk * CH + slot] = nodes[i];
        if (ntask[i]) atomicAdd(&pool.chunk_tasks[chunk], ntask[i]);
    }
}

__global__ void __launch_bounds__(1024) select_kernel(SearchDev* S, int nslots, PoolDev pool)
{
    __shared__ int64_t sh[32];
    __shared__ int s_min[33];
    __shared__ int32_t s_star, s_reason;
    __shared__ LexKey s_lex[1024];
    __shared__ NodeRec s_node[1024];
    __shared__ int s_has[1024];
    __shared__ unsigned long long s_ftop;
    const int tid = threadIdx.x;
    for (int si = blockIdx.x; si < nslots; si += gridDim.x) {
        SearchDev& f = S[si];
        Ctl* c = f.ctl;
        if (!c->active || c->done || c->err) continue;
        const int32_t best = c->best;
        if (tid == 0) {
            s_star = -1;
            s_reason = c->size > 0 ? 4 : 0;
        }
        __syncthreads();
        // 1. the bucket where popping stops
        int64_t carry = 0;
        for (int base = c->top; base >= 0; base -= blockDim.x) {
            const int s = base - tid;
            const bool have = s >= 0 && f.b_cnt[s] > 0;
            const int64_t kids = have ? f.b_kids[s] : 0;
            int64_t tot;
            const int64_t cum = carry + block_excl_scan(kids, &tot, sh);
            const bool stop = have && (cum >= f.batch || s <= best || f.b_leaf[s] > 0);
            const int first = block_min_int(stop ? tid : (int)blockDim.x, s_min);
            if (first < (int)blockDim.x) {
                if (tid == first) {
                    s_star = s;
                    s_reason = cum >= f.batch ? 1 : (s <= best ? 2 : 3);
                }
                __syncthreads();
                break;
            }
            carry += tot;
        }
        const int32_t sstar = s_star;
        const int reason = s_reason;
        const bool clear = reason == 2 || reason == 3;
        // 2. active list: pop chunks above s*, free the rest when clearing, lexmin leaf of s*
        LexKey my_lex;
        my_lex.t = ~0ull;
        my_lex.r = ~0u;
        NodeRec my_node;
        my_node.cx = my_node.cy = my_node.cz = 0;
        my_node.rl = 0;
        int my_has = 0;
        const int64_t n_act = c->n_act;
        int64_t keep = 0, npop = 0, nfree = 0, nparents = 0, ntasks = 0;
        // freed chunks go onto the shared stack: count them first, then claim
        int64_t nfree_total = 0;
        if (clear) {
            for (int64_t i = tid; i < n_act; i += blockDim.x) {
                const int32_t ch = f.act[i];
                if (pool.chunk_bucket[ch] <= sstar) ++nfree_total;
            }
            int64_t t;
            block_excl_scan(nfree_total, &t, sh);
            nfree_total = t;
        }
        if (tid == 0) s_ftop = nfree_total ? atomicAdd(pool.free_top, (unsigned long long)nfree_total) : 0ull;
        __syncthreads();
        const int64_t fbase = (int64_t)s_ftop;
        for (int64_t base = 0; base < n_act; base += blockDim.x) {
            const int64_t i = base + tid;
            const int32_t ch = i < n_act ? f.act[i] : -1;
            const int32_t bk = ch >= 0 ? pool.chunk_bucket[ch] : -1;
            const int32_t fill = ch >= 0 ? pool.chunk_fill[ch] : 0;
            const int32_t ctasks = ch >= 0 ? pool.chunk_tasks[ch] : 0;
            const bool popped = ch >= 0 && bk > sstar;
            const bool freed = ch >= 0 && !popped && clear;
            const bool kept = ch >= 0 && !popped && !clear;
            if (reason == 3 && ch >= 0 && bk == sstar) {
                for (int j = 0; j < fill; ++j) {
                    const NodeRec nd = pool.nodes[(int64_t)ch * CH + j];
                    if (rl_level(nd.rl) != 0) continue;
                    const LexKey k = lex_of(nd);
                    if (!my_has || lex_lt(k, my_lex)) {
                        my_lex = k;
                        my_node = nd;
                        my_has = 1;
                    }
                }
            }
            int64_t t1, t2, t3, t4, t5;
            const int64_t rp = block_excl_scan(popped ? 1 : 0, &t1, sh);
            const int64_t rf = block_excl_scan(freed ? 1 : 0, &t2, sh);
            const int64_t rk = block_excl_scan(kept ? 1 : 0, &t3, sh);
            const int64_t rs = block_excl_scan(popped ? fill : 0, &t4, sh);
            const int64_t rt = block_excl_scan(popped ? ctasks : 0, &t5, sh);
            if (popped) {
                f.pop_ids[npop + rp] = ch;
                f.pop_start[npop + rp] = nparents + rs;
                f.pop_tstart[npop + rp] = ntasks + rt;
                pool.chunk_bucket[ch] = -2;
            }
            if (freed) {
                pool.free_ids[fbase + nfree + rf] = ch;
                pool.chunk_bucket[ch] = -1;
            }
            __syncthreads();   // every read of act[base..] is done before the in-place write
            if (kept) f.act[keep + rk] = ch;
            npop += t1;
            nfree += t2;
            keep += t3;
            nparents += t4;
            ntasks += t5;
            __syncthreads();
        }
        // 3. lexmin leaf across the block
        if (reason == 3) {
            s_lex[tid] = my_lex;
            s_node[tid] = my_node;
            s_has[tid] = my_has;
            __syncthreads();
            for (int o = blockDim.x / 2; o > 0; o >>= 1) {
                if (tid < o && s_has[tid + o] && (!s_has[tid] || lex_lt(s_lex[tid + o], s_lex[tid]))) {
                    s_lex[tid] = s_lex[tid + o];
                    s_node[tid] = s_node[tid + o];
                    s_has[tid] = 1;
                }
                __syncthreads();
            }
        }
        // 4. bucket metadata of popped buckets and, when clearing, of all others
        int64_t popped_kids = 0;
        const int32_t top = c->top;
        for (int s = tid; s <= top; s += blockDim.x) {
            if (s > sstar || clear) {
                if (s > sstar) popped_kids += f.b_kids[s];
                f.b_cnt[s] = 0;
                f.b_kids[s] = 0;
                f.b_leaf[s] = 0;
                f.b_tail[s] = -1;
            }
        }
        int64_t pk;
        block_excl_scan(popped_kids, &pk, sh);
        if (tid == 0) {
            c->n_pop = npop;
            c->n_parents = nparents;
            c->n_tasks = ntasks;
            c->popped_kids = pk;
            c->n_act = keep;
            c->size = clear ? 0 : c->size - nparents;
            c->top = reason == 1 ? sstar : -1;
            c->reason = reason;
            c->match_changed = 0;
            if (reason == 3 && s_has[0]) {
                c->best = sstar;
                c->match = s_node[0];
                c->found = 1;
                c->match_changed = 1;
            }
            c->done = nparents == 0;
            // statistics
            const unsigned long long now = gtimer_ns();
            if (nparents > 0) {
                c->st_iters += 1;
                c->st_parents += nparents;
                c->st_nodes += pk;
                c->st_gathers += (pk / 8) * (int64_t)f.K;
            }
            if (c->match_changed) c->t_match_ns = now;
            if (c->done) c->t_end_ns = now;
        }
        __syncthreads();
    }
}

// push every chunk a search still holds back onto the shared stack
__global__ void slot_release_kernel(SearchDev* S, int slot, PoolDev pool)
{
    SearchDev& f = S[slot];
    Ctl* c = f.ctl;
    const int64_t n = c->n_act;
    __shared__ unsigned long long base;
    if (threadIdx.x == 0) base = n > 0 ? atomicAdd(pool.free_top, (unsigned long long)n) : 0ull;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const int32_t ch = f.act[i];
        pool.free_ids[base + i] = ch;
        pool.chunk_bucket[ch] = -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        c->n_act = 0;
        c->size = 0;
        c->active = 0;
    }
}

// the tasks (rotational children, Eq. (13)) of parent p, written at tasks[dst
// + t] for the t in [t0, t1): parent and rl (task_rows_kernel adds the rows)
__device__ __forceinline__ void write_tasks(const SearchDev& f, const NodeRec& nd, int64_t p, const int32_t lo[3],
                                            const int32_t ext[3], int32_t t0, int32_t t1, TaskRec* tasks, int64_t dst)
{
    const DevGrid& g = f.grid;
    const int l = rl_level(nd.rl);
    const int64_t nb = g.N[l - 1][1], ng = g.N[l - 1][2];
    int32_t t = 0;
    for (int32_t ja = 0; ja < ext[0]; ++ja)
        for (int32_t jb = 0; jb < ext[1]; ++jb)
            for (int32_t jg = 0; jg < ext[2]; ++jg, ++t) {
                if (t < t0 || t >= t1) continue;
                const uint32_t crot = (uint32_t)(((int64_t)(lo[0] + ja) * nb + (lo[1] + jb)) * ng + (lo[2] + jg));
                TaskRec& r = tasks[dst + t];   // the rows follow (task_rows_kernel)
                r.parent = (int32_t)p;
                r.rl = rl_pack(crot, l - 1);
            }
}

// popped chunks of every search -> the parent array at the search's offset,
// each parent's first task (its rotational children are numbered per
// search in parent order, from toff[search]) and, when the round is scored
// in one launch (PLAN_OK), the task records themselves.  One CTA of CH
// threads per popped chunk (one node per thread); the chunks are freed.
__global__ void __launch_bounds__(CH) gather_kernel(SearchDev* S, PoolDev pool, const int64_t* __restrict__ poff,
                                                    const int64_t* __restrict__ toff, int nslots,
                                                    NodeRec* __restrict__ parents, int64_t* __restrict__ pfirst,
                                                    TaskRec* __restrict__ tasks, const Plan* P)
{
    const int status = P->status;
    if (status != PLAN_OK && status != PLAN_SPLIT) return;
    __shared__ int64_t sh[32];
    const int j = threadIdx.x;
    for (int si = blockIdx.y; si < nslots; si += gridDim.y) {
        SearchDev& f = S[si];
        if (!f.ctl->active || f.ctl->err) continue;
        const int64_t npop = f.ctl->n_pop;
        for (int64_t i = blockIdx.x; i < npop; i += gridDim.x) {
            const int32_t ch = f.pop_ids[i];
            const int64_t start = poff[si] + f.pop_start[i];
            const int64_t tbase = toff[si] + f.pop_tstart[i];
            const int32_t fill = pool.chunk_fill[ch];
            NodeRec nd;
            int32_t lo[3], ext[3], T = 0;
            if (j < fill) {
                nd = pool.nodes[(int64_t)ch * CH + j];
                T = rot_children(f.grid, rl_level(nd.rl), rl_rot(nd.rl), lo, ext);
            }
            int64_t tot;
            const int64_t first = tbase + block_excl_scan(T, &tot, sh);   // synchronizes: every node is read
            if (j < fill) {
                parents[start + j] = nd;
                pfirst[start + j] = first;
                if (status == PLAN_OK && T > 0) {
                    if (first + T <= TASK_CAP) write_tasks(f, nd, start + j, lo, ext, 0, T, tasks, first);
                    else atomicOr(&f.ctl->err, 4);   // task counts disagree with the nodes: fail the search
                }
            }
            if (j == 0) {
                if (tot != pool.chunk_tasks[ch]) atomicOr(&f.ctl->err, 4);   // the chunk's task count is stale
                const unsigned long long pos = atomicAdd(pool.free_top, 1ull);
                pool.free_ids[pos] = ch;
                pool.chunk_bucket[ch] = -1;
            }
        }
    }
}

// the tasks [ga, gb) of one search's round (gathered parents [p0, p1), their
// first tasks in pfirst) -> tasks[la ..]: a round scored in several launches
__global__ void expand_kernel(const SearchDev* S, int sid, const NodeRec* __restrict__ parents,
                              const int64_t* __restrict__ pfirst, int64_t p0, int64_t p1, int64_t ga, int64_t gb,
                              int64_t la, TaskRec* __restrict__ tasks)
{
    const SearchDev& f = S[sid];
    const DevGrid& g = f.grid;
    for (int64_t p = p0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < p1; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = pfirst[p];
        if (b >= gb) continue;
        const NodeRec nd = parents[p];
        int32_t lo[3], ext[3];
        const int32_t T = rot_children(g, rl_level(nd.rl), rl_rot(nd.rl), lo, ext);
        if (b + T <= ga) continue;
        const int32_t t0 = (int32_t)(ga > b ? ga - b : 0), t1 = (int32_t)(gb < b + T ? gb - b : T);
        write_tasks(f, nd, p, lo, ext, t0, t1, tasks, la + b - ga);
    }
}

// The plan of the next scoring round, built on the device from every live
// search's popped parents: per-search parent and task offsets and one task
// run per search.  It ends the device-driven loop (sets the graph's while
// condition to 0) when no search popped anything, when the round's tasks do
// not fit one launch or the run table (the host finishes that round), or after
// P->max_iters iterations.
__global__ void __launch_bounds__(1024) plan_kernel(SearchDev* S, int nslots, Plan* P, int64_t* poff, int64_t* toff,
                                                    unsigned long long* surv_count, cudaGraphConditionalHandle cond)
{
    __shared__ int64_t sh[32];
    const int tid = threadIdx.x;
    if (tid == 0) *surv_count = 0;
    int64_t cp = 0, ct = 0, cs = 0, cn = 0;
    for (int base = 0; base < nslots; base += blockDim.x) {
        const int s = base + tid;
        int64_t np = 0, nt = 0, sl = 0, has = 0;
        if (s < nslots) {
            const Ctl* c = S[s].ctl;
            if (c->active && !c->done && !c->err) {
                np = c->n_parents;
                nt = c->n_tasks;
            }
            sl = nt * S[s].nblk;
            has = nt > 0;
        }
        int64_t tp, tt, ts, tn;
        const int64_t ep = block_excl_scan(np, &tp, sh);
        const int64_t et = block_excl_scan(nt, &tt, sh);
        const int64_t es = block_excl_scan(sl, &ts, sh);
        const int64_t en = block_excl_scan(has, &tn, sh);
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
                g.pad = 0;
            }
        }
        cp += tp;
        ct += tt;
        cs += ts;
        cn += tn;
    }
    if (tid == 0) {
        P->nseg = (int32_t)(cn < MAXSEG ? cn : MAXSEG);
        P->n_slices = cs;
        P->n_tasks = ct;
        P->next_slice = 0;
        P->mode = MODE_SEARCH;
        int st = PLAN_OK;
        if (cp == 0) st = PLAN_EMPTY;
        else if (cn > MAXSEG || ct > TASK_CAP) st = PLAN_OVERFLOW;
        P->status = st;
        P->iters += 1;
        if (st != PLAN_OK || P->iters >= P->max_iters) cudaGraphSetConditional(cond, 0);
    }
}

// ---- host engine ---------------------------------------------------------------

namespace {

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int64_t floor_div2(int64_t x) { return x >= 0 ? x / 2 : -((-x + 1) / 2); }

}  // namespace

Engine::Engine(cudaStream_t st, int max_slots, int64_t pool_nodes, bool timed)
    : st_(st), max_slots_(max_slots), timed_(timed)
{
    nchunks_ = (pool_nodes + CH - 1) / CH;
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
    if (h_poff_) cudaFreeHost(h_poff_);
    if (h_toff_) cudaFreeHost(h_toff_);
    if (h_misc_) cudaFreeHost(h_misc_);
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
    BBS_TRY(get(&pool_.nodes, (size_t)(nchunks_ * CH)));
    BBS_TRY(get(&pool_.chunk_bucket, (size_t)nchunks_));
    BBS_TRY(get(&pool_.chunk_fill, (size_t)nchunks_));
    BBS_TRY(get(&pool_.chunk_tasks, (size_t)nchunks_));
    BBS_TRY(get(&pool_.free_ids, (size_t)nchunks_));
    BBS_TRY(get(&pool_.free_top, 1));
    pool_.nchunks = nchunks_;
    BBS_TRY(get(&d_S_, (size_t)max_slots_));
    BBS_TRY(get(&d_ctl_, (size_t)max_slots_));
    BBS_TRY(get(&parents_, (size_t)(nchunks_ * CH)));
    BBS_TRY(get(&pfirst_, (size_t)(nchunks_ * CH)));
    BBS_TRY(get(&tasks_, (size_t)TASK_CAP));
    BBS_TRY(get(&d_poff_, (size_t)max_slots_));
    BBS_TRY(get(&d_toff_, (size_t)max_slots_));
    BBS_TRY(get(&d_plan_, 1));
    BBS_TRY(get(&d_slots_, (size_t)max_slots_));
    BBS_TRY(get(&dense_, (size_t)DENSE_CAP));
    BBS_TRY(get(&surv_.nodes, (size_t)DENSE_CAP));
    BBS_TRY(get(&surv_.scores, (size_t)DENSE_CAP));
    BBS_TRY(get(&surv_.sid, (size_t)DENSE_CAP));
    BBS_TRY(get(&surv_.ntask, (size_t)DENSE_CAP));
    BBS_TRY(get(&surv_.count, 1));
    BBS_TRY(get(&surv_.err, 1));
    surv_.cap = DENSE_CAP;
    BBS_CUDA_TRY(cudaMemsetAsync(d_ctl_, 0, sizeof(Ctl) * (size_t)max_slots_, st_));
    BBS_CUDA_TRY(cudaMemsetAsync(d_S_, 0, sizeof(SearchDev) * (size_t)max_slots_, st_));
    BBS_CUDA_TRY(cudaMemsetAsync(surv_.count, 0, sizeof(unsigned long long), st_));
    BBS_CUDA_TRY(cudaMemsetAsync(surv_.err, 0, sizeof(int), st_));
    BBS_CUDA_TRY(cudaMemsetAsync(d_plan_, 0, sizeof(Plan), st_));
    BBS_CUDA_TRY(cudaMemsetAsync(dense_, 0, sizeof(int32_t) * (size_t)DENSE_CAP, st_));
    BBS_CUDA_TRY(cudaMallocHost((void**)&h_ctl_, sizeof(Ctl) * (size_t)max_slots_));
    BBS_CUDA_TRY(cudaMallocHost((void**)&h_poff_, sizeof(int64_t) * (size_t)max_slots_));
    BBS_CUDA_TRY(cudaMallocHost((void**)&h_toff_, sizeof(int64_t) * (size_t)max_slots_));
    BBS_CUDA_TRY(cudaMallocHost((void**)&h_misc_, 4 * sizeof(int32_t)));
    std::memset(h_misc_, 0, 4 * sizeof(int32_t));
    {
        int dev = 0, nsm = 0;
        BBS_CUDA_TRY(cudaGetDevice(&dev));
        BBS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        if (nsm > 0) nsm_ = nsm;
    }
    std::memset(h_ctl_, 0, sizeof(Ctl) * (size_t)max_slots_);
    // every slot's record points at its control block even while unused
    std::vector<SearchDev> blank((size_t)max_slots_);
    for (int i = 0; i < max_slots_; ++i) {
        std::memset(&blank[(size_t)i], 0, sizeof(SearchDev));
        blank[(size_t)i].ctl = d_ctl_ + i;
    }
    BBS_CUDA_TRY(cudaMemcpyAsync(d_S_, blank.data(), sizeof(SearchDev) * blank.size(), cudaMemcpyHostToDevice, st_));
    BBS_CUDA_TRY(cudaStreamSynchronize(st_));   // the host copy above must outlive its transfer
    pool_init_kernel<<<(int)std::min<int64_t>((nchunks_ + 255) / 256, 4096), 256, 0, st_>>>(pool_);
    launches_ += 1;
    BBS_CUDA_TRY(cudaGetLastError());
    return BBS_OK;
}

int Engine::begin_run(cudaStream_t st, bool timed)
{
    st_ = st;
    timed_ = timed;
    score_ms_ = 0.0;
    launches_ = 0;
    score_launches_ = 0;
    for (cudaEvent_t e : evs_) cudaEventDestroy(e);
    evs_.clear();
    BBS_CUDA_TRY(cudaMemsetAsync(surv_.err, 0, sizeof(int), st_));
    BBS_CUDA_TRY(cudaMemsetAsync(surv_.count, 0, sizeof(unsigned long long), st_));
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
           sizeof(double2) * (size_t)g.n_cs + 68 * K1 +
           24 * (size_t)nchunks_ + 1024;
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
    else if (k > (1 << 24)) rc = set_error(BBS_EINVAL, "localize: more than 2^24 scan points");
    if (rc == BBS_OK) rc = scan_prepare(m, xyz, k, is_device, rg, opts, st_, &h.scan);
    if (rc < 0) {
        release(i);
        return rc;
    }
    const HostGrid& g = h.scan.grid;
    h.bytes += estimate_bytes(k, g) - (68 * ((size_t)k + 1) + 24 * (size_t)nchunks_ + 1024);
    h.thr = (int32_t)std::ceil(frac * (double)k);
    h.res.phase_ms[0] = now_ms() - h.t0;
    h.res.h2d_bytes += h.scan.h2d;
    h.res.d2h_bytes += h.scan.d2h;
    h.res.launches += 2;
    if (k == 0) return BBS_OK;   // never live: reported as not found
    SearchDev& d = h.dev;
    std::memset(&d, 0, sizeof(d));
    d.scan = h.scan.scan;
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
    if (rc == BBS_OK) rc = slot_get(h, &d.b_tail, K1);
    if (rc == BBS_OK) rc = slot_get(h, &d.h_cnt, K1);
    if (rc == BBS_OK) rc = slot_get(h, &d.h_kids, K1);
    if (rc == BBS_OK) rc = slot_get(h, &d.h_leaf, K1);
    if (rc == BBS_OK) rc = slot_get(h, &d.w_pos, K1);
    if (rc == BBS_OK) rc = slot_get(h, &d.w_space, K1);
    if (rc == BBS_OK) rc = slot_get(h, &d.w_choff, K1);
    if (rc == BBS_OK) rc = slot_get(h, &d.w_tail, K1);
    if (rc == BBS_OK) rc = slot_get(h, &d.w_fill0, K1);
    if (rc == BBS_OK) rc = slot_get(h, &d.act, (size_t)nchunks_);
    if (rc == BBS_OK) rc = slot_get(h, &d.pop_ids, (size_t)nchunks_);
    if (rc == BBS_OK) rc = slot_get(h, &d.pop_start, (size_t)nchunks_);
    if (rc == BBS_OK) rc = slot_get(h, &d.pop_tstart, (size_t)nchunks_);
    if (rc < 0) {
        release(i);
        return rc;
    }
    h.ctl0 = Ctl();
    h.ctl0.best = h.thr - 1;
    h.ctl0.top = -1;
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
    for (int i = 0; i < max_slots_; ++i)
        if (hosts_[(size_t)i].fresh) slots.push_back(i);
    if (slots.empty()) return BBS_OK;
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
        BBS_TRY(score_launch(MODE_INITIAL, segs, nsl, ntk));
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
        for (int64_t v0 = 0; v0 < vpn;) {
            const int64_t take = std::min<int64_t>(vpn - v0, (TASK_CAP - ntk) / R);
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
            segs.push_back(sg);
            ntk += take * R;
            nsl += take * R * h.dev.nblk;
            h.res.gathers += take * R * h.scan.k;
            v0 += take;
        }
    }
    BBS_TRY(flush());
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
    BBS_CUDA_TRY(cudaMemcpyAsync(&h_misc_[2], surv_.err, sizeof(int32_t), cudaMemcpyDeviceToHost, st_));
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
            // the shared pool ran out while this search inserted, or its
            // bookkeeping failed a check: it fails alone
            if (c.err & 4) h.status = set_error(BBS_ECORRUPT, "localize: frontier task counts are inconsistent");
            else
                h.status = set_error(BBS_ENOMEM, "localize: the frontier pool (%lld nodes) is exhausted",
                                     (long long)(nchunks_ * CH));
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

// host-side scoring of the parents the last select popped (h_ctl_ is current):
// one launch when the round's tasks fit, else launches over task windows
int Engine::process_popped()
{
    const int n = max_slots_;
    int64_t total_parents = 0, total_tasks = 0, maxpop = 1, nsearch = 0;
    for (int i = 0; i < n; ++i) {
        h_poff_[i] = total_parents;
        h_toff_[i] = total_tasks;
        if (!hosts_[(size_t)i].live) continue;
        total_parents += h_ctl_[i].n_parents;
        total_tasks += h_ctl_[i].n_tasks;
        nsearch += h_ctl_[i].n_tasks > 0 ? 1 : 0;
        maxpop = std::max<int64_t>(maxpop, h_ctl_[i].n_pop);
    }
    if (total_parents == 0) return BBS_OK;
    const bool one = total_tasks <= TASK_CAP && nsearch <= MAXSEG;
    BBS_CUDA_TRY(cudaMemcpyAsync(d_poff_, h_poff_, sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, st_));
    BBS_CUDA_TRY(cudaMemcpyAsync(d_toff_, h_toff_, sizeof(int64_t) * (size_t)n, cudaMemcpyHostToDevice, st_));
    h_plan_.status = one ? PLAN_OK : PLAN_SPLIT;
    h_plan_.nseg = 0;
    BBS_CUDA_TRY(cudaMemcpyAsync(d_plan_, &h_plan_, offsetof(Plan, seg), cudaMemcpyHostToDevice, st_));
    dim3 gg((unsigned)std::min<int64_t>(maxpop, 4096), (unsigned)std::min(n, 65535));
    gather_kernel<<<gg, CH, 0, st_>>>(d_S_, pool_, d_poff_, d_toff_, n, parents_, pfirst_, tasks_, d_plan_);
    launches_ += 1;
    BBS_CUDA_TRY(cudaGetLastError());
    std::vector<Seg> segs;
    int64_t nsl = 0, ntk = 0;
    auto flush = [&]() -> int {
        if (segs.empty()) return BBS_OK;
        BBS_TRY(score_launch(MODE_SEARCH, segs, nsl, ntk));
        segs.clear();
        nsl = ntk = 0;
        return BBS_OK;
    };
    for (int i = 0; i < n; ++i) {
        SearchHost& h = hosts_[(size_t)i];
        if (!h.live) continue;
        const int64_t nt = h_ctl_[i].n_tasks;
        for (int64_t t0 = 0; t0 < nt;) {
            const int64_t take = std::min<int64_t>(nt - t0, TASK_CAP - ntk);
            if (take <= 0 || (int)segs.size() == MAXSEG) {
                BBS_TRY(flush());
                continue;
            }
            if (!one) {   // the window's task records, from the gathered parents
                const int64_t np = h_ctl_[i].n_parents;
                const int blocks = (int)std::min<int64_t>((np + 255) / 256, 4096);
                expand_kernel<<<blocks, 256, 0, st_>>>(d_S_, i, parents_, pfirst_, h_poff_[i], h_poff_[i] + np,
                                                       h_toff_[i] + t0, h_toff_[i] + t0 + take, ntk, tasks_);
                launches_ += 1;
                BBS_CUDA_TRY(cudaGetLastError());
            }
            Seg sg;
            std::memset(&sg, 0, sizeof(sg));
            sg.first_parent = h_poff_[i];
            sg.first_task = one ? h_toff_[i] + t0 : ntk;
            sg.n_tasks = take;
            sg.first_slice = nsl;
            sg.sid = i;
            sg.nblk = h.dev.nblk;
            segs.push_back(sg);
            ntk += take;
            nsl += take * h.dev.nblk;
            t0 += take;
        }
    }
    if (one) ntk = total_tasks;
    return flush();
}

int Engine::step(std::vector<int>* finished)
{
    finish_never_live(finished);
    if (live_count() == 0) return BBS_OK;
    select_kernel<<<max_slots_, 1024, 0, st_>>>(d_S_, max_slots_, pool_);
    launches_ += 1;
    BBS_CUDA_TRY(cudaGetLastError());
    BBS_TRY(read_ctl());
    mark_finished(finished);
    return process_popped();
}

int Engine::build_graph()
{
    const int n = max_slots_;
    cudaStream_t cs;
    BBS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
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
    cudaGraph_t body = e == cudaSuccess ? np.conditional.phGraph_out[0] : nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // one iteration: select, plan, gather, score, survivors, insert
        select_kernel<<<n, 1024, 0, cs>>>(d_S_, n, pool_);
        plan_kernel<<<1, 1024, 0, cs>>>(d_S_, n, d_plan_, d_poff_, d_toff_, surv_.count, cond);
        gather_kernel<<<dim3(256, (unsigned)std::min(n, 65535)), CH, 0, cs>>>(d_S_, pool_, d_poff_, d_toff_, n, parents_,
                                                                              pfirst_, tasks_, d_plan_);
        launch_task_rows(d_plan_, d_S_, tasks_, nsm_ * 4, cs);
        launch_branch(MODE_SEARCH, d_plan_, d_S_, parents_, tasks_, dense_, nsm_ * BRANCH_CTAS_PER_SM, cs);
        launch_finalize(MODE_SEARCH, d_plan_, d_S_, parents_, tasks_, dense_, surv_, nsm_ * 8, cs);
        alloc_kernel<<<n, 1024, 0, cs>>>(d_S_, n, pool_, d_plan_);
        scatter_kernel<<<1024, 256, 0, cs>>>(d_S_, pool_, surv_.nodes, surv_.scores, surv_.sid, surv_.ntask, surv_.count,
                                             surv_.cap);
        cudaGraph_t out = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &out);
        e = e2 != cudaSuccess ? e2 : cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec_, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        exec_ = nullptr;
        return set_error(BBS_ECUDA, "engine: building the iteration graph: %s", cudaGetErrorString(e));
    }
    return BBS_OK;
}

int Engine::iterate(int max_iters, std::vector<int>* finished)
{
    // CUDA events cannot sit inside the graph's loop body: timed runs take
    // the host-driven path, whose scoring launches are the same kernels
    if (host_driven_ || timed_) return step(finished);
    finish_never_live(finished);
    if (live_count() == 0) return BBS_OK;
    if (!exec_) BBS_TRY(build_graph());
    h_plan_.iters = 0;
    h_plan_.max_iters = max_iters > 0 ? max_iters : 1;
    BBS_CUDA_TRY(cudaMemcpyAsync(&d_plan_->iters, &h_plan_.iters, 2 * sizeof(int32_t), cudaMemcpyHostToDevice, st_));
    BBS_CUDA_TRY(cudaGraphLaunch(exec_, st_));
    // status and the iterations the device loop ran, with the control blocks
    BBS_CUDA_TRY(cudaMemcpyAsync(h_misc_, &d_plan_->status, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st_));
    BBS_TRY(read_ctl());
    const int32_t status = h_misc_[0];
    launches_ += 8 * (int64_t)h_misc_[1];   // every iteration of the loop runs the body's 8 kernels
    mark_finished(finished);
    if (status == PLAN_OVERFLOW) return process_popped();   // the selected round did not fit on the device
    return BBS_OK;
}

int Engine::finalize(int i, bbs_result* out)
{
    SearchHost& h = hosts_[(size_t)i];
    // the control block and the staging error flag as the last read_ctl saw
    // them: a finished search's block no longer changes
    const int herr = h_misc_[2];
    Ctl c;
    std::memset(&c, 0, sizeof(c));
    if (h.scan.k > 0) c = h_ctl_[i];
    if (!evs_.empty()) BBS_CUDA_TRY(cudaEventSynchronize(evs_.back()));
    for (size_t e = 0; e + 1 < evs_.size(); e += 2) {
        float ms = 0.0f;
        BBS_CUDA_TRY(cudaEventElapsedTime(&ms, evs_[e], evs_[e + 1]));
        score_ms_ += ms;
    }
    for (cudaEvent_t e : evs_) cudaEventDestroy(e);
    evs_.clear();
    bbs_result* r = &h.res;
    const double t_fin = now_ms();
    if (h.t_end == 0) h.t_end = t_fin;
    r->launches += launches_;
    r->score_launches = score_launches_;
    r->score_ms = score_ms_;
    int status;
    if (herr) {
        status = set_error(BBS_ECORRUPT, "localize: survivor staging overflow");
    } else if (h.status < 0) {
        status = h.status;
    } else if (h.scan.k == 0) {
        r->best_score = h.thr - 1;
        status = BBS_NOT_FOUND;
    } else {
        const HostGrid& g = h.scan.grid;
        r->iterations = c.st_iters;
        r->parents_branched = c.st_parents;
        r->nodes_scored += c.st_nodes;
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
        if (c.found) {
            const NodeRec& nd = c.match;
            const uint32_t rot = rl_rot(nd.rl);
            const int64_t ng = g.N[0][2], nb = g.N[0][1];
            r->found = 1;
            r->node[0] = nd.cx;
            r->node[1] = nd.cy;
            r->node[2] = nd.cz;
            r->node[3] = (int32_t)(rot / (ng * nb));
            r->node[4] = (int32_t)((rot / ng) % nb);
            r->node[5] = (int32_t)(rot % ng);
            r->node[6] = 0;
            for (int a = 0; a < 3; ++a) r->pose[a] = (double)r->node[a] * g.r;
            for (int a = 0; a < 3; ++a) r->pose[3 + a] = grid_angle(g, 0, a, r->node[3 + a]);
            r->ms_to_optimum = r->phase_ms[0] + dev_match;
            status = BBS_OK;
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
    // chunks still held (a search stopped early) go back to the pool
    if (h.dev.K > 0 && d_S_) {
        slot_release_kernel<<<1, 1024, 0, st_>>>(d_S_, i, pool_);
        launches_ += 1;
    }
    Ctl z;
    std::memset(&z, 0, sizeof(z));
    h_ctl_[i] = z;
    if (d_ctl_) cudaMemcpyAsync(d_ctl_ + i, &h_ctl_[i], sizeof(Ctl), cudaMemcpyHostToDevice, st_);
    for (void* p : h.bufs) cudaFreeAsync(p, st_);
    scan_release(&h.scan, st_);
    cudaError_t e = cudaStreamSynchronize(st_);   // the zeroed control block must land before the slot is reused
    h = SearchHost();
    if (e != cudaSuccess) return set_error(BBS_ECUDA, "engine: %s", cudaGetErrorString(e));
    return BBS_OK;
}

int Engine::score_launch(int mode, const std::vector<Seg>& segs, int64_t n_slices, int64_t n_tasks)
{
    h_plan_.n_slices = n_slices;
    h_plan_.n_tasks = n_tasks;
    h_plan_.next_slice = 0;
    h_plan_.nseg = (int32_t)segs.size();
    h_plan_.mode = mode;
    h_plan_.status = PLAN_OK;
    for (size_t i = 0; i < segs.size(); ++i) h_plan_.seg[i] = segs[i];
    // pageable source: staged before cudaMemcpyAsync returns, so h_plan_ may be rewritten
    BBS_CUDA_TRY(cudaMemcpyAsync(d_plan_, &h_plan_, offsetof(Plan, seg) + sizeof(Seg) * segs.size(),
                                 cudaMemcpyHostToDevice, st_));
    if (mode == MODE_SEARCH) {
        BBS_CUDA_TRY(launch_task_rows(d_plan_, d_S_, tasks_, (int)std::min<int64_t>((n_tasks + 31) / 32, 4 * nsm_), st_));
        launches_ += 1;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timed_) {
        BBS_CUDA_TRY(cudaEventCreate(&e0));
        evs_.push_back(e0);
        BBS_CUDA_TRY(cudaEventCreate(&e1));
        evs_.push_back(e1);
        BBS_CUDA_TRY(cudaEventRecord(e0, st_));
    }
    const int bb = (int)std::min<int64_t>(n_slices, (int64_t)nsm_ * BRANCH_CTAS_PER_SM);
    BBS_CUDA_TRY(launch_branch(mode, d_plan_, d_S_, parents_, tasks_, dense_, bb, st_));
    if (timed_) BBS_CUDA_TRY(cudaEventRecord(e1, st_));
    // the device-driven loop leaves its last round's survivor count behind
    BBS_CUDA_TRY(cudaMemsetAsync(surv_.count, 0, sizeof(unsigned long long), st_));
    const int fb = (int)std::min<int64_t>((8 * n_tasks + 255) / 256, (int64_t)nsm_ * 32);
    BBS_CUDA_TRY(launch_finalize(mode, d_plan_, d_S_, parents_, tasks_, dense_, surv_, fb, st_));
    alloc_kernel<<<max_slots_, 1024, 0, st_>>>(d_S_, max_slots_, pool_, d_plan_);
    scatter_kernel<<<1024, 256, 0, st_>>>(d_S_, pool_, surv_.nodes, surv_.scores, surv_.sid, surv_.ntask, surv_.count,
                                          surv_.cap);
    BBS_CUDA_TRY(cudaMemsetAsync(surv_.count, 0, sizeof(unsigned long long), st_));
    BBS_CUDA_TRY(cudaGetLastError());
    launches_ += 4;
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
    const int64_t max_frontier = (opts && opts->max_frontier > 0) ? opts->max_frontier : ((int64_t)1 << 24);
    const bool timed = opts && (opts->flags & BBS_TIME_KERNELS);
    const int64_t pool_nodes = max_frontier + (int64_t)CH * std::min<int64_t>(k + 1, 8192);
    std::memset(res, 0, sizeof(*res));
    int rc = BBS_OK;
    Engine* E = acquire_engine(1, pool_nodes, st, timed, &rc);
    if (!E) return rc;
    int slot = -1;
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
    const int64_t max_frontier = (opts && opts->max_frontier > 0) ? opts->max_frontier : ((int64_t)1 << 24);
    const bool timed = opts && (opts->flags & BBS_TIME_KERNELS);
    int64_t kmax = 1;
    for (int i = 0; i < n; ++i) kmax = std::max(kmax, ks[i]);
    const int64_t pool_nodes = max_frontier + (int64_t)CH * std::min<int64_t>((kmax + 1) * n, 8192 * (int64_t)n);
    int rc = BBS_OK;
    Engine* E = acquire_engine(n, pool_nodes, st, timed, &rc);
    if (!E) return rc;
    std::vector<int> slot_of((size_t)n, -1);
    for (int i = 0; i < n && rc == BBS_OK; ++i) {
        std::memset(&res[i], 0, sizeof(res[i]));
        rc = E->add(m, scans[i], ks[i], is_device, rg, opts, (uint64_t)i, &slot_of[(size_t)i]);
    }
    if (rc == BBS_OK) rc = E->start();
    E->set_host_driven(opts && (opts->flags & BBS_HOST_DRIVEN));
    std::vector<int> fin;
    while (rc == BBS_OK && E->used_count() > 0) {
        fin.clear();
        rc = E->iterate(1 << 20, &fin);
        for (int s_ : fin) E->finalize(s_, &res[E->tag(s_)]);
    }
    release_engine(E, rc == BBS_OK);
    return rc;
}

}  // namespace bbs
