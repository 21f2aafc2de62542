// search.cu -- device-resident best-first batched BnB (Sec. III-E, Algorithm 2).
//
// Frontier F: scored nodes bucketed by integer score.  Nodes live in chunks of
// CH node records drawn from a free-chunk stack; every non-empty bucket owns
// its chunks (all full except its tail), and the list of chunks in use (the
// "active list") tags each chunk with its bucket.
//
// One iteration of the canonical batched best-first rule:
//   select  (1 CTA)  walk buckets from the top with a block-wide prefix of their
//                    children counts; the first bucket reached with
//                    children(P) >= b stops the pop, one at or below best clears
//                    F, one holding a leaf sets (best, lexmin leaf) and clears F;
//                    every bucket above it is popped whole.
//   gather           popped chunks -> a dense parent array; chunks freed.
//   branch (score.cu) every child of every parent scored; survivors > best
//                    staged with per-score histograms.
//   alloc   (1 CTA)  chunks for each bucket's survivors from the free stack.
//   scatter          survivors into their buckets' chunks.
// Only popping a leaf changes best, so how a batch is split into launches and
// in which order survivors land in a bucket cannot change the result.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "branch.cuh"

namespace bbs {

constexpr int CH = 256;   // nodes per frontier chunk

struct Ctl {
    int32_t best;          // provisional best score (threshold - 1 at start)
    int32_t top;           // every bucket above top is empty
    int32_t found;
    int32_t done;
    NodeRec match;
    int64_t size;          // nodes in F
    int64_t n_parents;     // parents popped by the last select
    int64_t n_pop;         // chunks popped by the last select
    unsigned long long free_top;   // height of the free-chunk stack
    int64_t n_act;         // chunks in use
    unsigned long long surv;       // survivors staged
    int32_t err;           // 1 pool exhausted, 2 staging overflow
    int32_t reason;        // last select: 1 batch full, 2 below best, 3 leaf, 4 F emptied, 0 F was empty
    int64_t popped_kids;   // children of the parents popped by the last select
    int32_t match_changed;
    int32_t pad;
};

struct FrontierDev {
    int32_t K;
    int64_t nchunks;
    int64_t batch;
    NodeRec* pool;
    int32_t* chunk_bucket;
    int32_t* chunk_fill;
    int32_t* free_ids;
    int32_t* act;
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
    int32_t* new_chunks;
    int32_t* pop_ids;
    int64_t* pop_start;
    NodeRec* parents;
    const NodeRec* surv_nodes;
    const int32_t* surv_scores;
    int64_t surv_cap;
    Ctl* ctl;
};

// ---- block helpers (1024 threads) -------------------------------------------

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
    if (wid == 0) {
        int64_t s = sh[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const int64_t before = (wid > 0 ? sh[wid - 1] : 0) + x - v;
    *total = sh[31];
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

// ---- kernels ------------------------------------------------------------------

__global__ void iota_kernel(int32_t* p, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)(n - 1 - i);
}

__global__ void fill_i32(int32_t* p, int64_t n, int32_t v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

__global__ void __launch_bounds__(1024) alloc_kernel(FrontierDev f)
{
    __shared__ int64_t sh[32];
    __shared__ int64_t s_need_total;
    __shared__ int s_min[33];
    Ctl* c = f.ctl;
    if (c->err) return;
    const int64_t ftop = (int64_t)c->free_top;
    const int64_t act0 = c->n_act;
    // pass 1: total chunks needed
    int64_t need_sum = 0;
    for (int s = threadIdx.x; s <= f.K; s += blockDim.x) {
        const uint32_t h = f.h_cnt[s];
        if (!h) continue;
        const int32_t tail = f.b_tail[s];
        const int32_t space = tail >= 0 ? CH - f.chunk_fill[tail] : 0;
        if ((int64_t)h > space) need_sum += ((int64_t)h - space + CH - 1) / CH;
    }
    int64_t tot;
    block_excl_scan(need_sum, &tot, sh);
    if (threadIdx.x == 0) s_need_total = tot;
    __syncthreads();
    if (s_need_total > ftop) {
        if (threadIdx.x == 0) c->err |= 1;
        return;
    }
    // pass 2: allocate
    int64_t carry = 0, added = 0;
    int top = -1;
    for (int base = 0; base <= f.K; base += blockDim.x) {
        const int s = base + threadIdx.x;
        uint32_t h = 0;
        int32_t tail = -1, fill0 = CH, space = 0;
        int64_t need = 0;
        if (s <= f.K) {
            h = f.h_cnt[s];
            if (h) {
                tail = f.b_tail[s];
                fill0 = tail >= 0 ? f.chunk_fill[tail] : CH;
                space = CH - fill0;
                need = (int64_t)h > space ? ((int64_t)h - space + CH - 1) / CH : 0;
            }
        }
        int64_t total;
        const int64_t off = carry + block_excl_scan(need, &total, sh);
        if (h) {
            int32_t last = tail;
            for (int64_t i = 0; i < need; ++i) {
                const int32_t id = f.free_ids[ftop - 1 - (off + i)];
                f.new_chunks[off + i] = id;
                f.chunk_bucket[id] = s;
                f.chunk_fill[id] = (int32_t)(i < need - 1 ? CH : ((int64_t)h - space) - (need - 1) * CH);
                f.act[act0 + off + i] = id;
                last = id;
            }
            if (tail >= 0) f.chunk_fill[tail] = fill0 + (int32_t)((int64_t)h < space ? h : space);
            f.w_space[s] = space;
            f.w_choff[s] = off;
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
        c->free_top = (unsigned long long)(ftop - carry);
        c->n_act = act0 + carry;
        c->size += all_added;
        if (maxtop > c->top) c->top = maxtop;
    }
}

__global__ void scatter_kernel(FrontierDev f)
{
    const Ctl* c = f.ctl;
    if (c->err) return;
    int64_t n = (int64_t)c->surv;
    if (n > f.surv_cap) n = f.surv_cap;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = f.surv_scores[i];
        const uint32_t rank = atomicAdd(&f.w_pos[s], 1u);
        int32_t chunk, slot;
        if ((int32_t)rank < f.w_space[s]) {
            chunk = f.w_tail[s];
            slot = f.w_fill0[s] + (int32_t)rank;
        } else {
            const int64_t idx = (int64_t)rank - f.w_space[s];
            chunk = f.new_chunks[f.w_choff[s] + idx / CH];
            slot = (int32_t)(idx % CH);
        }
        f.pool[(int64_t)chunk * CH + slot] = f.surv_nodes[i];
    }
}

__global__ void __launch_bounds__(1024) select_kernel(FrontierDev f)
{
    __shared__ int64_t sh[32];
    __shared__ int s_min[33];
    __shared__ int32_t s_star, s_reason;
    __shared__ LexKey s_lex[1024];
    __shared__ NodeRec s_node[1024];
    __shared__ int s_has[1024];
    Ctl* c = f.ctl;
    if (c->err) return;
    const int32_t best = c->best;
    const int tid = threadIdx.x;
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
    // 2. the active list: pop chunks above s*, free the rest when clearing,
    //    lexmin leaf of bucket s* on a leaf stop
    LexKey my_lex;
    my_lex.t = ~0ull;
    my_lex.r = ~0u;
    NodeRec my_node;
    my_node.cx = my_node.cy = my_node.cz = 0;
    my_node.rl = 0;
    int my_has = 0;
    const int64_t n_act = c->n_act;
    int64_t keep = 0, npop = 0, nfree = 0, nparents = 0;
    const int64_t ftop = (int64_t)c->free_top;
    for (int64_t base = 0; base < n_act; base += blockDim.x) {
        const int64_t i = base + tid;
        const int32_t ch = i < n_act ? f.act[i] : -1;
        const int32_t bk = ch >= 0 ? f.chunk_bucket[ch] : -1;
        const int32_t fill = ch >= 0 ? f.chunk_fill[ch] : 0;
        const bool popped = ch >= 0 && bk > sstar;
        const bool freed = ch >= 0 && !popped && clear;
        const bool kept = ch >= 0 && !popped && !clear;
        if (reason == 3 && ch >= 0 && bk == sstar) {
            for (int j = 0; j < fill; ++j) {
                const NodeRec nd = f.pool[(int64_t)ch * CH + j];
                if (rl_level(nd.rl) != 0) continue;
                const LexKey k = lex_of(nd);
                if (!my_has || lex_lt(k, my_lex)) {
                    my_lex = k;
                    my_node = nd;
                    my_has = 1;
                }
            }
        }
        int64_t t1, t2, t3, t4;
        const int64_t rp = block_excl_scan(popped ? 1 : 0, &t1, sh);
        const int64_t rf = block_excl_scan(freed ? 1 : 0, &t2, sh);
        const int64_t rk = block_excl_scan(kept ? 1 : 0, &t3, sh);
        const int64_t rs = block_excl_scan(popped ? fill : 0, &t4, sh);
        if (popped) {
            f.pop_ids[npop + rp] = ch;
            f.pop_start[npop + rp] = nparents + rs;
            f.chunk_bucket[ch] = -2;
        }
        if (freed) {
            f.free_ids[ftop + nfree + rf] = ch;
            f.chunk_bucket[ch] = -1;
        }
        __syncthreads();   // every read of act[base..] is done before the in-place write
        if (kept) f.act[keep + rk] = ch;
        npop += t1;
        nfree += t2;
        keep += t3;
        nparents += t4;
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
    // 4. bucket metadata: popped buckets and (when clearing) everything else
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
        c->popped_kids = pk;
        c->n_act = keep;
        c->free_top = (unsigned long long)(ftop + nfree);
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
    }
}

__global__ void gather_kernel(FrontierDev f)
{
    Ctl* c = f.ctl;
    const int64_t npop = c->n_pop;
    for (int64_t i = blockIdx.x; i < npop; i += gridDim.x) {
        const int32_t ch = f.pop_ids[i];
        const int64_t start = f.pop_start[i];
        const int32_t fill = f.chunk_fill[ch];
        for (int j = threadIdx.x; j < fill; j += blockDim.x) f.parents[start + j] = f.pool[(int64_t)ch * CH + j];
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned long long pos = atomicAdd(&c->free_top, 1ull);
            f.free_ids[pos] = ch;
            f.chunk_bucket[ch] = -1;
        }
    }
}

// ---- host driver ------------------------------------------------------------

namespace {

struct DevBuf {
    cudaStream_t st;
    std::vector<void*> ptrs;
    ~DevBuf()
    {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
    template <class T>
    int get(T** p, size_t n)
    {
        void* q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, n * sizeof(T) + 16, st);
        if (e != cudaSuccess) return set_error(BBS_ENOMEM, "search: cudaMallocAsync(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
        ptrs.push_back(q);
        *p = (T*)q;
        return BBS_OK;
    }
};

double ms_since(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

int64_t floor_div2(int64_t x) { return x >= 0 ? x / 2 : -((-x + 1) / 2); }

}  // namespace

int search_run(const bbs_maps* m, const float* xyz, int64_t k, int is_device, const bbs_ranges* rg,
               const bbs_opts* opts, cudaStream_t st, bbs_result* res)
{
    const auto t0 = std::chrono::steady_clock::now();
    std::memset(res, 0, sizeof(*res));
    res->num_points = (int32_t)k;
    const double frac = (opts && opts->score_frac > 0.0) ? opts->score_frac : 0.95;
    const int64_t batch = (opts && opts->batch > 0) ? opts->batch : 10000;
    const int64_t max_frontier = (opts && opts->max_frontier > 0) ? opts->max_frontier : ((int64_t)1 << 24);
    const uint32_t flags = opts ? opts->flags : 0u;
    if (!(frac > 0.0 && frac <= 1.0)) return set_error(BBS_EINVAL, "localize: score_frac %g outside (0, 1]", frac);
    if (flags & BBS_PRUNE_GE) return set_error(BBS_EINVAL, "localize: BBS_PRUNE_GE is not supported");
    if (k > (1 << 24)) return set_error(BBS_EINVAL, "localize: more than 2^24 scan points");

    ScanState S;
    BBS_TRY(scan_prepare(m, xyz, k, is_device, rg, opts, st, &S));
    struct Rel {
        ScanState* s;
        cudaStream_t st;
        ~Rel() { scan_release(s, st); }
    } rel{&S, st};
    const HostGrid& g = S.grid;
    const int32_t thr = (int32_t)std::ceil(frac * (double)k);
    res->phase_ms[0] = ms_since(t0);
    if (k == 0) {
        res->best_score = thr - 1;
        res->status = BBS_NOT_FOUND;
        res->ms_total = ms_since(t0);
        return BBS_NOT_FOUND;
    }

    // ---- frontier storage ----
    DevBuf B{st, {}};
    FrontierDev f;
    std::memset(&f, 0, sizeof(f));
    f.K = (int32_t)k;
    f.batch = batch;
    const int64_t K1 = k + 1;
    f.nchunks = (max_frontier + CH - 1) / CH + std::min<int64_t>(K1, 8192);
    const int64_t cap_nodes = f.nchunks * CH;
    int rmax = 1;
    for (int l = 1; l < g.levels; ++l) rmax = std::max<int>(rmax, (int)(g.a[l][0] * g.a[l][1] * g.a[l][2]));
    const int64_t surv_cap = (int64_t)1 << 22;
    f.surv_cap = surv_cap;
    BBS_TRY(B.get(&f.pool, (size_t)cap_nodes));
    BBS_TRY(B.get(&f.chunk_bucket, (size_t)f.nchunks));
    BBS_TRY(B.get(&f.chunk_fill, (size_t)f.nchunks));
    BBS_TRY(B.get(&f.free_ids, (size_t)f.nchunks));
    BBS_TRY(B.get(&f.act, (size_t)f.nchunks));
    BBS_TRY(B.get(&f.new_chunks, (size_t)f.nchunks));
    BBS_TRY(B.get(&f.pop_ids, (size_t)f.nchunks));
    BBS_TRY(B.get(&f.pop_start, (size_t)f.nchunks));
    BBS_TRY(B.get(&f.parents, (size_t)cap_nodes));
    BBS_TRY(B.get(&f.b_cnt, (size_t)K1));
    BBS_TRY(B.get(&f.b_kids, (size_t)K1));
    BBS_TRY(B.get(&f.b_leaf, (size_t)K1));
    BBS_TRY(B.get(&f.b_tail, (size_t)K1));
    BBS_TRY(B.get(&f.h_cnt, (size_t)K1));
    BBS_TRY(B.get(&f.h_kids, (size_t)K1));
    BBS_TRY(B.get(&f.h_leaf, (size_t)K1));
    BBS_TRY(B.get(&f.w_pos, (size_t)K1));
    BBS_TRY(B.get(&f.w_space, (size_t)K1));
    BBS_TRY(B.get(&f.w_choff, (size_t)K1));
    BBS_TRY(B.get(&f.w_tail, (size_t)K1));
    BBS_TRY(B.get(&f.w_fill0, (size_t)K1));
    NodeRec* surv_nodes;
    int32_t* surv_scores;
    int* d_err;
    BBS_TRY(B.get(&surv_nodes, (size_t)surv_cap));
    BBS_TRY(B.get(&surv_scores, (size_t)surv_cap));
    BBS_TRY(B.get(&f.ctl, 1));
    BBS_TRY(B.get(&d_err, 1));
    f.surv_nodes = surv_nodes;
    f.surv_scores = surv_scores;

    const int nb = (int)std::min<int64_t>((f.nchunks + 255) / 256, 4096);
    const int kb = (int)std::min<int64_t>((K1 + 255) / 256, 4096);
    fill_i32<<<nb, 256, 0, st>>>(f.chunk_bucket, f.nchunks, -1);
    iota_kernel<<<nb, 256, 0, st>>>(f.free_ids, f.nchunks);
    fill_i32<<<kb, 256, 0, st>>>(f.b_tail, K1, -1);
    BBS_CUDA_TRY(cudaMemsetAsync(f.b_cnt, 0, sizeof(int64_t) * K1, st));
    BBS_CUDA_TRY(cudaMemsetAsync(f.b_kids, 0, sizeof(int64_t) * K1, st));
    BBS_CUDA_TRY(cudaMemsetAsync(f.b_leaf, 0, sizeof(int64_t) * K1, st));
    BBS_CUDA_TRY(cudaMemsetAsync(f.h_cnt, 0, sizeof(uint32_t) * K1, st));
    BBS_CUDA_TRY(cudaMemsetAsync(f.h_kids, 0, sizeof(unsigned long long) * K1, st));
    BBS_CUDA_TRY(cudaMemsetAsync(f.h_leaf, 0, sizeof(uint32_t) * K1, st));
    BBS_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    Ctl hc;
    std::memset(&hc, 0, sizeof(hc));
    hc.best = thr - 1;
    hc.top = -1;
    hc.free_top = (unsigned long long)f.nchunks;
    BBS_CUDA_TRY(cudaMemcpyAsync(f.ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice, st));
    res->h2d_bytes = S.h2d + (int64_t)sizeof(hc);
    res->d2h_bytes = S.d2h;

    BranchArgs ba;
    fill_branch_common(m, S, &ba);
    ba.best = &f.ctl->best;
    ba.surv_nodes = surv_nodes;
    ba.surv_scores = surv_scores;
    ba.surv_count = &f.ctl->surv;
    ba.surv_cap = surv_cap;
    ba.h_cnt = f.h_cnt;
    ba.h_kids = f.h_kids;
    ba.h_leaf = f.h_leaf;
    ba.err = d_err;

    const bool timed = (flags & BBS_TIME_KERNELS) != 0;
    std::vector<cudaEvent_t> evs;
    struct EvRel {
        std::vector<cudaEvent_t>* v;
        ~EvRel()
        {
            for (cudaEvent_t e : *v) cudaEventDestroy(e);
        }
    } evrel{&evs};
    // scoring launch with optional CUDA-event timing on the call's stream
    auto score = [&](int mode, const BranchArgs& a2, int64_t items) -> int {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (timed) {
            BBS_CUDA_TRY(cudaEventCreate(&e0));
            evs.push_back(e0);
            BBS_CUDA_TRY(cudaEventCreate(&e1));
            evs.push_back(e1);
            BBS_CUDA_TRY(cudaEventRecord(e0, st));
        }
        BBS_CUDA_TRY(launch_branch(mode, a2, st));
        if (timed) BBS_CUDA_TRY(cudaEventRecord(e1, st));
        res->score_launches++;
        res->launches++;
        res->gathers += items * k;
        return BBS_OK;
    };
    auto insert = [&]() -> int {
        res->launches += 2;
        alloc_kernel<<<1, 1024, 0, st>>>(f);
        scatter_kernel<<<1024, 256, 0, st>>>(f);
        BBS_CUDA_TRY(cudaMemsetAsync(&f.ctl->surv, 0, sizeof(unsigned long long), st));
        BBS_CUDA_TRY(cudaGetLastError());
        return BBS_OK;
    };

    // ---- initial set C_lmax (Eq. (3)-(5)) --------------------------------
    const int lmax = g.levels - 1;
    ba.init_level = lmax;
    int64_t vpn = 1;
    for (int i = 0; i < 3; ++i) {
        const int64_t pmin = floor_div2(g.wmin[i]), pmax = floor_div2(g.wmax[i]);
        ba.pmin[i] = (int32_t)pmin;
        ba.pext[i] = (int32_t)(pmax - pmin + 1);
        ba.wmin[i] = (int32_t)g.wmin[i];
        ba.wmax[i] = (int32_t)g.wmax[i];
        vpn *= ba.pext[i];
        res->nodes_scored = (i == 0 ? 1 : res->nodes_scored) * (g.wmax[i] - g.wmin[i] + 1);
    }
    res->nodes_scored *= g.nrot[lmax];
    const int64_t init_items = vpn * g.nrot[lmax];
    const int64_t islice = surv_cap / 8;   // every item yields at most 8 survivors
    for (int64_t i0 = 0; i0 < init_items; i0 += islice) {
        BranchArgs a2 = ba;
        a2.item0 = i0;
        a2.n_items = std::min(islice, init_items - i0);
        BBS_TRY(score(MODE_INITIAL, a2, a2.n_items));
        BBS_TRY(insert());
    }
    res->phase_ms[1] = ms_since(t0) - res->phase_ms[0];

    // ---- iterations ---------------------------------------------------------
    const int64_t pslice = std::max<int64_t>(1, surv_cap / (8 * (int64_t)rmax));
    double t_match = -1.0;
    const double t_loop = ms_since(t0);
    int64_t iters = 0;
    for (;;) {
        select_kernel<<<1, 1024, 0, st>>>(f);
        res->launches++;
        BBS_CUDA_TRY(cudaGetLastError());
        BBS_CUDA_TRY(cudaMemcpyAsync(&hc, f.ctl, sizeof(hc), cudaMemcpyDeviceToHost, st));
        BBS_CUDA_TRY(cudaStreamSynchronize(st));
        res->d2h_bytes += (int64_t)sizeof(hc);
        if (hc.err & 1) return set_error(BBS_ENOMEM, "localize: frontier exceeds %lld nodes", (long long)max_frontier);
        if (hc.err) return set_error(BBS_ECORRUPT, "localize: device error flags 0x%x", hc.err);
        if (hc.match_changed) t_match = ms_since(t0);
        if (hc.done) break;
        ++iters;
        if (iters > (int64_t)1 << 24) return set_error(BBS_ETIMEOUT, "localize: iteration limit");
        res->parents_branched += hc.n_parents;
        res->nodes_scored += hc.popped_kids;
        res->gathers += (hc.popped_kids / 8) * k;   // one brick probe per point per rotational child
        gather_kernel<<<(int)std::min<int64_t>(std::max<int64_t>(hc.n_pop, 1), 8192), CH, 0, st>>>(f);
        res->launches++;
        BBS_CUDA_TRY(cudaGetLastError());
        for (int64_t p0 = 0; p0 < hc.n_parents; p0 += pslice) {
            BranchArgs a2 = ba;
            a2.parents = f.parents + p0;
            a2.items_per = rmax;
            a2.n_items = std::min(pslice, hc.n_parents - p0) * rmax;
            BBS_TRY(score(MODE_SEARCH, a2, 0));
            BBS_TRY(insert());
        }
        // frontier size after this iteration's insertions
        int64_t sz = 0;
        BBS_CUDA_TRY(cudaMemcpyAsync(&sz, &f.ctl->size, sizeof(sz), cudaMemcpyDeviceToHost, st));
        res->d2h_bytes += (int64_t)sizeof(sz);
        BBS_CUDA_TRY(cudaStreamSynchronize(st));
        res->peak_frontier = std::max(res->peak_frontier, sz);
    }
    int herr = 0;
    BBS_CUDA_TRY(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    res->d2h_bytes += (int64_t)sizeof(int);
    BBS_CUDA_TRY(cudaStreamSynchronize(st));
    if (herr) return set_error(BBS_ECORRUPT, "localize: survivor staging overflow (0x%x)", herr);
    const double t_end = ms_since(t0);
    for (size_t i = 0; i + 1 < evs.size(); i += 2) {
        float ms = 0.0f;
        BBS_CUDA_TRY(cudaEventElapsedTime(&ms, evs[i], evs[i + 1]));
        res->score_ms += ms;
    }
    res->iterations = iters;
    res->probes = res->nodes_scored * k;
    res->best_score = hc.best;
    res->phase_ms[2] = (t_match >= 0 ? t_match : t_end) - t_loop;
    res->phase_ms[3] = t_match >= 0 ? t_end - t_match : 0.0;
    if (hc.found) {
        const NodeRec& n = hc.match;
        const uint32_t rot = rl_rot(n.rl);
        const int64_t ng = g.N[0][2], nbb = g.N[0][1];
        res->found = 1;
        res->node[0] = n.cx;
        res->node[1] = n.cy;
        res->node[2] = n.cz;
        res->node[3] = (int32_t)(rot / (ng * nbb));
        res->node[4] = (int32_t)((rot / ng) % nbb);
        res->node[5] = (int32_t)(rot % ng);
        res->node[6] = 0;
        for (int i = 0; i < 3; ++i) res->pose[i] = (double)res->node[i] * g.r;
        for (int i = 0; i < 3; ++i) res->pose[3 + i] = grid_angle(g, 0, i, res->node[3 + i]);
        res->status = BBS_OK;
        res->ms_to_optimum = t_match;
    } else {
        res->status = BBS_NOT_FOUND;
        res->ms_to_optimum = t_end;
    }
    res->ms_total = ms_since(t0);
    res->phase_ms[4] = res->ms_total - t_end;
    return res->status;
}

}  // namespace bbs
