// hostqueue.cu -- the search with its frontier on the host, Algorithm 2's own
// shape (Sec. III-E): a priority structure in host memory, and per batch the
// popped parents' rotational children go to the GPU as task records (H2D),
// are scored there by the same kernels as the device-resident engine, and
// their 8 translational children's scores come back (D2H) for the host to
// keep those above best.  The canonical iteration is the engine's (select:
// whole score buckets from the top until the popped parents have b
// children; a bucket at or below best clears F; a bucket holding a leaf sets
// best and the lexmin leaf and clears F), so the results are the engine's.
// It exists to measure what keeping the frontier on the device buys.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <vector>

#include "branch.cuh"

namespace bbs {

namespace {

double ms_now()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int64_t floor_half(int64_t x) { return x >= 0 ? x / 2 : -((-x + 1) / 2); }

struct HostBucket {
    std::vector<NodeRec> nodes;
    int64_t kids = 0;
    int64_t leaves = 0;
};

// device buffers of one host-queue search, grown as batches need
struct DevBufs {
    cudaStream_t st;
    TaskRec* tasks = nullptr;
    int32_t* dense = nullptr;
    Plan* plan = nullptr;
    SearchDev* sd = nullptr;
    int64_t cap = 0;
    ~DevBufs()
    {
        if (tasks) cudaFreeAsync(tasks, st);
        if (dense) cudaFreeAsync(dense, st);
        if (plan) cudaFreeAsync(plan, st);
        if (sd) cudaFreeAsync(sd, st);
        cudaStreamSynchronize(st);
    }
    int reserve(int64_t n)
    {
        if (n <= cap) return BBS_OK;
        int64_t c = std::max<int64_t>(n, 2 * cap);
        if (tasks) cudaFreeAsync(tasks, st);
        if (dense) cudaFreeAsync(dense, st);
        tasks = nullptr;
        dense = nullptr;
        BBS_CUDA_TRY(cudaMallocAsync((void**)&tasks, sizeof(TaskRec) * (size_t)c, st));
        BBS_CUDA_TRY(cudaMallocAsync((void**)&dense, sizeof(int32_t) * 8 * (size_t)c, st));
        cap = c;
        return BBS_OK;
    }
};

}  // namespace

int hostqueue_run(const bbs_maps* m, const float* xyz, int64_t k, int is_device, const bbs_ranges* rg,
                  const bbs_opts* opts, cudaStream_t st, bbs_result* res)
{
    std::memset(res, 0, sizeof(*res));
    const double t0 = ms_now();
    res->num_points = (int32_t)k;
    const double frac = (opts && opts->score_frac > 0.0) ? opts->score_frac : 0.95;
    const int64_t batch = (opts && opts->batch > 0) ? opts->batch : 10000;
    const uint32_t flags = opts ? opts->flags : 0u;
    if (!(frac > 0.0 && frac <= 1.0)) return res->status = set_error(BBS_EINVAL, "localize: score_frac %g outside (0, 1]", frac);
    if (flags & BBS_PRUNE_GE) return res->status = set_error(BBS_EINVAL, "localize: BBS_PRUNE_GE is not supported");
    if (k > (1 << 24) - 2) return res->status = set_error(BBS_EINVAL, "localize: more than 2^24 - 2 scan points");
    ScanState S;
    {
        const int rc = scan_prepare(m, xyz, k, is_device, rg, opts, st, &S);
        if (rc < 0) return res->status = rc;
    }
    struct Rel {
        ScanState* s;
        cudaStream_t st;
        ~Rel() { scan_release(s, st); }
    } rel{&S, st};
    res->h2d_bytes += S.h2d;
    res->d2h_bytes += S.d2h;
    const HostGrid& g = S.grid;
    if ((m->flags & BBS_EXACT_BOUND) && k > 0) {
        const int need = exact_dilation_needed(g, S.norm_max);
        if (need < 0 || need > (int)((m->flags >> 12) & 15u))
            return res->status = set_error(BBS_EINVAL, "localize: exact-bound maps widened too little for this scan");
    }
    const int32_t thr = (int32_t)std::ceil(frac * (double)k);
    res->phase_ms[0] = ms_now() - t0;
    if (k == 0) {
        res->best_score = thr - 1;
        res->ms_total = ms_now() - t0;
        return res->status = BBS_NOT_FOUND;
    }
    const DevGrid dg = dev_grid(g);
    const int lmax = g.levels - 1;
    SearchDev sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.scan = S.scan;
    sd.cbox = S.cbox;
    sd.rot = S.rot;
    sd.cs = S.cs;
    sd.K = (int32_t)k;
    sd.lmax = lmax;
    sd.nblk = (int32_t)((k + PBLK - 1) / PBLK);
    sd.grid = dg;
    for (int l = 0; l < MAX_LEVELS; ++l) sd.maps[l] = l < m->levels ? level_view(m, l) : LevelView{};
    DevBufs D;
    D.st = st;
    BBS_CUDA_TRY(cudaMallocAsync((void**)&D.plan, sizeof(Plan), st));
    BBS_CUDA_TRY(cudaMallocAsync((void**)&D.sd, sizeof(SearchDev), st));
    BBS_CUDA_TRY(cudaMemcpyAsync(D.sd, &sd, sizeof(sd), cudaMemcpyHostToDevice, st));
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const Tuning tn = current_tuning();

    // scores of the 8 translational children of every task, on the GPU
    std::vector<TaskRec> tk;
    std::vector<int32_t> dense;
    auto score_tasks = [&]() -> int {
        const int64_t n = (int64_t)tk.size();
        if (n == 0) return BBS_OK;
        BBS_TRY(D.reserve(n));
        Plan P;
        std::memset(&P, 0, sizeof(P));
        P.mode = MODE_SEARCH;
        P.status = PLAN_OK;
        P.nseg = 1;
        P.n_tasks = n;
        P.n_slices = n * sd.nblk;
        P.static_pm = tn.static_pm;
        P.grab_min = tn.grab_min;
        P.seg[0].n_tasks = n;
        P.seg[0].nblk = sd.nblk;
        BBS_CUDA_TRY(cudaMemcpyAsync(D.tasks, tk.data(), sizeof(TaskRec) * (size_t)n, cudaMemcpyHostToDevice, st));
        BBS_CUDA_TRY(cudaMemcpyAsync(D.plan, &P, offsetof(Plan, seg) + sizeof(Seg), cudaMemcpyHostToDevice, st));
        BBS_CUDA_TRY(cudaMemsetAsync(D.dense, 0, sizeof(int32_t) * 8 * (size_t)n, st));
        res->h2d_bytes += (int64_t)(sizeof(TaskRec) * (size_t)n + offsetof(Plan, seg) + sizeof(Seg));
        BBS_CUDA_TRY(launch_branch(MODE_SEARCH, D.plan, D.sd, D.tasks, D.dense,
                                   (int)std::min<int64_t>(P.n_slices, (int64_t)nsm * tn.ctas_per_sm), st,
                                   maps_all_bytes(m)));
        dense.resize((size_t)(8 * n));
        BBS_CUDA_TRY(cudaMemcpyAsync(dense.data(), D.dense, sizeof(int32_t) * dense.size(), cudaMemcpyDeviceToHost, st));
        BBS_CUDA_TRY(cudaStreamSynchronize(st));   // P, tk and dense are host memory of this call
        res->d2h_bytes += (int64_t)(sizeof(int32_t) * dense.size());
        res->score_launches += 1;
        return BBS_OK;
    };

    // best-first: one frontier of score buckets; depth-first: one per level
    const bool dfs = (flags & BBS_SEARCH_DFS) != 0;
    const int nfr = dfs ? g.levels : 1;
    std::vector<std::vector<HostBucket>> FL((size_t)nfr, std::vector<HostBucket>((size_t)k + 1));
    std::vector<int32_t> ltop((size_t)nfr, -1);
    std::vector<int64_t> lsize((size_t)nfr, 0);
    std::vector<HostBucket>& F = FL[0];
    int64_t size = 0, peak = 0;
    int32_t top = -1, best = thr - 1;
    bool found = false;
    NodeRec match{};
    auto insert = [&](const NodeRec& nd, int32_t score) {
        const int f = dfs ? rl_level(nd.rl) : 0;
        HostBucket& b = FL[(size_t)f][(size_t)score];
        b.nodes.push_back(nd);
        b.kids += node_children(dg, rl_level(nd.rl), rl_rot(nd.rl));
        b.leaves += rl_level(nd.rl) == 0 ? 1 : 0;
        top = std::max(top, score);
        ltop[(size_t)f] = std::max(ltop[(size_t)f], score);
        lsize[(size_t)f] += 1;
        ++size;
    };
    auto lex_before = [](const NodeRec& a, const NodeRec& b) {
        return lex_translation(a) < lex_translation(b) ||
               (lex_translation(a) == lex_translation(b) && rl_rot(a.rl) < rl_rot(b.rl));
    };

    // the initial set: every translation of the Eq. (3)-(5) window times every
    // rotation at l_max, as tasks of virtual parents (2 x their translation)
    {
        const HostGrid& hg = g;
        int64_t pmin[3], pext[3];
        for (int a = 0; a < 3; ++a) {
            pmin[a] = floor_half(hg.wmin[a]);
            pext[a] = floor_half(hg.wmax[a]) - pmin[a] + 1;
        }
        const int64_t R = hg.nrot[lmax];
        tk.clear();
        for (int64_t px = 0; px < pext[0]; ++px)
            for (int64_t py = 0; py < pext[1]; ++py)
                for (int64_t pz = 0; pz < pext[2]; ++pz)
                    for (int64_t r = 0; r < R; ++r) {
                        TaskRec t;
                        std::memset(&t, 0, sizeof(t));
                        t.tx = (int32_t)(2 * (pmin[0] + px));
                        t.ty = (int32_t)(2 * (pmin[1] + py));
                        t.tz = (int32_t)(2 * (pmin[2] + pz));
                        t.rl = rl_pack((uint32_t)r, lmax);
                        tk.push_back(t);
                    }
        BBS_TRY(score_tasks());
        int64_t n0 = 1;
        for (int a = 0; a < 3; ++a) n0 *= hg.wmax[a] - hg.wmin[a] + 1;
        res->nodes_scored = n0 * R;
        res->gathers += pext[0] * pext[1] * pext[2] * R * k;
        for (size_t u = 0; u < tk.size(); ++u)
            for (int j = 0; j < 8; ++j) {
                NodeRec nd{tk[u].tx + (j >> 2), tk[u].ty + ((j >> 1) & 1), tk[u].tz + (j & 1), tk[u].rl};
                if (nd.cx < hg.wmin[0] || nd.cx > hg.wmax[0] || nd.cy < hg.wmin[1] || nd.cy > hg.wmax[1] ||
                    nd.cz < hg.wmin[2] || nd.cz > hg.wmax[2])
                    continue;
                const int32_t sc = dense[8 * u + j];
                if (sc > best) insert(nd, sc);
            }
        res->phase_ms[1] = ms_now() - t0 - res->phase_ms[0];
    }

    // the popped parents' rotational children (Eq. (13)), scored in launches of
    // at most the tuning's task count; children above best join the frontier
    std::vector<NodeRec> parents;
    std::vector<int32_t> pscores;   // the score of each parent (the bucket it was popped from)
    std::vector<int32_t> tps;       // each task's parent score
    auto branch_parents = [&](int64_t pk) -> int {
        res->iterations += 1;
        res->parents_branched += (int64_t)parents.size();
        res->nodes_scored += pk;
        res->gathers += (pk / 8) * k;
        tk.clear();
        tps.clear();
        for (size_t pi = 0; pi < parents.size(); ++pi) {
            const NodeRec& nd = parents[pi];
            const int l = rl_level(nd.rl);
            int32_t lo[3], ext[3];
            if (rot_children(dg, l, rl_rot(nd.rl), lo, ext) == 0) continue;
            const int64_t nb = g.N[l - 1][1], ng = g.N[l - 1][2];
            for (int32_t ja = 0; ja < ext[0]; ++ja)
                for (int32_t jb = 0; jb < ext[1]; ++jb)
                    for (int32_t jg = 0; jg < ext[2]; ++jg) {
                        TaskRec t;
                        std::memset(&t, 0, sizeof(t));
                        t.tx = 2 * nd.cx;
                        t.ty = 2 * nd.cy;
                        t.tz = 2 * nd.cz;
                        t.rl = rl_pack((uint32_t)(((int64_t)(lo[0] + ja) * nb + (lo[1] + jb)) * ng + (lo[2] + jg)), l - 1);
                        tk.push_back(t);
                        tps.push_back(pscores[pi]);
                    }
        }
        std::vector<TaskRec> all;
        all.swap(tk);
        for (size_t u0 = 0; u0 < all.size(); u0 += (size_t)tn.launch_tasks) {
            const size_t u1 = std::min(all.size(), u0 + (size_t)tn.launch_tasks);
            tk.assign(all.begin() + (long)u0, all.begin() + (long)u1);
            res->children_scored += 8 * (int64_t)tk.size();
            BBS_TRY(score_tasks());
            for (size_t u = 0; u < tk.size(); ++u)
                for (int j = 0; j < 8; ++j) {
                    const int32_t sc = dense[8 * u + j];
                    const int32_t ps = tps[u0 + u];
                    if (sc > ps) {   // Sec. IV-A: the child beats its parent's bound
                        res->bound_violations += 1;
                        res->bound_excess += (double)(sc - ps) / (double)sc;
                    }
                    if (sc <= best) continue;
                    insert(NodeRec{tk[u].tx + (j >> 2), tk[u].ty + ((j >> 1) & 1), tk[u].tz + (j & 1), tk[u].rl}, sc);
                }
        }
        return BBS_OK;
    };
    const double t_search = ms_now();
    double t_match = -1.0;

    // the depth-first order: leaves first (the best sets best and the match,
    // and every node at or below it goes), then whole (level, score) buckets,
    // deepest level first, highest score first, until the children reach b
    while (dfs) {
        peak = std::max(peak, size);
        if (lsize[0] > 0) {
            int32_t s0 = ltop[0];
            while (s0 >= 0 && FL[0][(size_t)s0].nodes.empty()) --s0;
            const HostBucket& b = FL[0][(size_t)s0];
            match = b.nodes[0];
            for (const NodeRec& nd : b.nodes)
                if (lex_before(nd, match)) match = nd;
            best = s0;
            found = true;
            t_match = ms_now();
            for (int l = 0; l < nfr; ++l)
                for (int32_t t = 0; t <= best && t <= ltop[(size_t)l]; ++t) {
                    HostBucket& hb = FL[(size_t)l][(size_t)t];
                    lsize[(size_t)l] -= (int64_t)hb.nodes.size();
                    size -= (int64_t)hb.nodes.size();
                    hb = HostBucket();
                }
        }
        parents.clear();
        pscores.clear();
        int64_t pk = 0;
        for (int l = 1; l < nfr && pk < batch; ++l)
            for (int32_t t = ltop[(size_t)l]; t > best && pk < batch; --t) {
                HostBucket& hb = FL[(size_t)l][(size_t)t];
                if (hb.nodes.empty()) continue;
                pk += hb.kids;
                parents.insert(parents.end(), hb.nodes.begin(), hb.nodes.end());
                pscores.insert(pscores.end(), hb.nodes.size(), t);
                lsize[(size_t)l] -= (int64_t)hb.nodes.size();
                size -= (int64_t)hb.nodes.size();
                hb = HostBucket();
            }
        if (parents.empty()) break;
        BBS_TRY(branch_parents(pk));
    }

    // the canonical best-first iteration
    while (!dfs) {
        peak = std::max(peak, size);
        int32_t sstar = -1;
        int reason = size > 0 ? 4 : 0;
        int64_t cum = 0;
        for (int32_t s = top; s >= 0; --s) {
            const HostBucket& b = F[(size_t)s];
            if (b.nodes.empty()) continue;
            if (cum >= batch || s <= best || b.leaves > 0) {
                sstar = s;
                reason = cum >= batch ? 1 : (s <= best ? 2 : 3);
                break;
            }
            cum += b.kids;
        }
        const bool clear = reason == 2 || reason == 3;
        if (reason == 3) {   // the lexmin leaf of the stop bucket sets the match
            const HostBucket& b = F[(size_t)sstar];
            bool have = false;
            for (const NodeRec& nd : b.nodes) {
                if (rl_level(nd.rl) != 0) continue;
                if (!have || lex_translation(nd) < lex_translation(match) ||
                    (lex_translation(nd) == lex_translation(match) && rl_rot(nd.rl) < rl_rot(match.rl))) {
                    match = nd;
                    have = true;
                }
            }
            best = sstar;
            found = true;
            t_match = ms_now();
        }
        parents.clear();
        pscores.clear();
        int64_t pk = 0;
        for (int32_t s = top; s > sstar; --s) {
            HostBucket& b = F[(size_t)s];
            pk += b.kids;
            parents.insert(parents.end(), b.nodes.begin(), b.nodes.end());
            pscores.insert(pscores.end(), b.nodes.size(), s);
            b = HostBucket();
        }
        if (clear)
            for (int32_t s = std::min(sstar, top); s >= 0; --s) F[(size_t)s] = HostBucket();
        size = clear ? 0 : size - (int64_t)parents.size();
        top = reason == 1 ? sstar : -1;
        if (parents.empty()) break;
        BBS_TRY(branch_parents(pk));
    }
    const double t_end = ms_now();
    res->best_score = best;
    res->peak_frontier = peak;
    res->probes = res->nodes_scored * k;
    res->phase_ms[2] = (t_match >= 0 ? t_match : t_end) - t_search;
    res->phase_ms[3] = t_match >= 0 ? t_end - t_match : 0.0;
    res->ms_total = ms_now() - t0;
    res->ms_to_optimum = (t_match >= 0 ? t_match : t_end) - t0;
    if (!found) return res->status = BBS_NOT_FOUND;
    const uint32_t rot = rl_rot(match.rl);
    const int64_t ng = g.N[0][2], nb = g.N[0][1];
    res->found = 1;
    res->node[0] = match.cx;
    res->node[1] = match.cy;
    res->node[2] = match.cz;
    res->node[3] = (int32_t)(rot / (ng * nb));
    res->node[4] = (int32_t)((rot / ng) % nb);
    res->node[5] = (int32_t)(rot % ng);
    res->node[6] = 0;
    for (int a = 0; a < 3; ++a) res->pose[a] = (double)res->node[a] * g.r;
    for (int a = 0; a < 3; ++a) res->pose[3 + a] = grid_angle(g, 0, a, res->node[3 + a]);
    return res->status = BBS_OK;
}

}  // namespace bbs
