// capi.cu -- the extern "C" entry points of libbbs (declared in include/bbs.h).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "branch.cuh"
#include "engine.cuh"

namespace bbs {

static thread_local char g_err[512];

int set_error(int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

void clear_error() { g_err[0] = 0; }

int maps_build(const float* xyz, int64_t n, int is_device, float r, int levels, uint32_t flags, cudaStream_t st,
               bbs_maps** out);
int maps_keys(const bbs_maps* m, int level, int32_t* out, int64_t cap, int64_t* n);
int maps_set_load(double load);
int maps_set_layout(int layout);
int search_run(const bbs_maps* m, const float* xyz, int64_t k, int is_device, const bbs_ranges* rg,
               const bbs_opts* opts, cudaStream_t st, bbs_result* res);
int search_run_many(const bbs_maps* m, int n, const float* const* scans, const int64_t* ks, int is_device,
                    const bbs_ranges* rg, const bbs_opts* opts, cudaStream_t st, bbs_result* res);

// Keep memory freed by cudaFreeAsync in the device's default pool instead of
// returning it to the driver at every synchronization: the search allocates
// its frontier per call, and re-mapping hundreds of MB each time would cost
// milliseconds.  Set once per device for this process.
static void keep_pool_memory(int dev)
{
    static std::mutex mu;
    static bool done[64] = {};
    if (dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}

// make the maps' device current for the duration of a call
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
        keep_pool_memory(dev);
    }
    ~DeviceGuard()
    {
        if (changed) cudaSetDevice(prev);
    }
};

static cudaStream_t stream_of(const bbs_opts* o) { return o ? (cudaStream_t)o->cuda_stream : (cudaStream_t)0; }

static int copy_in(const void* src, size_t bytes, int is_device, void** dst, cudaStream_t st, bool* owned)
{
    *owned = false;
    if (is_device) {
        *dst = const_cast<void*>(src);
        return BBS_OK;
    }
    BBS_CUDA_TRY(cudaMallocAsync(dst, bytes > 0 ? bytes : 1, st));
    *owned = true;
    if (bytes) BBS_CUDA_TRY(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st));
    return BBS_OK;
}

}  // namespace bbs

using namespace bbs;

extern "C" {

int bbs_build_maps(const float* xyz, int64_t n, int is_device, float r, int levels, uint32_t flags, void* cuda_stream,
                   bbs_maps** out)
{
    clear_error();
    if (!out) return set_error(BBS_EINVAL, "build_maps: out is NULL");
    int dev = 0;
    cudaGetDevice(&dev);
    keep_pool_memory(dev);
    return maps_build(xyz, n, is_device, r, levels, flags, (cudaStream_t)cuda_stream, out);
}

void bbs_free_maps(bbs_maps* m)
{
    if (!m) return;
    DeviceGuard g(m->device);
    for (int l = 0; l < BBS_MAX_LEVELS; ++l)
        if (m->lv[l].slots) cudaFree(m->lv[l].slots);
    delete m;
}

int bbs_maps_bbox(const bbs_maps* m, double lo[3], double hi[3])
{
    clear_error();
    if (!m || !lo || !hi) return set_error(BBS_EINVAL, "maps_bbox: NULL argument");
    for (int i = 0; i < 3; ++i) {
        lo[i] = m->lo[i];
        hi[i] = m->hi[i];
    }
    return BBS_OK;
}

int bbs_maps_info(const bbs_maps* m, int level, int64_t* n_voxels, int64_t* n_buckets, int64_t* table_size,
                  int32_t* max_probe, double* collision_rate)
{
    clear_error();
    if (!m || level < 0 || level >= m->levels) return set_error(BBS_EINVAL, "maps_info: bad handle or level");
    const LevelTable& t = m->lv[level];
    if (n_voxels) *n_voxels = t.n_voxels;
    if (n_buckets) *n_buckets = t.n_bricks;
    if (table_size) *table_size = t.n_slots;
    if (max_probe) *max_probe = t.maxp;
    if (collision_rate) *collision_rate = t.n_bricks ? (double)t.displaced / (double)t.n_bricks : 0.0;
    return BBS_OK;
}

int bbs_gicp_target_build(const float* xyz, int64_t n, int is_device, float r, void* cuda_stream,
                          bbs_gicp_target** out)
{
    clear_error();
    if (!out) return set_error(BBS_EINVAL, "gicp_target: NULL out");
    *out = nullptr;
    int dev = 0;
    cudaGetDevice(&dev);
    DeviceGuard g(dev);
    return gicp_target_build(xyz, n, is_device, r, (cudaStream_t)cuda_stream, out);
}

void bbs_gicp_target_free(bbs_gicp_target* t)
{
    if (!t) return;
    DeviceGuard g(gicp_target_device(t));
    gicp_target_free(t);
}

int bbs_gicp_target_info(const bbs_gicp_target* t, int64_t* n_voxels, int64_t* table_size, int32_t* max_probe)
{
    clear_error();
    if (!t) return set_error(BBS_EINVAL, "gicp_target_info: NULL target");
    return gicp_target_info(t, n_voxels, table_size, max_probe);
}

int bbs_gicp(const bbs_gicp_target* t, const float* scan_xyz, int64_t k, int is_device, const double R0[9],
             const double t0[3], const bbs_gicp_opts* opts, bbs_gicp_result* out)
{
    clear_error();
    if (!t || !out || !R0 || !t0) return set_error(BBS_EINVAL, "gicp: NULL argument");
    DeviceGuard g(gicp_target_device(t));
    return gicp_run(t, scan_xyz, k, is_device, R0, t0, opts, out);
}

int bbs_gicp_linearize(const bbs_gicp_target* t, const float* scan_xyz, int64_t k, int is_device, const double R[9],
                       const double tr[3], const bbs_gicp_opts* opts, double H[36], double g[6], double* cost,
                       int64_t* n, int32_t* voxels, uint8_t* found)
{
    clear_error();
    if (!t || !R || !tr || !H || !g || !cost || !n) return set_error(BBS_EINVAL, "gicp_linearize: NULL argument");
    DeviceGuard dg(gicp_target_device(t));
    return gicp_linearize(t, scan_xyz, k, is_device, R, tr, opts, H, g, cost, n, voxels, found);
}

int bbs_maps_layout(const bbs_maps* m, int level, int32_t* layout)
{
    clear_error();
    if (!m || !layout || level < 0 || level >= m->levels) return set_error(BBS_EINVAL, "maps_layout: bad argument");
    *layout = m->lv[level].layout;
    return BBS_OK;
}

int bbs_maps_device(const bbs_maps* m, int32_t* device)
{
    clear_error();
    if (!m || !device) return set_error(BBS_EINVAL, "maps_device: NULL argument");
    *device = m->device;
    return BBS_OK;
}

// R = Rz(yaw) Ry(pitch) Rx(roll) of a result pose (Sec. III-A), the same
// composition as the pose grid's rotations, FP64, row-major; t = (x, y, z)
int bbs_pose_matrix(const double pose[6], double R[9], double t[3])
{
    clear_error();
    if (!pose || !R || !t) return set_error(BBS_EINVAL, "pose_matrix: NULL argument");
    for (int i = 0; i < 6; ++i)
        if (!std::isfinite(pose[i])) return set_error(BBS_EINVAL, "pose_matrix: non-finite pose");
    const double ca = std::cos(pose[3]), sa = std::sin(pose[3]);
    const double cb = std::cos(pose[4]), sb = std::sin(pose[4]);
    const double cg = std::cos(pose[5]), sg = std::sin(pose[5]);
    R[0] = cg * cb;
    R[1] = cg * sb * sa - sg * ca;
    R[2] = cg * sb * ca + sg * sa;
    R[3] = sg * cb;
    R[4] = sg * sb * sa + cg * ca;
    R[5] = sg * sb * ca - cg * sa;
    R[6] = -sb;
    R[7] = cb * sa;
    R[8] = cb * ca;
    for (int i = 0; i < 3; ++i) t[i] = pose[i];
    return BBS_OK;
}

int bbs_maps_keys(const bbs_maps* m, int level, int32_t* out, int64_t cap, int64_t* n)
{
    clear_error();
    if (!m || !n) return set_error(BBS_EINVAL, "maps_keys: NULL argument");
    DeviceGuard g(m->device);
    return maps_keys(m, level, out, cap, n);
}

int bbs_pose_grid(const bbs_maps* m, const float* scan_xyz, int64_t k, int is_device, const bbs_ranges* ranges,
                  const bbs_opts* opts, int level, int64_t* dims, float* A_out, int64_t cap, int64_t* n_rot)
{
    clear_error();
    if (!m || !dims || !n_rot) return set_error(BBS_EINVAL, "pose_grid: NULL argument");
    DeviceGuard dg(m->device);
    cudaStream_t st = stream_of(opts);
    ScanState S;
    BBS_TRY(scan_prepare(m, scan_xyz, k, is_device, ranges, opts, st, &S));
    const HostGrid& g = S.grid;
    int rc = BBS_OK;
    if (level < 0 || level >= g.levels) rc = set_error(BBS_EINVAL, "pose_grid: level %d", level);
    if (rc == BBS_OK) {
        for (int i = 0; i < 3; ++i) {
            dims[i] = g.N[level][i];
            dims[3 + i] = g.a[level][i];
            dims[6 + i] = g.wmin[i];
            dims[9 + i] = g.wmax[i];
        }
        *n_rot = g.nrot[level];
        if (A_out) {
            if (cap < g.nrot[level]) {
                rc = set_error(BBS_EINVAL, "pose_grid: capacity %lld < %lld", (long long)cap, (long long)g.nrot[level]);
            } else {
                std::vector<float4> h((size_t)(3 * g.nrot[level]));
                float4* d_rows = nullptr;
                cudaError_t e = cudaMallocAsync((void**)&d_rows, sizeof(float4) * h.size(), st);
                if (e == cudaSuccess) e = launch_level_rows(S, level, d_rows, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(h.data(), d_rows, sizeof(float4) * h.size(), cudaMemcpyDeviceToHost, st);
                if (d_rows) cudaFreeAsync(d_rows, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e != cudaSuccess) rc = set_error(BBS_ECUDA, "pose_grid: %s", cudaGetErrorString(e));
                for (int64_t t = 0; rc == BBS_OK && t < g.nrot[level]; ++t)
                    for (int row = 0; row < 3; ++row) {
                        const float4 v = h[(size_t)(3 * t + row)];
                        A_out[9 * t + 3 * row + 0] = v.x;
                        A_out[9 * t + 3 * row + 1] = v.y;
                        A_out[9 * t + 3 * row + 2] = v.z;
                    }
            }
        }
    }
    scan_release(&S, st);
    cudaStreamSynchronize(st);
    return rc;
}

int bbs_score_batch(const bbs_maps* m, const float* scan_xyz, int64_t k, int is_device, const bbs_ranges* ranges,
                    const bbs_opts* opts, const int32_t* nodes, int64_t n, int32_t* scores)
{
    clear_error();
    if (!m || n < 0 || (n > 0 && (!nodes || !scores))) return set_error(BBS_EINVAL, "score_batch: bad arguments");
    if (n == 0) return BBS_OK;
    DeviceGuard dg(m->device);
    cudaStream_t st = stream_of(opts);
    ScanState S;
    BBS_TRY(scan_prepare(m, scan_xyz, k, is_device, ranges, opts, st, &S));
    int rc = BBS_OK;
    void* d_nodes = nullptr;
    bool own_nodes = false;
    int32_t* d_scores = scores;
    int* d_err = nullptr;
    rc = copy_in(nodes, sizeof(int32_t) * 7 * (size_t)n, is_device, &d_nodes, st, &own_nodes);
    if (rc == BBS_OK && !is_device && cudaMallocAsync((void**)&d_scores, sizeof(int32_t) * (size_t)n, st) != cudaSuccess)
        rc = set_error(BBS_ENOMEM, "score_batch: scores buffer");
    if (rc == BBS_OK && cudaMallocAsync((void**)&d_err, sizeof(int), st) != cudaSuccess)
        rc = set_error(BBS_ENOMEM, "score_batch: status word");
    if (rc == BBS_OK && cudaMemsetAsync(d_err, 0, sizeof(int), st) != cudaSuccess) rc = set_error(BBS_ECUDA, "memset");
    if (rc == BBS_OK) rc = launch_score_nodes(m, S, (const int32_t*)d_nodes, n, d_scores, d_err, st);
    int herr = 0;
    if (rc == BBS_OK) {
        cudaError_t e = cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && !is_device)
            e = cudaMemcpyAsync(scores, d_scores, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = set_error(BBS_ECUDA, "score_batch: %s", cudaGetErrorString(e));
        else if (herr) rc = set_error(BBS_EINVAL, "score_batch: a node lies outside the pose grid");
    }
    if (own_nodes) cudaFreeAsync(d_nodes, st);
    if (!is_device && d_scores && d_scores != scores) cudaFreeAsync(d_scores, st);
    if (d_err) cudaFreeAsync(d_err, st);
    scan_release(&S, st);
    cudaStreamSynchronize(st);
    return rc;
}

int bbs_score_children(const bbs_maps* m, const float* scan_xyz, int64_t k, int is_device, const bbs_ranges* ranges,
                       const bbs_opts* opts, const int32_t* parents, int64_t n, int32_t* child_nodes,
                       int32_t* child_scores, int64_t cap, int64_t* n_children)
{
    clear_error();
    if (!m || n < 0 || !n_children || (n > 0 && !parents)) return set_error(BBS_EINVAL, "score_children: bad arguments");
    DeviceGuard dg(m->device);
    cudaStream_t st = stream_of(opts);
    std::vector<int32_t> hp((size_t)(7 * n));
    if (n > 0) {
        if (is_device) {
            BBS_CUDA_TRY(cudaMemcpyAsync(hp.data(), parents, sizeof(int32_t) * hp.size(), cudaMemcpyDeviceToHost, st));
            BBS_CUDA_TRY(cudaStreamSynchronize(st));
        } else {
            std::memcpy(hp.data(), parents, sizeof(int32_t) * hp.size());
        }
    }
    ScanState S;
    BBS_TRY(scan_prepare(m, scan_xyz, k, is_device, ranges, opts, st, &S));
    struct Rel {
        ScanState* s;
        cudaStream_t st;
        ~Rel()
        {
            scan_release(s, st);
            cudaStreamSynchronize(st);
        }
    } rel{&S, st};
    const HostGrid& g = S.grid;
    const DevGrid dgr = dev_grid(g);
    std::vector<NodeRec> recs((size_t)n);
    std::vector<int32_t> cnt((size_t)n), lo((size_t)(3 * n)), ext((size_t)(3 * n));
    int64_t total = 0;
    for (int64_t p = 0; p < n; ++p) {
        const int32_t* c = &hp[(size_t)(7 * p)];
        const int l = c[6];
        bool ok = l >= 0 && l < g.levels;
        for (int i = 0; ok && i < 3; ++i) {
            ok = c[3 + i] >= 0 && c[3 + i] < g.N[l][i];
            const int64_t t = (int64_t)c[i] * ((int64_t)1 << l);
            ok = ok && t >= -(int64_t)KEY_LIMIT && t <= (int64_t)KEY_LIMIT;
        }
        if (!ok) return set_error(BBS_EINVAL, "score_children: parent %lld lies outside the pose grid", (long long)p);
        const uint32_t rot = (uint32_t)(((int64_t)c[3] * g.N[l][1] + c[4]) * g.N[l][2] + c[5]);
        recs[(size_t)p] = NodeRec{c[0], c[1], c[2], rl_pack(rot, l)};
        const int32_t count = rot_children(dgr, l, rot, &lo[(size_t)(3 * p)], &ext[(size_t)(3 * p)]);
        cnt[(size_t)p] = count;
        total += 8 * (int64_t)count;
    }
    *n_children = total;
    if (total > cap) return set_error(BBS_EINVAL, "score_children: capacity %lld < %lld children", (long long)cap, (long long)total);
    if (total == 0) return BBS_OK;
    if (!child_nodes || !child_scores) return set_error(BBS_EINVAL, "score_children: NULL output buffer");
    // the tasks (rotational children) in parent order, child order ja, jb, jg
    const int64_t ntask = total / 8;
    std::vector<TaskRec> tk((size_t)ntask);
    std::vector<int64_t> tk_parent((size_t)ntask);
    {
        int64_t u = 0;
        for (int64_t p = 0; p < n; ++p) {
            const int l = recs[(size_t)p].rl & 31;
            const int32_t* plo = &lo[(size_t)(3 * p)];
            const int32_t* pex = &ext[(size_t)(3 * p)];
            for (int32_t ja = 0; ja < pex[0]; ++ja)
                for (int32_t jb = 0; jb < pex[1]; ++jb)
                    for (int32_t jg = 0; jg < pex[2]; ++jg) {
                        const uint32_t crot =
                            (uint32_t)(((int64_t)(plo[0] + ja) * g.N[l - 1][1] + (plo[1] + jb)) * g.N[l - 1][2] + (plo[2] + jg));
                        TaskRec r;
                        std::memset(&r, 0, sizeof(r));
                        r.tx = 2 * recs[(size_t)p].cx;
                        r.ty = 2 * recs[(size_t)p].cy;
                        r.tz = 2 * recs[(size_t)p].cz;
                        r.rl = rl_pack(crot, l - 1);
                        tk_parent[(size_t)u] = p;
                        tk[(size_t)u++] = r;   // the scoring kernel forms the rows
                    }
        }
    }
    // one search slot for the fused kernel (no frontier: dense scores only)
    SearchDev sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.scan = S.scan;
    sd.cbox = S.cbox;
    sd.rot = S.rot;
    sd.cs = S.cs;
    sd.K = (int32_t)k;
    sd.lmax = g.levels - 1;
    sd.nblk = (int32_t)((k + PBLK - 1) / PBLK);
    sd.grid = dgr;
    for (int l = 0; l < MAX_LEVELS; ++l) sd.maps[l] = l < m->levels ? level_view(m, l) : LevelView{};
    SearchDev* d_sd = nullptr;
    TaskRec* d_tk = nullptr;
    int32_t* d_dense = nullptr;
    Plan* d_plan = nullptr;
    struct Bufs {   // freed on every return below, in stream order
        void** p[4];
        cudaStream_t st;
        ~Bufs()
        {
            for (void** q : p)
                if (*q) cudaFreeAsync(*q, st);
        }
    } bufs{{(void**)&d_sd, (void**)&d_tk, (void**)&d_dense, (void**)&d_plan}, st};
    BBS_CUDA_TRY(cudaMallocAsync((void**)&d_sd, sizeof(SearchDev), st));
    BBS_CUDA_TRY(cudaMallocAsync((void**)&d_tk, sizeof(TaskRec) * (size_t)ntask, st));
    BBS_CUDA_TRY(cudaMallocAsync((void**)&d_dense, sizeof(int32_t) * (size_t)total, st));
    BBS_CUDA_TRY(cudaMallocAsync((void**)&d_plan, sizeof(Plan), st));
    Plan P;
    std::memset(&P, 0, sizeof(P));
    P.mode = MODE_SEARCH;
    P.status = PLAN_OK;
    P.nseg = 1;
    P.n_tasks = ntask;
    P.n_slices = ntask * sd.nblk;
    {
        const Tuning tn = current_tuning();
        P.static_pm = tn.static_pm;
        P.grab_min = tn.grab_min;
    }
    P.seg[0].first_task = 0;
    P.seg[0].n_tasks = ntask;
    P.seg[0].first_slice = 0;
    P.seg[0].sid = 0;
    P.seg[0].nblk = sd.nblk;
    BBS_CUDA_TRY(cudaMemcpyAsync(d_sd, &sd, sizeof(sd), cudaMemcpyHostToDevice, st));
    BBS_CUDA_TRY(cudaMemcpyAsync(d_tk, tk.data(), sizeof(TaskRec) * tk.size(), cudaMemcpyHostToDevice, st));
    BBS_CUDA_TRY(cudaMemcpyAsync(d_plan, &P, offsetof(Plan, seg) + sizeof(Seg), cudaMemcpyHostToDevice, st));
    BBS_CUDA_TRY(cudaMemsetAsync(d_dense, 0, sizeof(int32_t) * (size_t)total, st));
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int rc = BBS_OK;
    cudaError_t e = launch_branch(MODE_SEARCH, d_plan, d_sd, d_tk, d_dense,
                                  (int)std::min<int64_t>(P.n_slices, (int64_t)nsm * BRANCH_CTAS_PER_SM), st,
                                  maps_all_bytes(m));
    std::vector<int32_t> dense((size_t)total);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dense.data(), d_dense, sizeof(int32_t) * dense.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host copies of P and the tasks outlive their transfers
    if (e != cudaSuccess) rc = set_error(BBS_ECUDA, "score_children: %s", cudaGetErrorString(e));
    if (rc != BBS_OK) return rc;
    std::vector<int32_t> on((size_t)(7 * total)), os((size_t)total);
    int64_t o = 0;
    for (int64_t u = 0; u < ntask; ++u) {
        const TaskRec& r = tk[(size_t)u];
        const int32_t* c = &hp[(size_t)(7 * tk_parent[(size_t)u])];
        const int l = c[6];
        const uint32_t crot = rl_rot(r.rl);
        const int32_t ng = g.N[l - 1][2], nb = g.N[l - 1][1];
        for (int t = 0; t < 8; ++t) {
            int32_t* d = &on[(size_t)(7 * o)];
            d[0] = 2 * c[0] + (t >> 2);
            d[1] = 2 * c[1] + ((t >> 1) & 1);
            d[2] = 2 * c[2] + (t & 1);
            d[3] = (int32_t)(crot / (uint32_t)(ng * nb));
            d[4] = (int32_t)((crot / (uint32_t)ng) % (uint32_t)nb);
            d[5] = (int32_t)(crot % (uint32_t)ng);
            d[6] = l - 1;
            os[(size_t)o] = dense[(size_t)(8 * u + t)];
            ++o;
        }
    }
    if (is_device) {
        BBS_CUDA_TRY(cudaMemcpyAsync(child_nodes, on.data(), sizeof(int32_t) * on.size(), cudaMemcpyHostToDevice, st));
        BBS_CUDA_TRY(cudaMemcpyAsync(child_scores, os.data(), sizeof(int32_t) * os.size(), cudaMemcpyHostToDevice, st));
        BBS_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        std::memcpy(child_nodes, on.data(), sizeof(int32_t) * on.size());
        std::memcpy(child_scores, os.data(), sizeof(int32_t) * os.size());
    }
    return BBS_OK;
}

int bbs_localize_hostqueue(const bbs_maps* m, const float* scan_xyz, int64_t k, int is_device,
                           const bbs_ranges* ranges, const bbs_opts* opts, bbs_result* out)
{
    clear_error();
    if (!m || !out) return set_error(BBS_EINVAL, "localize_hostqueue: NULL argument");
    DeviceGuard g(m->device);
    return hostqueue_run(m, scan_xyz, k, is_device, ranges, opts, stream_of(opts), out);
}

int bbs_localize(const bbs_maps* m, const float* scan_xyz, int64_t k, int is_device, const bbs_ranges* ranges,
                 const bbs_opts* opts, bbs_result* out)
{
    clear_error();
    if (!m || !out) return set_error(BBS_EINVAL, "localize: NULL argument");
    DeviceGuard dg(m->device);
    cudaStream_t st = stream_of(opts);
    int rc = search_run(m, scan_xyz, k, is_device, ranges, opts, st, out);
    out->status = rc;
    cudaStreamSynchronize(st);
    return rc;
}

int bbs_localize_many(const bbs_maps* m, int n, const float* const* scans, const int64_t* ks, int is_device,
                      const bbs_ranges* ranges, const bbs_opts* opts, bbs_result* out)
{
    clear_error();
    if (!m || n < 0 || (n > 0 && (!scans || !ks || !out))) return set_error(BBS_EINVAL, "localize_many: bad arguments");
    if (n > 4096) return set_error(BBS_EINVAL, "localize_many: more than 4096 scans");
    if (n == 0) return BBS_OK;
    DeviceGuard dg(m->device);
    cudaStream_t st = stream_of(opts);
    int rc = search_run_many(m, n, scans, ks, is_device, ranges, opts, st, out);
    cudaStreamSynchronize(st);
    if (rc < 0)
        for (int i = 0; i < n; ++i) out[i].status = rc;
    return rc;
}

const char* bbs_last_error(void) { return g_err; }

const char* bbs_version(void) { return "bbs-gb300 0.1 sm_103a"; }

int bbs_set_load_factor(double load)
{
    clear_error();
    return maps_set_load(load);
}

int bbs_set_probe_layout(int layout)
{
    clear_error();
    return maps_set_layout(layout);
}

int bbs_exact_dilation(const bbs_maps* m, const float* scan_xyz, int64_t k, int is_device, const bbs_ranges* ranges,
                       const bbs_opts* opts, int32_t* e)
{
    clear_error();
    if (!m || !e) return set_error(BBS_EINVAL, "exact_dilation: NULL argument");
    DeviceGuard g(m->device);
    cudaStream_t st = opts ? (cudaStream_t)opts->cuda_stream : nullptr;
    ScanState S;
    BBS_TRY(scan_prepare(m, scan_xyz, k, is_device, ranges, opts, st, &S));
    *e = exact_dilation_needed(S.grid, S.norm_max);
    scan_release(&S, st);
    BBS_CUDA_TRY(cudaStreamSynchronize(st));
    return BBS_OK;
}

int bbs_set_tuning(const bbs_tuning* t)
{
    clear_error();
    return set_tuning(t);
}

int bbs_launch_log(int64_t* units, double* ms, int64_t cap, int64_t* n)
{
    clear_error();
    if (!n) return set_error(BBS_EINVAL, "launch_log: n is NULL");
    const LaunchLog& L = launch_log();
    *n = (int64_t)L.ms.size();
    if (cap < *n || (*n > 0 && (!units || !ms))) return *n == 0 ? BBS_OK : set_error(BBS_EINVAL, "launch_log: capacity %lld < %lld", (long long)cap, (long long)*n);
    for (size_t i = 0; i < L.ms.size(); ++i) {
        units[i] = L.units[i];
        ms[i] = L.ms[i];
    }
    return BBS_OK;
}

int bbs_get_tuning(bbs_tuning* t)
{
    clear_error();
    if (!t) return set_error(BBS_EINVAL, "get_tuning: NULL");
    const Tuning v = current_tuning();
    std::memset(t, 0, sizeof(*t));
    t->launch_tasks = v.launch_tasks;
    t->static_pm = v.static_pm;
    t->grab_min = v.grab_min;
    t->ctas_per_sm = v.ctas_per_sm;
    t->frontier_log2 = v.frontier_log2;
    return BBS_OK;
}

}  // extern "C"
