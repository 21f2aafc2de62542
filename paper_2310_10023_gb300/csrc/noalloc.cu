// noalloc.cu -- bbs_score_batch_noalloc: Eq. (11) scores of caller nodes
// without allocating anything.
//
// Some callers cannot allocate device memory while they run: real-time
// control loops that must not touch the allocator after start-up (allocation
// latency and fragmentation are unbounded), frameworks that own every byte of
// device memory through their own pool, and code that budgets memory up front.
// This entry point gives them the scores of bbs_score_batch with every buffer
// either supplied by the caller (scan, nodes, scores, all device memory) or
// taken from one file-scope scratch array in device memory:
//
//   [0, 256)                 status words (error flag, d_max, bad-input flag)
//   [256, 256 + 1 MiB)       (cos, sin) of every angle segment of every level
//   [SCAN_OFF, + 2 MiB)      the scan packed to float4
//
// so at most BBS_NOALLOC_MAX_POINTS scan points and BBS_NOALLOC_MAX_ANGLES
// angle segments (summed over levels and axes) per call.  Instead of the
// per-level rotation tables of the other entry points, each node's matrix
// A = fl32(R / r) is formed in the kernel from the segment cosines and sines
// with the same FP64 operations, so the scores are bit-identical.
//
// The array lives in every GPU that loads the library until the process
// exits.  Every call shares it and it keeps the last call's contents; the
// status words are cleared at the start of each call.  Calls that overlapped
// on the GPU would race on it; each call holds a process-wide mutex until its
// final stream synchronization, so calls from several host threads run one
// after the other.  Host code cannot use the array's name as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it; make that
// first call before any stream capture.  Only bad arguments and a scan above
// BBS_NOALLOC_MAX_POINTS are refused before GPU work; the angle-segment limit
// and bad coordinates are found after the scan has been packed into the
// array.  The call synchronizes its stream twice (the scan's d_max is read
// back before the pose grid is formed, and the status words at the end).
#include <cmath>
#include <cstring>
#include <mutex>

#include "bbs_internal.cuh"

namespace {
constexpr size_t NA_CTRL_BYTES = 256;
constexpr size_t NA_CS_OFF = NA_CTRL_BYTES;
constexpr size_t NA_CS_BYTES = (size_t)BBS_NOALLOC_MAX_ANGLES * 16;        // double2 entries
constexpr size_t NA_SCAN_OFF = NA_CS_OFF + NA_CS_BYTES + 256;
constexpr size_t NA_SCAN_BYTES = (size_t)BBS_NOALLOC_MAX_POINTS * 16;      // float4 points
constexpr size_t NA_BYTES = NA_SCAN_OFF + NA_SCAN_BYTES + 3840;             // 3 MiB + 4 KiB
}  // namespace

// the scratch of bbs_score_batch_noalloc (layout above); a host-side stand-in
// in host code, its device address comes from cudaGetSymbolAddress
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace bbs {

namespace {

struct NaCtrl {
    int err;
    int bad;
    unsigned long long dmax_bits;
};

struct NaArgs {
    LevelView maps[MAX_LEVELS];
    DevGrid grid;                    // its cs_off: first (cos, sin) entry of each level and axis
    const double2* cs;
    const float4* scan;
    int64_t k;
    const int32_t* nodes;
    int64_t n;
    int32_t* scores;
    NaCtrl* ctrl;
};

__global__ void na_pack_kernel(const float* __restrict__ xyz, int64_t k, float4* __restrict__ out, double bound,
                               NaCtrl* ctrl)
{
    double m = 0.0;
    int b = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        out[i] = make_float4(x, y, z, 0.0f);
        const double dx = x, dy = y, dz = z;
        if (!(fabs(dx) <= bound && fabs(dy) <= bound && fabs(dz) <= bound)) b = 1;
        const double d = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
        if (d > m) m = d;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_down_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
        b |= __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (b) atomicOr(&ctrl->bad, 1);
        atomicMax(&ctrl->dmax_bits, (unsigned long long)__double_as_longlong(m));
    }
}

// one warp per node: the node's A from the segment cosines / sines, then the
// Eq. (11) count over the scan
__global__ void __launch_bounds__(256) na_score_kernel(NaArgs a)
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
                atomicOr(&a.ctrl->err, 1);
            }
            continue;
        }
        // A = fl32(R / r), the same FP64 operations as every other entry point
        const uint32_t rot = (uint32_t)(((int64_t)c[3] * a.grid.N[l][1] + c[4]) * a.grid.N[l][2] + c[5]);
        float A[9];
        rotation_rows(a.cs, a.grid, l, rot, A);
        const float4 r0 = make_float4(A[0], A[1], A[2], 0.0f);
        const float4 r1 = make_float4(A[3], A[4], A[5], 0.0f);
        const float4 r2 = make_float4(A[6], A[7], A[8], 0.0f);
        const LevelView L = a.maps[l];
        uint32_t hits = 0;
        for (int64_t k = lane; k < a.k; k += 32) {
            const float4 s = a.scan[k];
            const int32_t kx = (fine_key(r0, s) >> l) + c[0];
            const int32_t ky = (fine_key(r1, s) >> l) + c[1];
            const int32_t kz = (fine_key(r2, s) >> l) + c[2];
            hits += voxel_bit(L, kx, ky, kz);
        }
        hits = __reduce_add_sync(0xffffffffu, hits);
        if (lane == 0) a.scores[w] = (int32_t)hits;
    }
}

// per-device address of the scratch array, looked up once with the device current
std::mutex g_na_mutex;
void* g_na_ptr[64];
double2 g_na_cs_host[BBS_NOALLOC_MAX_ANGLES];   // host staging of the (cos, sin) table

int na_scratch(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= 64) return set_error(BBS_EINVAL, "score_batch_noalloc: device %d out of range", dev);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return set_error(BBS_ECUDA, "score_batch_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_na_ptr[dev] = p;
    }
    *out = (unsigned char*)g_na_ptr[dev];
    return BBS_OK;
}

// whether p is device (or managed) memory of device dev; the query allocates nothing
bool on_device(const void* p, int dev)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // an unregistered host pointer: clear the sticky-free error
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

}  // namespace bbs

using namespace bbs;

extern "C" int bbs_score_batch_noalloc(const bbs_maps* m, const float* scan_xyz, int64_t k, const bbs_ranges* ranges,
                                       const bbs_opts* opts, const int32_t* nodes, int64_t n, int32_t* scores)
{
    clear_error();
    if (!m || k < 0 || n < 0 || (k > 0 && !scan_xyz) || (n > 0 && (!nodes || !scores)))
        return set_error(BBS_EINVAL, "score_batch_noalloc: bad arguments");
    if (k > BBS_NOALLOC_MAX_POINTS)
        return set_error(BBS_EINVAL, "score_batch_noalloc: %lld scan points exceed the maximum of %d", (long long)k,
                         BBS_NOALLOC_MAX_POINTS);
    if (n == 0) return BBS_OK;
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != m->device && cudaSetDevice(m->device) != cudaSuccess)
        return set_error(BBS_ECUDA, "score_batch_noalloc: cannot select device %d", m->device);
    struct Restore {
        int prev, dev;
        ~Restore()
        {
            if (prev >= 0 && prev != dev) cudaSetDevice(prev);
        }
    } restore{prev, m->device};

    // every buffer must be memory the kernels can read on the maps' device
    if ((k > 0 && !on_device(scan_xyz, m->device)) || !on_device(nodes, m->device) || !on_device(scores, m->device))
        return set_error(BBS_EINVAL, "score_batch_noalloc: scan, nodes and scores must be device memory on device %d",
                         m->device);

    std::lock_guard<std::mutex> lock(g_na_mutex);
    unsigned char* base = nullptr;
    BBS_TRY(na_scratch(m->device, &base));
    cudaStream_t st = opts ? (cudaStream_t)opts->cuda_stream : (cudaStream_t)0;
    NaCtrl* ctrl = (NaCtrl*)base;
    double2* cs = (double2*)(base + NA_CS_OFF);
    float4* scan = (float4*)(base + NA_SCAN_OFF);

    // 1. scan -> float4 in the scratch array, d_max and validation
    BBS_CUDA_TRY(cudaMemsetAsync(ctrl, 0, sizeof(NaCtrl), st));
    if (k > 0) {
        int blocks = (int)((k + 255) / 256);
        if (blocks > 1024) blocks = 1024;
        na_pack_kernel<<<blocks, 256, 0, st>>>(scan_xyz, k, scan, std::ldexp((double)m->r, 18), ctrl);
        BBS_CUDA_TRY(cudaGetLastError());
    }
    NaCtrl h;
    BBS_CUDA_TRY(cudaMemcpyAsync(&h, ctrl, sizeof(h), cudaMemcpyDeviceToHost, st));
    BBS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h.bad) return set_error(BBS_EINVAL, "score_batch_noalloc: a scan coordinate is not finite or exceeds 2^18 r");

    // 2. pose grid on the host, segment cosines / sines into the scratch array
    bbs_ranges rg;
    if (ranges) rg = *ranges;
    else default_ranges(m, &rg);
    double dm;
    std::memcpy(&dm, &h.dmax_bits, sizeof(dm));
    const double d_max = (opts && opts->d_max > 0.0) ? opts->d_max : dm;
    HostGrid g;
    BBS_TRY(grid_build((double)m->r, m->levels, d_max, &rg, opts ? opts->flags : 0u, &g));
    NaArgs a;
    std::memset(&a, 0, sizeof(a));
    int64_t cnt = 0;
    for (int l = 0; l < g.levels; ++l)
        for (int i = 0; i < 3; ++i) {
            if (g.cs_off[l][i] != cnt) return set_error(BBS_ECORRUPT, "score_batch_noalloc: angle table layout");
            if (cnt + g.N[l][i] > BBS_NOALLOC_MAX_ANGLES)
                return set_error(BBS_EINVAL, "score_batch_noalloc: more than %d angle segments in the grid",
                                 BBS_NOALLOC_MAX_ANGLES);
            for (int64_t c = 0; c < g.N[l][i]; ++c) {
                const double ang = grid_angle(g, l, i, c);
                g_na_cs_host[cnt++] = make_double2(std::cos(ang), std::sin(ang));
            }
        }
    BBS_CUDA_TRY(cudaMemcpyAsync(cs, g_na_cs_host, sizeof(double2) * (size_t)cnt, cudaMemcpyHostToDevice, st));

    // 3. one warp per node
    for (int l = 0; l < MAX_LEVELS; ++l) a.maps[l] = l < m->levels ? level_view(m, l) : LevelView{};
    a.grid = dev_grid(g);
    a.cs = cs;
    a.scan = scan;
    a.k = k;
    a.nodes = nodes;
    a.n = n;
    a.scores = scores;
    a.ctrl = ctrl;
    int nsm = 0;
    BBS_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, m->device));
    int64_t blocks = (n + 7) / 8;
    if (blocks > (int64_t)nsm * 64) blocks = (int64_t)nsm * 64;
    na_score_kernel<<<(int)blocks, 256, 0, st>>>(a);
    BBS_CUDA_TRY(cudaGetLastError());
    BBS_CUDA_TRY(cudaMemcpyAsync(&h, ctrl, sizeof(h), cudaMemcpyDeviceToHost, st));
    BBS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h.err) return set_error(BBS_EINVAL, "score_batch_noalloc: a node lies outside the pose grid");
    return BBS_OK;
}
