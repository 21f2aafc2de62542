// grid.cu -- pose grid (Sec. III-B Eq. (2)-(5), Sec. III-D Eq. (12)-(14)),
// scan upload and the per-level rotation tables.
//
// The grid is host FP64 arithmetic (a few hundred values).  Rotation rows
// are formed on the GPU from host cos/sin values with IEEE FP64 products and
// sums (__dmul_rn, __dadd_rn), then A = fl32(R / r) with the correctly
// rounded quotient (rotation_rows, bbs_internal.cuh): the top level's table
// here, every other level's rows as the search expands rotations.  Host code is
// compiled with -ffp-contract=off and device code with -fmad=false, so every
// FP64 operation rounds on its own.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include <algorithm>

#include "bbs_internal.cuh"

namespace bbs {

// Eq. (2): delta(r) = arccos(1 - r^2 / (2 d_max^2)), argument clamped to
// [-1, 1]; d_max <= 0 gives pi.
static double angular_step(double r, double d_max)
{
    if (!(d_max > 0.0)) return std::acos(-1.0);
    double x = 1.0 - (r * r) / (2.0 * d_max * d_max);
    if (x < -1.0) x = -1.0;
    if (x > 1.0) x = 1.0;
    return std::acos(x);
}

int grid_build(double r, int levels, double d_max, const bbs_ranges* rg, uint32_t flags, HostGrid* g)
{
    if (!(r > 0.0) || levels < 1 || levels > MAX_LEVELS)
        return set_error(BBS_EINVAL, "grid: bad r (%g) or levels (%d)", r, levels);
    std::memset(g, 0, sizeof(*g));
    g->levels = levels;
    g->r = r;
    g->d_max = d_max;
    g->flags = flags;
    for (int i = 0; i < 3; ++i) {
        if (!(rg->ang_hi[i] >= rg->ang_lo[i]) || !std::isfinite(rg->ang_lo[i]) || !std::isfinite(rg->ang_hi[i]))
            return set_error(BBS_EINVAL, "grid: angle range %d is empty or not finite", i);
        if (!(rg->hi[i] >= rg->lo[i]) || !std::isfinite(rg->lo[i]) || !std::isfinite(rg->hi[i]))
            return set_error(BBS_EINVAL, "grid: translation range %d is empty or not finite", i);
        g->ang_lo[i] = rg->ang_lo[i];
        g->ang_range[i] = rg->ang_hi[i] - rg->ang_lo[i];
    }
    for (int l = 0; l < levels; ++l) {
        // translation-only branching keeps the level-0 rotation grid everywhere
        const int src = (flags & BBS_TRANSLATION_ONLY) ? 0 : l;
        g->delta[l] = angular_step(std::ldexp(r, src), d_max);
        for (int i = 0; i < 3; ++i) {
            const double W = g->ang_range[i];
            int64_t n = 1;  // a zero-width range is one segment of width 0
            if (W > 0.0) {
                const double q = std::ceil(W / g->delta[l]);   // Eq. (12)
                if (!(q < 1e9)) return set_error(BBS_EINVAL, "grid: %g angle segments", q);
                n = (int64_t)q;
                if (n < 1) n = 1;
            }
            g->N[l][i] = n;
            g->dprime[l][i] = W / (double)n;
        }
    }
    // Eq. (14): a = ceil(delta'_l / delta'_{l-1}) = ceil(N_{l-1} / N_l) in
    // integers; 1 when the finer level has a single segment.
    for (int l = 1; l < levels; ++l)
        for (int i = 0; i < 3; ++i) {
            const int64_t np = g->N[l][i], nc = g->N[l - 1][i];
            g->a[l][i] = ((flags & BBS_TRANSLATION_ONLY) || nc <= 1) ? 1 : (nc + np - 1) / np;
        }
    for (int i = 0; i < 3; ++i) g->a[0][i] = 1;
    // Eq. (3)-(5): initial translation indices at l_max
    const double rmax = std::ldexp(r, levels - 1);
    for (int i = 0; i < 3; ++i) {
        const double lo = std::floor(rg->lo[i] / rmax), hi = std::ceil(rg->hi[i] / rmax);
        if (!(std::fabs(lo) < 1e15) || !(std::fabs(hi) < 1e15))
            return set_error(BBS_EKEYRANGE, "grid: translation range beyond the key range");
        g->wmin[i] = (int64_t)lo;
        g->wmax[i] = (int64_t)hi;
        const int64_t tlo = g->wmin[i] * ((int64_t)1 << (levels - 1));
        const int64_t thi = (g->wmax[i] + 1) * ((int64_t)1 << (levels - 1));
        if (tlo < -((int64_t)1 << 20) || thi > ((int64_t)1 << 20))
            return set_error(BBS_EKEYRANGE, "grid: leaf translations beyond +-2^20 voxels on axis %d", i);
    }
    int64_t off = 0;
    for (int l = 0; l < levels; ++l) {
        const int64_t n = g->N[l][0] * g->N[l][1] * g->N[l][2];
        if (n > ((int64_t)1 << 25))
            return set_error(BBS_EINVAL, "grid: %lld rotations at level %d exceed 2^25", (long long)n, l);
        g->nrot[l] = n;
        g->rot_off[l] = off;
        off += n;
    }
    if (off > ((int64_t)1 << 26)) return set_error(BBS_EINVAL, "grid: %lld rotations in total", (long long)off);
    g->total_rot = off;
    int64_t cso = 0;
    for (int l = 0; l < levels; ++l)
        for (int i = 0; i < 3; ++i) {
            g->cs_off[l][i] = cso;
            cso += g->N[l][i];
        }
    g->n_cs = cso;
    return BBS_OK;
}

// Angle of segment c: the segment centre W_min + (c + 1/2) delta' (the
// paper gives no offset), or W_min + c delta' with BBS_ANGLE_LOWER_EDGE.
double grid_angle(const HostGrid& g, int level, int axis, int64_t c)
{
    const double dp = g.dprime[level][axis];
    if (g.flags & BBS_ANGLE_LOWER_EDGE) return g.ang_lo[axis] + (double)c * dp;
    return g.ang_lo[axis] + ((double)c + 0.5) * dp;
}

DevGrid dev_grid(const HostGrid& g)
{
    DevGrid d;
    std::memset(&d, 0, sizeof(d));
    d.levels = g.levels;
    d.flags = g.flags;
    for (int l = 0; l < g.levels; ++l) {
        for (int i = 0; i < 3; ++i) {
            d.N[l][i] = (int32_t)g.N[l][i];
            d.a[l][i] = (int32_t)g.a[l][i];
        }
        for (int i = 0; i < 3; ++i) d.cs_off[l][i] = (int32_t)g.cs_off[l][i];
    }
    d.r = g.r;
    d.inv_r = 1.0 / g.r;
    return d;
}

void default_ranges(const bbs_maps* m, bbs_ranges* rg)
{
    for (int i = 0; i < 3; ++i) {
        rg->lo[i] = m->lo[i];
        rg->hi[i] = m->hi[i];
    }
    rg->ang_lo[0] = rg->ang_lo[1] = -0.02;   // Sec. IV: roll, pitch (-0.02, 0.02)
    rg->ang_hi[0] = rg->ang_hi[1] = 0.02;
    rg->ang_lo[2] = 0.0;                      // Sec. III-D: yaw (0, 2 pi)
    rg->ang_hi[2] = 2.0 * std::acos(-1.0);
}

// ---------------------------------------------------------------------------
// scan upload: K x 3 float -> K float4; d_max and validation in FP64
// ---------------------------------------------------------------------------

// One CTA per chunk of SCAN_CHUNK points: pack xyz into float4, check the
// coordinate bound, write the chunk's box (the scoring kernel tests a run
// against it to drop the per-point range checks), and raise smax_bits to the
// chunk's largest s = (x^2 + y^2) + z^2 in FP64, each operation rounded on
// its own (the norm is sqrt of the maximum: sqrt rounds monotonically).
// FP64 is slow on this part, so s is formed in FP64 only for the points
// whose FP32 estimate lies within 1e-6 of the chunk's largest estimate (the
// two differ by under 4e-7 relative, so the FP64 maximum is among them).
constexpr int PACK_THREADS = 256;
constexpr int PACK_PER = (SCAN_CHUNK + PACK_THREADS - 1) / PACK_THREADS;
__global__ void __launch_bounds__(PACK_THREADS) scan_pack_kernel(const float* __restrict__ xyz, int64_t k,
                                                                 float4* __restrict__ out, float4* __restrict__ cbox,
                                                                 float bound, unsigned long long* __restrict__ smax_bits,
                                                                 int* __restrict__ bad)
{
    __shared__ float red[7][PACK_THREADS / 32];
    const int64_t c0 = (int64_t)blockIdx.x * SCAN_CHUNK;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int b = 0;
    float v[7] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0f};   // box, largest s
    float px[PACK_PER], py[PACK_PER], pz[PACK_PER], ps[PACK_PER];
#pragma unroll
    for (int j = 0; j < PACK_PER; ++j) {
        const int r = (int)threadIdx.x + j * PACK_THREADS;   // the point's place in the chunk
        const int64_t i = c0 + r;
        ps[j] = -1.0f;
        if (r < SCAN_CHUNK && i < k) {
            const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
            out[i] = make_float4(x, y, z, 0.0f);
            if (!(fabsf(x) <= bound && fabsf(y) <= bound && fabsf(z) <= bound)) b = 1;   // also catches NaN
            px[j] = x, py[j] = y, pz[j] = z;
            ps[j] = __fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z));
            v[0] = fminf(v[0], x), v[1] = fminf(v[1], y), v[2] = fminf(v[2], z);
            v[3] = fmaxf(v[3], x), v[4] = fmaxf(v[4], y), v[5] = fmaxf(v[5], z);
            v[6] = fmaxf(v[6], ps[j]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        b |= __shfl_xor_sync(0xffffffffu, b, o);
        for (int a = 0; a < 7; ++a) {
            const float t = __shfl_xor_sync(0xffffffffu, v[a], o);
            v[a] = a < 3 ? fminf(v[a], t) : fmaxf(v[a], t);
        }
    }
    if (lane == 0) {
        if (b) atomicOr(bad, 1);
        for (int a = 0; a < 7; ++a) red[a][w] = v[a];
    }
    __syncthreads();
    float r[7];
    for (int a = 0; a < 7; ++a) {
        r[a] = red[a][0];
        for (int j = 1; j < PACK_THREADS / 32; ++j) r[a] = a < 3 ? fminf(r[a], red[a][j]) : fmaxf(r[a], red[a][j]);
    }
    if (threadIdx.x == 0) {
        cbox[2 * blockIdx.x] = make_float4(r[0], r[1], r[2], 0.0f);
        cbox[2 * blockIdx.x + 1] = make_float4(r[3], r[4], r[5], 0.0f);
    }
    const float thr = __fmul_rn(r[6], 0.999999f);
    double m = 0.0;
#pragma unroll
    for (int j = 0; j < PACK_PER; ++j)
        if (ps[j] >= thr && ps[j] >= 0.0f) {
            const double dx = px[j], dy = py[j], dz = pz[j];
            const double sd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            m = sd > m ? sd : m;
        }
    // non-negative doubles order like their bit patterns
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if (lane == 0 && m > 0.0) atomicMax(smax_bits, (unsigned long long)__double_as_longlong(m));
}

// the rows of every rotation of one level (search_rows: the search's own
// row formation, so the pose grid's rows pin it)
__global__ void level_rows_kernel(const double2* __restrict__ cs, DevGrid g, int level, int64_t n, float4* __restrict__ out)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        float A[9];
        search_rows(cs, g, level, (uint32_t)t, A);
        out[3 * t + 0] = make_float4(A[0], A[1], A[2], 0.0f);
        out[3 * t + 1] = make_float4(A[3], A[4], A[5], 0.0f);
        out[3 * t + 2] = make_float4(A[6], A[7], A[8], 0.0f);
    }
}

static int grid_blocks(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;
    return (int)b;
}

// cos / sin of the segment angles of levels [l0, l1), uploaded to their place
// in s.cs (a copy from pageable memory has staged its source by the time
// cudaMemcpyAsync returns, so the host vector may go)
static cudaError_t upload_angles(ScanState& s, int l0, int l1, cudaStream_t st)
{
    const HostGrid& g = s.grid;
    if (l0 >= l1) return cudaSuccess;
    const int64_t a = g.cs_off[l0][0], b = l1 < g.levels ? g.cs_off[l1][0] : g.n_cs;
    if (b <= a) return cudaSuccess;
    std::vector<double2> cs((size_t)(b - a));
    for (int l = l0; l < l1; ++l)
        for (int i = 0; i < 3; ++i)
            for (int64_t c = 0; c < g.N[l][i]; ++c) {
                const double ang = grid_angle(g, l, i, c);
                cs[(size_t)(g.cs_off[l][i] + c - a)] = make_double2(std::cos(ang), std::sin(ang));
            }
    s.h2d += (int64_t)(sizeof(double2) * cs.size());
    return cudaMemcpyAsync(s.cs + a, cs.data(), sizeof(double2) * cs.size(), cudaMemcpyHostToDevice, st);
}

int scan_finish_angles(ScanState* s, cudaStream_t st)
{
    if (!s->angles_pending) return BBS_OK;
    s->angles_pending = 0;
    BBS_CUDA_TRY(upload_angles(*s, 0, s->grid.levels - 1, st));
    return BBS_OK;
}

int scan_prepare(const bbs_maps* m, const float* xyz, int64_t k, int is_device, const bbs_ranges* rg_in,
                 const bbs_opts* opts, cudaStream_t st, ScanState* out, bool defer_lower)
{
    std::memset(out, 0, sizeof(*out));
    if (k < 0) return set_error(BBS_EINVAL, "scan: k < 0");
    if (k > 0 && !xyz) return set_error(BBS_EINVAL, "scan: NULL points");
    bbs_ranges rg;
    if (rg_in) rg = *rg_in;
    else default_ranges(m, &rg);
    out->k = k;
    const int64_t kk = k > 0 ? k : 1;
    BBS_CUDA_TRY(cudaMallocAsync((void**)&out->scan, sizeof(float4) * (size_t)kk, st));
    BBS_CUDA_TRY(cudaMallocAsync((void**)&out->cbox, sizeof(float4) * 2 * (size_t)((kk + SCAN_CHUNK - 1) / SCAN_CHUNK), st));
    if (k == 0) BBS_CUDA_TRY(cudaMemsetAsync(out->cbox, 0, sizeof(float4) * 2, st));
    struct Aux { unsigned long long dmax; int bad; int pad; };
    Aux* d_aux = nullptr;
    float* d_xyz = nullptr;
    BBS_CUDA_TRY(cudaMallocAsync((void**)&d_aux, sizeof(Aux), st));
    BBS_CUDA_TRY(cudaMemsetAsync(d_aux, 0, sizeof(Aux), st));
    const float* src = xyz;
    if (k > 0 && !is_device) {
        BBS_CUDA_TRY(cudaMallocAsync((void**)&d_xyz, sizeof(float) * 3 * (size_t)k, st));
        BBS_CUDA_TRY(cudaMemcpyAsync(d_xyz, xyz, sizeof(float) * 3 * (size_t)k, cudaMemcpyHostToDevice, st));
        out->h2d += (int64_t)(sizeof(float) * 3 * (size_t)k);
        src = d_xyz;
    }
    const double bound = std::ldexp((double)m->r, 18);
    float bound_f = (float)bound;   // the largest float <= bound: |x| <= bound_f iff |x| <= bound
    if ((double)bound_f > bound) bound_f = std::nextafter(bound_f, 0.0f);
    if (k > 0) {
        scan_pack_kernel<<<(unsigned)((k + SCAN_CHUNK - 1) / SCAN_CHUNK), 256, 0, st>>>(src, k, out->scan, out->cbox,
                                                                                    bound_f, &d_aux->dmax, &d_aux->bad);
        BBS_CUDA_TRY(cudaGetLastError());
    }
    Aux aux;
    BBS_CUDA_TRY(cudaMemcpyAsync(&aux, d_aux, sizeof(Aux), cudaMemcpyDeviceToHost, st));
    out->d2h += (int64_t)sizeof(Aux);
    BBS_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFreeAsync(d_aux, st);
    if (d_xyz) cudaFreeAsync(d_xyz, st);
    if (aux.bad) {
        scan_release(out, st);
        return set_error(BBS_EINVAL, "scan: a coordinate is not finite or exceeds 2^18 r");
    }
    double smax;
    std::memcpy(&smax, &aux.dmax, sizeof(smax));
    const double dm = std::sqrt(smax);   // correctly rounded, as the per-point sqrt
    out->norm_max = dm;
    out->d_max = (opts && opts->d_max > 0.0) ? opts->d_max : dm;
    const uint32_t flags = opts ? opts->flags : 0u;
    int rc = grid_build((double)m->r, m->levels, out->d_max, &rg, flags, &out->grid);
    if (rc < 0) {
        scan_release(out, st);
        return rc;
    }
    // cos / sin of every segment angle (host libm, FP64), kept on the device:
    // the search forms the rotation rows of the rotations it expands.  The
    // top level's entries come first (the initial set needs only them); with
    // defer_lower the other levels' follow in scan_finish_angles, which the
    // engine calls while the GPU scores the initial set.
    const HostGrid& g = out->grid;
    const int top = g.levels - 1;
    BBS_CUDA_TRY(cudaMallocAsync((void**)&out->cs, sizeof(double2) * (size_t)g.n_cs, st));
    BBS_CUDA_TRY(upload_angles(*out, top, g.levels, st));
    if (defer_lower) out->angles_pending = 1;
    else BBS_CUDA_TRY(upload_angles(*out, 0, top, st));
    // the top level's rows (the initial set scores every one of them)
    BBS_CUDA_TRY(cudaMallocAsync((void**)&out->rot, sizeof(float4) * 3 * (size_t)g.nrot[top], st));
    BBS_CUDA_TRY(launch_level_rows(*out, top, out->rot, st));
    // the host vector may go: a copy from pageable memory has staged its
    // source by the time cudaMemcpyAsync returns
    return BBS_OK;
}

cudaError_t launch_level_rows(const ScanState& s, int level, float4* out, cudaStream_t st)
{
    const int64_t n = s.grid.nrot[level];
    if (n <= 0) return cudaSuccess;
    level_rows_kernel<<<grid_blocks(n, 256), 256, 0, st>>>(s.cs, dev_grid(s.grid), level, n, out);
    return cudaGetLastError();
}

// Extra dilation the exact-bound mode needs (BBS_EXACT_BOUND in bbs.h): a
// leaf's angle lies within sum_{k=1..l} w delta'_k of a level-l node's per
// axis (w = 1/2, a whole segment with the lower-edge angles; nothing where a
// level and its finer one both have a single segment), so the rotation
// between them is at most theta_l, the sum over the axes, and a point of norm
// at most d moves by theta_l d / r fine voxels; with 2 for the floors and the
// FP32 keys, e = max over l >= 1 of ceil((theta_l d / r + 2) / 2^l).
int exact_dilation_needed(const HostGrid& g, double norm_max)
{
    if (g.flags & BBS_CHILD_LITERAL) return -1;
    const double w = (g.flags & BBS_ANGLE_LOWER_EDGE) ? 1.0 : 0.5;
    const double d = norm_max > g.d_max ? norm_max : g.d_max;
    double acc[3] = {0.0, 0.0, 0.0};
    int need = 0;
    for (int l = 1; l < g.levels; ++l) {
        double theta = 0.0;
        for (int a = 0; a < 3; ++a) {
            if (g.N[l][a] != 1 || g.N[l - 1][a] != 1) acc[a] += w * g.dprime[l][a];
            theta += acc[a];
        }
        const int e = (int)std::ceil((theta * d / g.r + 2.0) / std::ldexp(1.0, l));
        need = std::max(need, e);
    }
    return need;
}

void scan_release(ScanState* s, cudaStream_t st)
{
    if (s->scan) cudaFreeAsync(s->scan, st);
    if (s->rot) cudaFreeAsync(s->rot, st);
    if (s->cs) cudaFreeAsync(s->cs, st);
    if (s->cbox) cudaFreeAsync(s->cbox, st);
    s->cbox = nullptr;
    s->scan = nullptr;
    s->rot = nullptr;
    s->cs = nullptr;
}

}  // namespace bbs
