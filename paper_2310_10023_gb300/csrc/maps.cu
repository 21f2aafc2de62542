// maps.cu -- GPU builder of the per-level sparse hash voxel maps H^l
// (Sec. III-C, Eq. (10)).
//
//   1. fine keys u = floor(fl32(m * fl32(1/r))) of every map point,
//      de-duplicated in a 64-bit open-addressing key set        -> B_0
//   2. B_l = { b >> 1 : b in B_{l-1} }, de-duplicated            (the identity
//      floor(floor(x) / 2) = floor(x / 2) makes this the paper's per-level
//      recomputation floor(x / r_l) without touching the points again)
//   3. D_l = { v - j : v in B_l, j in {0,1}^3 }   (the dilation "for upper
//      bound calculation"; level 0 too unless BBS_LEAF_UNDILATED)
//      scattered into 5x5x5-overlap bricks with atomicOr
//   4. the bricks are moved into the final table at the target load factor,
//      recording the longest probe distance so lookups stop early.
#include <climits>
#include <cstring>

#include "bbs_internal.cuh"

namespace bbs {

namespace {

constexpr unsigned long long VEMPTY = ~0ull;

__host__ __device__ __forceinline__ unsigned long long vpack(int32_t x, int32_t y, int32_t z)
{
    return ((unsigned long long)(uint32_t)(x + KEY_LIMIT) << 42) | ((unsigned long long)(uint32_t)(y + KEY_LIMIT) << 21) |
           (unsigned long long)(uint32_t)(z + KEY_LIMIT);
}

__device__ __forceinline__ void vunpack(unsigned long long k, int32_t& x, int32_t& y, int32_t& z)
{
    x = (int32_t)((k >> 42) & 0x1FFFFF) - KEY_LIMIT;
    y = (int32_t)((k >> 21) & 0x1FFFFF) - KEY_LIMIT;
    z = (int32_t)(k & 0x1FFFFF) - KEY_LIMIT;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return x;
}

struct BuildStatus {
    unsigned long long count;   // keys / bricks inserted
    int overflow;
    int keyrange;
    int bad;
    int maxp;
    unsigned long long displaced;
    unsigned long long voxels;
    int kmin[3], kmax[3];       // bounds of a level's undilated keys
};

// insert-if-absent into a key set of size mask + 1; returns true if inserted
__device__ __forceinline__ bool set_insert(unsigned long long* set, unsigned long long mask, unsigned long long key,
                                           BuildStatus* st, unsigned long long limit)
{
    unsigned long long s = mix64(key) & mask;
    for (unsigned long long p = 0; p <= mask; ++p) {
        unsigned long long* slot = set + ((s + p) & mask);
        unsigned long long cur = *slot;
        if (cur == key) return false;
        if (cur == VEMPTY) {
            cur = atomicCAS(slot, VEMPTY, key);
            if (cur == VEMPTY) {
                if (atomicAdd(&st->count, 1ull) + 1 > limit) st->overflow = 1;
                return true;
            }
            if (cur == key) return false;
        }
        if (*(volatile int*)&st->overflow) return false;
    }
    st->overflow = 1;
    return false;
}

__global__ void fill_u64(unsigned long long* p, int64_t n, unsigned long long v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void init_bricks(Brick* b, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Brick e;
        e.key = EMPTY_KEY;
        for (int z = 0; z < 5; ++z) e.plane[z] = 0;
        e.pad = 0;
        b[i] = e;
    }
}

// bounding box (ordered-bit encoding for atomics) and fine keys into the set
__device__ __forceinline__ unsigned long long ord(double d)
{
    unsigned long long u = (unsigned long long)__double_as_longlong(d);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void quantize_kernel(const float* __restrict__ xyz, int64_t n, float rho, unsigned long long* set,
                                unsigned long long mask, BuildStatus* st, unsigned long long* bbox)
{
    unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t u[3];
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
            const float v = xyz[3 * i + a];
            if (!isfinite(v)) {
                st->bad = 1;
                ok = false;
                break;
            }
            const unsigned long long o = ord((double)v);
            mn[a] = o < mn[a] ? o : mn[a];
            mx[a] = o > mx[a] ? o : mx[a];
            const float f = floorf(__fmul_rn(v, rho));
            if (!(f >= -(float)MAP_KEY_MAX && f <= (float)MAP_KEY_MAX)) {
                st->keyrange = 1;
                ok = false;
                break;
            }
            u[a] = (int32_t)f;
        }
        if (ok) set_insert(set, mask, vpack(u[0], u[1], u[2]), st, ~0ull);
    }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long x = __shfl_down_sync(0xffffffffu, mn[a], o);
            const unsigned long long y = __shfl_down_sync(0xffffffffu, mx[a], o);
            mn[a] = x < mn[a] ? x : mn[a];
            mx[a] = y > mx[a] ? y : mx[a];
        }
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            atomicMin(&bbox[a], mn[a]);
            atomicMax(&bbox[3 + a], mx[a]);
        }
}

// stream-compact the occupied slots of a key set
__global__ void compact_set(const unsigned long long* set, int64_t T, unsigned long long* out, unsigned long long* n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = set[i];
        if (k != VEMPTY) out[atomicAdd(n, 1ull)] = k;
    }
}

// B_l = { b >> 1 } de-duplicated
__global__ void halve_kernel(const unsigned long long* in, int64_t n, unsigned long long* set, unsigned long long mask,
                             BuildStatus* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t x, y, z;
        vunpack(in[i], x, y, z);
        set_insert(set, mask, vpack(x >> 1, y >> 1, z >> 1), st, ~0ull);
    }
}

// find-or-insert a brick; returns the slot or nullptr on overflow
__device__ __forceinline__ Brick* brick_slot(Brick* tab, uint32_t shift, uint32_t mask, int32_t bx, int32_t by,
                                             int32_t bz, BuildStatus* st, unsigned long long limit)
{
    const unsigned long long key = brick_pack(bx, by, bz);
    const uint32_t s = brick_hash(bx, by, bz) >> shift;
    for (uint32_t p = 0; p <= mask; ++p) {
        Brick* b = tab + ((s + p) & mask);
        unsigned long long cur = b->key;
        if (cur == key) return b;
        if (cur == EMPTY_KEY) {
            cur = atomicCAS(&b->key, EMPTY_KEY, key);
            if (cur == EMPTY_KEY) {
                if (atomicAdd(&st->count, 1ull) + 1 > limit) st->overflow = 1;
                return b;
            }
            if (cur == key) return b;
        }
        if (*(volatile int*)&st->overflow) return nullptr;
    }
    st->overflow = 1;
    return nullptr;
}

__device__ __forceinline__ void set_voxel(Brick* tab, uint32_t shift, uint32_t mask, int32_t vx, int32_t vy,
                                          int32_t vz, BuildStatus* st, unsigned long long limit)
{
    const int32_t bx = vx >> 2, by = vy >> 2, bz = vz >> 2;
    const int32_t ox = vx & 3, oy = vy & 3, oz = vz & 3;
    // the home brick, plus the lower neighbours in whose overlap face (local 4) v lies
    for (int sx = 0; sx <= (ox == 0); ++sx)
        for (int sy = 0; sy <= (oy == 0); ++sy)
            for (int sz = 0; sz <= (oz == 0); ++sz) {
                Brick* b = brick_slot(tab, shift, mask, bx - sx, by - sy, bz - sz, st, limit);
                if (!b) return;
                atomicOr(&b->plane[oz + 4 * sz], 1u << ((ox + 4 * sx) + 5 * (oy + 4 * sy)));
            }
}

// D_l: every key minus j, j in [jlo, jhi]^3 ({0,1}^3 is the dilation of
// Sec. III-C; the exact-bound mode widens it; jlo = jhi = 0 stores B_l)
__global__ void dilate_kernel(const unsigned long long* keys, int64_t n, int jlo, int jhi, Brick* tab, uint32_t shift,
                              uint32_t mask, BuildStatus* st, unsigned long long limit)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (*(volatile int*)&st->overflow) return;
        int32_t x, y, z;
        vunpack(keys[i], x, y, z);
        for (int jx = jlo; jx <= jhi; ++jx)
            for (int jy = jlo; jy <= jhi; ++jy)
                for (int jz = jlo; jz <= jhi; ++jz) set_voxel(tab, shift, mask, x - jx, y - jy, z - jz, st, limit);
    }
}

// bounds of the undilated keys of a level
__global__ void key_bounds_kernel(const unsigned long long* keys, int64_t n, BuildStatus* st)
{
    int mn[3] = {INT_MAX, INT_MAX, INT_MAX}, mx[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[3];
        vunpack(keys[i], v[0], v[1], v[2]);
        for (int a = 0; a < 3; ++a) {
            mn[a] = min(mn[a], v[a]);
            mx[a] = max(mx[a], v[a]);
        }
    }
    for (int a = 0; a < 3; ++a) {
        mn[a] = __reduce_min_sync(0xffffffffu, mn[a]);
        mx[a] = __reduce_max_sync(0xffffffffu, mx[a]);
    }
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            atomicMin(&st->kmin[a], mn[a]);
            atomicMax(&st->kmax[a], mx[a]);
        }
}

// move every brick into a compact final table: relative 32-bit key, each
// 16-byte half [key, 3 planes]
__global__ void relayout_compact_kernel(const Brick* src, int64_t T, Brick* dst, uint32_t shift, uint32_t mask,
                                        int bx0, int by0, int bz0, BuildStatus* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x) {
        const Brick b = src[i];
        if (b.key == EMPTY_KEY) continue;
        const int32_t bx = (int32_t)((b.key >> 40) & 0xFFFFF) - BRICK_BIAS;
        const int32_t by = (int32_t)((b.key >> 20) & 0xFFFFF) - BRICK_BIAS;
        const int32_t bz = (int32_t)(b.key & 0xFFFFF) - BRICK_BIAS;
        const uint32_t key = cbrick_pack((uint32_t)(bx - bx0), (uint32_t)(by - by0), (uint32_t)(bz - bz0));
        const uint32_t s = cbrick_hash(key) >> shift;
        for (uint32_t p = 0; p <= mask; ++p) {
            Brick* d = dst + ((s + p) & mask);
            uint32_t* w = reinterpret_cast<uint32_t*>(d);
            if (atomicCAS(w, CEMPTY, key) == CEMPTY) {
                w[1] = b.plane[0];
                w[2] = b.plane[1];
                w[3] = b.plane[2];
                w[5] = b.plane[2];
                w[6] = b.plane[3];
                w[7] = b.plane[4];
                w[4] = key;
                atomicMax(&st->maxp, (int)p);
                if (p) atomicAdd(&st->displaced, 1ull);
                unsigned c = 0;
                for (int z = 0; z < 4; ++z) c += __popc(b.plane[z] & 0x7BDEFu);
                atomicAdd(&st->voxels, (unsigned long long)c);
                break;
            }
        }
    }
}

// move every brick to its index in a dense table over the level's brick box
// (relative brick coordinates, x slowest): 16-byte halves [0, 3 planes];
// bricks of the box that hold no voxel stay zero
__global__ void relayout_dense_kernel(const Brick* src, int64_t T, Brick* dst, int bx0, int by0, int bz0, uint32_t nby,
                                      uint32_t nbz, BuildStatus* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x) {
        const Brick b = src[i];
        if (b.key == EMPTY_KEY) continue;
        const int32_t bx = (int32_t)((b.key >> 40) & 0xFFFFF) - BRICK_BIAS;
        const int32_t by = (int32_t)((b.key >> 20) & 0xFFFFF) - BRICK_BIAS;
        const int32_t bz = (int32_t)(b.key & 0xFFFFF) - BRICK_BIAS;
        const int64_t idx = ((int64_t)(bx - bx0) * nby + (uint32_t)(by - by0)) * nbz + (uint32_t)(bz - bz0);
        uint32_t* w = reinterpret_cast<uint32_t*>(dst + idx);
        w[0] = 0u;
        w[1] = b.plane[0];
        w[2] = b.plane[1];
        w[3] = b.plane[2];
        w[4] = 0u;
        w[5] = b.plane[2];
        w[6] = b.plane[3];
        w[7] = b.plane[4];
        unsigned c = 0;
        for (int z = 0; z < 4; ++z) c += __popc(b.plane[z] & 0x7BDEFu);
        atomicAdd(&st->voxels, (unsigned long long)c);
    }
}

// byte grid from a dense brick table: cell (x, y, z) of nx x ny x nz (x
// slowest) gets bit jx + 2 jy + 4 jz when key (x, y, z) + (jx, jy, jz) of the
// box is in the set (the brick planes carry the +1 halo)
__global__ void bytes_fill_kernel(const Brick* bricks, uint32_t nbx, uint32_t nby, uint32_t nbz, uint8_t* out,
                                  uint32_t nx, uint32_t ny, uint32_t nz)
{
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t z = (uint32_t)(i % nz), y = (uint32_t)((i / nz) % ny), x = (uint32_t)(i / ((int64_t)nz * ny));
        uint32_t v = 0;
        if ((x >> 2) < nbx && (y >> 2) < nby && (z >> 2) < nbz) {
            const uint32_t* w =
                reinterpret_cast<const uint32_t*>(bricks + ((int64_t)(x >> 2) * nby + (y >> 2)) * nbz + (z >> 2));
            const uint32_t p[5] = {w[1], w[2], w[3], w[6], w[7]};
            const uint32_t oz = z & 3u, sh = (x & 3u) + 5u * (y & 3u);
            for (uint32_t jz = 0; jz < 2; ++jz)
                for (uint32_t jy = 0; jy < 2; ++jy)
                    for (uint32_t jx = 0; jx < 2; ++jx)
                        v |= ((p[oz + jz] >> (sh + jx + 5u * jy)) & 1u) << (jx + 2u * jy + 4u * jz);
        }
        out[i] = (uint8_t)v;
    }
}

// the voxels of a byte grid (bit 0 of each cell)
__global__ void bytes_keys_kernel(const uint8_t* cells, uint32_t nx, uint32_t ny, uint32_t nz, int x0, int y0, int z0,
                                  int32_t* out, unsigned long long* n, int64_t cap)
{
    const int64_t T = (int64_t)nx * ny * nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x) {
        if (!(cells[i] & 1u)) continue;
        const unsigned long long o = atomicAdd(n, 1ull);
        if ((int64_t)o < cap) {
            out[3 * o] = (int32_t)(i / ((int64_t)nz * ny)) + x0;
            out[3 * o + 1] = (int32_t)((i / nz) % ny) + y0;
            out[3 * o + 2] = (int32_t)(i % nz) + z0;
        }
    }
}

// the voxels of a dense table (brick index -> relative brick coordinates)
__global__ void dense_keys_kernel(const Brick* tab, int64_t T, int bx0, int by0, int bz0, uint32_t nby, uint32_t nbz,
                                  int32_t* out, unsigned long long* n, int64_t cap)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t* w = reinterpret_cast<const uint32_t*>(tab + i);
        const uint32_t planes[4] = {w[1], w[2], w[3], w[6]};
        if (!(planes[0] | planes[1] | planes[2] | planes[3])) continue;
        const int32_t bz = (int32_t)(i % nbz) + bz0, by = (int32_t)((i / nbz) % nby) + by0;
        const int32_t bx = (int32_t)(i / ((int64_t)nbz * nby)) + bx0;
        for (int z = 0; z < 4; ++z)
            for (int y = 0; y < 4; ++y)
                for (int x = 0; x < 4; ++x)
                    if ((planes[z] >> (x + 5 * y)) & 1u) {
                        const unsigned long long o = atomicAdd(n, 1ull);
                        if ((int64_t)o < cap) {
                            out[3 * o] = 4 * bx + x;
                            out[3 * o + 1] = 4 * by + y;
                            out[3 * o + 2] = 4 * bz + z;
                        }
                    }
    }
}

__global__ void fill_u32(uint32_t* p, int64_t n, uint32_t v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void compact_keys_kernel(const Brick* tab, int64_t T, int bx0, int by0, int bz0, int32_t* out,
                                    unsigned long long* n, int64_t cap)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t* w = reinterpret_cast<const uint32_t*>(tab + i);
        if (w[0] == CEMPTY) continue;
        const int32_t bx = (int32_t)(w[0] & 0x7FF) + bx0, by = (int32_t)((w[0] >> 11) & 0x7FF) + by0;
        const int32_t bz = (int32_t)(w[0] >> 22) + bz0;
        const uint32_t planes[4] = {w[1], w[2], w[3], w[6]};
        for (int z = 0; z < 4; ++z)
            for (int y = 0; y < 4; ++y)
                for (int x = 0; x < 4; ++x)
                    if ((planes[z] >> (x + 5 * y)) & 1u) {
                        const unsigned long long o = atomicAdd(n, 1ull);
                        if ((int64_t)o < cap) {
                            out[3 * o] = 4 * bx + x;
                            out[3 * o + 1] = 4 * by + y;
                            out[3 * o + 2] = 4 * bz + z;
                        }
                    }
    }
}

// move every brick into the final table, recording probe distances
__global__ void relayout_kernel(const Brick* src, int64_t T, Brick* dst, uint32_t shift, uint32_t mask, BuildStatus* st)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x) {
        const Brick b = src[i];
        if (b.key == EMPTY_KEY) continue;
        const int32_t bx = (int32_t)((b.key >> 40) & 0xFFFFF) - BRICK_BIAS;
        const int32_t by = (int32_t)((b.key >> 20) & 0xFFFFF) - BRICK_BIAS;
        const int32_t bz = (int32_t)(b.key & 0xFFFFF) - BRICK_BIAS;
        const uint32_t s = brick_hash(bx, by, bz) >> shift;
        for (uint32_t p = 0; p <= mask; ++p) {
            Brick* d = dst + ((s + p) & mask);
            if (atomicCAS(&d->key, EMPTY_KEY, b.key) == EMPTY_KEY) {
                for (int z = 0; z < 5; ++z) d->plane[z] = b.plane[z];
                atomicMax(&st->maxp, (int)p);
                if (p) atomicAdd(&st->displaced, 1ull);
                // voxels owned by this brick: local coordinates in [0,4)^3
                unsigned c = 0;
                for (int z = 0; z < 4; ++z) c += __popc(b.plane[z] & 0x7BDEFu);
                atomicAdd(&st->voxels, (unsigned long long)c);
                break;
            }
        }
    }
}

__global__ void brick_keys_kernel(const Brick* tab, int64_t T, int32_t* out, unsigned long long* n, int64_t cap)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < T; i += (int64_t)gridDim.x * blockDim.x) {
        const Brick b = tab[i];
        if (b.key == EMPTY_KEY) continue;
        const int32_t bx = (int32_t)((b.key >> 40) & 0xFFFFF) - BRICK_BIAS;
        const int32_t by = (int32_t)((b.key >> 20) & 0xFFFFF) - BRICK_BIAS;
        const int32_t bz = (int32_t)(b.key & 0xFFFFF) - BRICK_BIAS;
        for (int z = 0; z < 4; ++z)
            for (int y = 0; y < 4; ++y)
                for (int x = 0; x < 4; ++x)
                    if ((b.plane[z] >> (x + 5 * y)) & 1u) {
                        const unsigned long long o = atomicAdd(n, 1ull);
                        if ((int64_t)o < cap) {
                            out[3 * o] = 4 * bx + x;
                            out[3 * o + 1] = 4 * by + y;
                            out[3 * o + 2] = 4 * bz + z;
                        }
                    }
    }
}

int blocks_for(int64_t n)
{
    int64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 8192) b = 8192;
    return (int)b;
}

int log2_ceil(unsigned long long x)
{
    int l = 0;
    while ((1ull << l) < x) ++l;
    return l;
}

}  // namespace

// target load of the final brick tables (bricks / buckets)
static double g_load_target = 0.25;
// 0: byte grid where a level's box is small enough, else compact where it
// fits, else wide; 1: always wide; 2: hashed only (compact where it fits);
// 3: dense bricks where the box qualifies, else hashed; 4: byte grid where
// the box qualifies, else hashed
static int g_layout = 0;
// a dense table (bricks or bytes) spans a box of at most this many bricks, and
// at most DENSE_RATIO times the level's occupied bricks plus DENSE_SLACK
// (small maps always qualify)
constexpr int64_t DENSE_MAX = (int64_t)1 << 24;
constexpr int64_t DENSE_RATIO = 64;
constexpr int64_t DENSE_SLACK = (int64_t)1 << 16;

int maps_set_layout(int layout)
{
    if (layout < 0 || layout > 4)
        return set_error(BBS_EINVAL, "probe layout %d (0 auto, 1 wide, 2 hashed, 3 dense, 4 bytes)", layout);
    g_layout = layout;
    return BBS_OK;
}

int maps_set_load(double load)
{
    if (!(load > 0.01 && load <= 0.9)) return set_error(BBS_EINVAL, "load factor %g outside (0.01, 0.9]", load);
    g_load_target = load;
    return BBS_OK;
}

int maps_build(const float* xyz, int64_t n, int is_device, float r, int levels, uint32_t flags, cudaStream_t st,
               bbs_maps** out)
{
    *out = nullptr;
    if (!(r > 0.0f) || !isfinite(r)) return set_error(BBS_EINVAL, "build_maps: r must be positive and finite");
    if (levels < 1 || levels > MAX_LEVELS) return set_error(BBS_EINVAL, "build_maps: levels %d outside 1..16", levels);
    if (n < 0 || (n > 0 && !xyz)) return set_error(BBS_EINVAL, "build_maps: bad point array");
    if (flags & ~(uint32_t)(BBS_LEAF_UNDILATED | BBS_EXACT_BOUND | (15u << 12)))
        return set_error(BBS_EINVAL, "build_maps: unsupported flags 0x%x", flags);
    const int exact_e = (flags & BBS_EXACT_BOUND) ? (int)((flags >> 12) & 15u) : 0;
    if ((flags & BBS_EXACT_BOUND) ? exact_e < 1 : ((flags >> 12) & 15u) != 0)
        return set_error(BBS_EINVAL, "build_maps: BBS_EXACT_BOUND needs an extra dilation e in 1..15");

    bbs_maps* m = new bbs_maps;
    std::memset(m, 0, sizeof(*m));
    cudaGetDevice(&m->device);
    m->levels = levels;
    m->r = r;
    m->flags = flags;

    // device scratch freed on every exit path
    struct Scratch {
        cudaStream_t st;
        void* p[8] = {};
        ~Scratch()
        {
            for (void* q : p)
                if (q) cudaFreeAsync(q, st);
        }
    } sc{st};
    auto fail = [&](int code) {
        for (int l = 0; l < MAX_LEVELS; ++l)
            if (m->lv[l].slots) cudaFree(m->lv[l].slots);
        delete m;
        return code;
    };
#define TRYC(call)                                                                                           \
    do {                                                                                                     \
        cudaError_t e_ = (call);                                                                             \
        if (e_ != cudaSuccess) return fail(set_error(BBS_ECUDA, "build_maps: %s: %s", #call, cudaGetErrorString(e_))); \
    } while (0)

    const float* d_xyz = xyz;
    if (n > 0 && !is_device) {
        TRYC(cudaMallocAsync(&sc.p[0], sizeof(float) * 3 * (size_t)n, st));
        TRYC(cudaMemcpyAsync(sc.p[0], xyz, sizeof(float) * 3 * (size_t)n, cudaMemcpyHostToDevice, st));
        d_xyz = (const float*)sc.p[0];
    }
    BuildStatus* d_st = nullptr;
    TRYC(cudaMallocAsync(&sc.p[1], sizeof(BuildStatus) + 6 * sizeof(unsigned long long), st));
    d_st = (BuildStatus*)sc.p[1];
    unsigned long long* d_bbox = (unsigned long long*)(d_st + 1);
    BuildStatus hs;

    auto reset_status = [&]() -> int {
        BuildStatus z;
        std::memset(&z, 0, sizeof(z));
        if (cudaMemcpyAsync(d_st, &z, sizeof(z), cudaMemcpyHostToDevice, st) != cudaSuccess) return BBS_ECUDA;
        return BBS_OK;
    };
    auto read_status = [&]() -> int {
        if (cudaMemcpyAsync(&hs, d_st, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess) return BBS_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return BBS_ECUDA;
        return BBS_OK;
    };

    // ---- 1. fine keys B_0 ------------------------------------------------
    const float rho = (float)(1.0 / (double)r);
    const int lT0 = log2_ceil((unsigned long long)(2 * (n > 512 ? n : 512)));
    const int64_t T0 = (int64_t)1 << lT0;
    TRYC(cudaMallocAsync(&sc.p[2], sizeof(unsigned long long) * (size_t)T0, st));
    unsigned long long* set0 = (unsigned long long*)sc.p[2];
    fill_u64<<<blocks_for(T0), 256, 0, st>>>(set0, T0, VEMPTY);
    if (reset_status()) return fail(set_error(BBS_ECUDA, "build_maps: status upload"));
    {
        unsigned long long init[6] = {~0ull, ~0ull, ~0ull, 0, 0, 0};
        TRYC(cudaMemcpyAsync(d_bbox, init, sizeof(init), cudaMemcpyHostToDevice, st));
    }
    if (n > 0) quantize_kernel<<<blocks_for(n), 256, 0, st>>>(d_xyz, n, rho, set0, (unsigned long long)(T0 - 1), d_st, d_bbox);
    TRYC(cudaGetLastError());
    if (read_status()) return fail(set_error(BBS_ECUDA, "build_maps: status read"));
    if (hs.bad) return fail(set_error(BBS_EINVAL, "build_maps: a map coordinate is not finite"));
    if (hs.keyrange) return fail(set_error(BBS_EKEYRANGE, "build_maps: a fine key exceeds 2^20 - 4 voxels"));
    if (hs.overflow) return fail(set_error(BBS_ECORRUPT, "build_maps: key set overflow"));
    {
        unsigned long long bb[6];
        TRYC(cudaMemcpyAsync(bb, d_bbox, sizeof(bb), cudaMemcpyDeviceToHost, st));
        TRYC(cudaStreamSynchronize(st));
        for (int a = 0; a < 6; ++a) {
            unsigned long long u = bb[a];
            u = (u & 0x8000000000000000ull) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
            double d;
            std::memcpy(&d, &u, sizeof(d));
            if (a < 3) m->lo[a] = n > 0 ? d : 0.0;
            else m->hi[a - 3] = n > 0 ? d : 0.0;
        }
    }
    int64_t nb = (int64_t)hs.count;
    TRYC(cudaMallocAsync(&sc.p[3], sizeof(unsigned long long) * (size_t)(nb > 0 ? nb : 1), st));
    unsigned long long* keys = (unsigned long long*)sc.p[3];
    unsigned long long* d_cnt = &d_st->count;
    TRYC(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st));
    compact_set<<<blocks_for(T0), 256, 0, st>>>(set0, T0, keys, d_cnt);
    TRYC(cudaGetLastError());
    cudaFreeAsync(sc.p[2], st);
    sc.p[2] = nullptr;

    // ---- 2-4. levels -----------------------------------------------------
    for (int l = 0; l < levels; ++l) {
        if (l > 0 && nb > 0) {
            // B_l = unique(B_{l-1} >> 1)
            const int lT = log2_ceil((unsigned long long)(2 * (nb > 512 ? nb : 512)));
            const int64_t T = (int64_t)1 << lT;
            TRYC(cudaMallocAsync(&sc.p[4], sizeof(unsigned long long) * (size_t)T, st));
            unsigned long long* set = (unsigned long long*)sc.p[4];
            fill_u64<<<blocks_for(T), 256, 0, st>>>(set, T, VEMPTY);
            if (reset_status()) return fail(set_error(BBS_ECUDA, "build_maps: status upload"));
            halve_kernel<<<blocks_for(nb), 256, 0, st>>>(keys, nb, set, (unsigned long long)(T - 1), d_st);
            TRYC(cudaGetLastError());
            if (read_status()) return fail(set_error(BBS_ECUDA, "build_maps: status read"));
            if (hs.overflow) return fail(set_error(BBS_ECORRUPT, "build_maps: key set overflow at level %d", l));
            const int64_t nn = (int64_t)hs.count;
            TRYC(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), st));
            compact_set<<<blocks_for(T), 256, 0, st>>>(set, T, keys, d_cnt);   // nn <= nb: fits in place
            TRYC(cudaGetLastError());
            cudaFreeAsync(sc.p[4], st);
            sc.p[4] = nullptr;
            nb = nn;
        }
        const int dilate = !(l == 0 && (flags & BBS_LEAF_UNDILATED));
        const int ee = l > 0 ? exact_e : 0;                  // exact-bound widening above the leaves
        const int jlo = dilate ? -ee : 0, jhi = dilate ? 1 + ee : 0;
        // bounds of B_l (D_l extends one voxel lower when dilated)
        int kmin[3] = {0, 0, 0}, kmax[3] = {0, 0, 0};
        if (nb > 0) {
            BuildStatus z;
            std::memset(&z, 0, sizeof(z));
            for (int a = 0; a < 3; ++a) {
                z.kmin[a] = INT_MAX;
                z.kmax[a] = INT_MIN;
            }
            TRYC(cudaMemcpyAsync(d_st, &z, sizeof(z), cudaMemcpyHostToDevice, st));
            key_bounds_kernel<<<blocks_for(nb), 256, 0, st>>>(keys, nb, d_st);
            TRYC(cudaGetLastError());
            if (read_status()) return fail(set_error(BBS_ECUDA, "build_maps: status read"));
            for (int a = 0; a < 3; ++a) {
                kmin[a] = hs.kmin[a] - jhi;
                kmax[a] = hs.kmax[a] - jlo;
            }
        }
        // scatter D_l into a roomy temporary brick table, growing on overflow
        int lt = log2_ceil((unsigned long long)(4 * (nb > 256 ? nb : 256)));
        if (lt < 10) lt = 10;
        for (int attempt = 0;; ++attempt) {
            if (lt > 31) return fail(set_error(BBS_ENOMEM, "build_maps: brick table beyond 2^31 buckets"));
            const int64_t T = (int64_t)1 << lt;
            TRYC(cudaMallocAsync(&sc.p[5], sizeof(Brick) * (size_t)T, st));
            init_bricks<<<blocks_for(T), 256, 0, st>>>((Brick*)sc.p[5], T);
            if (reset_status()) return fail(set_error(BBS_ECUDA, "build_maps: status upload"));
            if (nb > 0)
                dilate_kernel<<<blocks_for(nb), 256, 0, st>>>(keys, nb, jlo, jhi, (Brick*)sc.p[5], (uint32_t)(32 - lt),
                                                             (uint32_t)(T - 1), d_st, (unsigned long long)(T / 2));
            TRYC(cudaGetLastError());
            if (read_status()) return fail(set_error(BBS_ECUDA, "build_maps: status read"));
            if (!hs.overflow) break;
            cudaFreeAsync(sc.p[5], st);
            sc.p[5] = nullptr;
            lt += 2;
        }
        const int64_t nbricks = (int64_t)hs.count;
        // the level's brick box: origin a multiple of 4 at least 4 below kmin
        int base[3];
        uint32_t rmax[3], nbk[3];
        for (int a = 0; a < 3; ++a) {
            base[a] = ((kmin[a] - 4) >> 2) * 4;
            rmax[a] = (uint32_t)(kmax[a] - base[a]);
            nbk[a] = (rmax[a] >> 2) + 1;
        }
        const int64_t nbox = (int64_t)nbk[0] * nbk[1] * nbk[2];
        // compact keys when the box fits 11 / 11 / 10 bits of bricks
        const bool fits = nbk[0] <= 2048u && nbk[1] <= 2048u && nbk[2] <= 1023u;
        // dense: every relative key below 2^20, so that a key offset clamped to
        // +-2^21 (a run far outside the map) still lands outside the box
        const bool short_axes = rmax[0] < (1u << 20) && rmax[1] < (1u << 20) && rmax[2] < (1u << 20);
        const bool box_ok = nb > 0 && short_axes && nbox < DENSE_MAX && nbox <= DENSE_RATIO * nbricks + DENSE_SLACK;
        const uint32_t ncell[3] = {rmax[0] + 2u, rmax[1] + 2u, rmax[2] + 2u};   // bytes: one empty key past rmax
        const int64_t cells = (int64_t)ncell[0] * ncell[1] * ncell[2];
        const bool bytes = box_ok && (g_layout == 0 || g_layout == 4) && cells < ((int64_t)1 << 31);
        const bool dense = box_ok && !bytes && (g_layout == 0 || g_layout == 3);
        const bool compact = !dense && !bytes && fits && g_layout != 1 && nb > 0;
        int lf = log2_ceil((unsigned long long)((double)(nbricks > 0 ? nbricks : 1) / g_load_target + 0.5));
        if (lf < 10) lf = 10;
        const int64_t TF = bytes ? cells : (dense ? nbox + 1 : (int64_t)1 << lf);   // dense: + the zero brick
        const size_t table_bytes = bytes ? (size_t)cells : sizeof(Brick) * (size_t)TF;
        TRYC(cudaMalloc((void**)&m->lv[l].slots, table_bytes));
        if (reset_status()) return fail(set_error(BBS_ECUDA, "build_maps: status upload"));
        if (bytes) {
            // dense bricks first (voxel count), then one byte per key of the box
            TRYC(cudaMallocAsync(&sc.p[6], sizeof(Brick) * (size_t)nbox, st));
            TRYC(cudaMemsetAsync(sc.p[6], 0, sizeof(Brick) * (size_t)nbox, st));
            relayout_dense_kernel<<<blocks_for((int64_t)1 << lt), 256, 0, st>>>(
                (Brick*)sc.p[5], (int64_t)1 << lt, (Brick*)sc.p[6], base[0] >> 2, base[1] >> 2, base[2] >> 2, nbk[1],
                nbk[2], d_st);
            bytes_fill_kernel<<<blocks_for(cells), 256, 0, st>>>((const Brick*)sc.p[6], nbk[0], nbk[1], nbk[2],
                                                                 (uint8_t*)m->lv[l].slots, ncell[0], ncell[1],
                                                                 ncell[2]);
        } else if (dense) {
            TRYC(cudaMemsetAsync(m->lv[l].slots, 0, sizeof(Brick) * (size_t)TF, st));
            relayout_dense_kernel<<<blocks_for((int64_t)1 << lt), 256, 0, st>>>(
                (Brick*)sc.p[5], (int64_t)1 << lt, m->lv[l].slots, base[0] >> 2, base[1] >> 2, base[2] >> 2, nbk[1],
                nbk[2], d_st);
        } else if (compact) {
            fill_u32<<<blocks_for(8 * TF), 256, 0, st>>>((uint32_t*)m->lv[l].slots, 8 * TF, CEMPTY);
            relayout_compact_kernel<<<blocks_for((int64_t)1 << lt), 256, 0, st>>>(
                (Brick*)sc.p[5], (int64_t)1 << lt, m->lv[l].slots, (uint32_t)(32 - lf), (uint32_t)(TF - 1), base[0] >> 2,
                base[1] >> 2, base[2] >> 2, d_st);
        } else {
            init_bricks<<<blocks_for(TF), 256, 0, st>>>(m->lv[l].slots, TF);
            relayout_kernel<<<blocks_for((int64_t)1 << lt), 256, 0, st>>>(
                (Brick*)sc.p[5], (int64_t)1 << lt, m->lv[l].slots, (uint32_t)(32 - lf), (uint32_t)(TF - 1), d_st);
        }
        TRYC(cudaGetLastError());
        m->lv[l].layout = bytes ? LAYOUT_BYTES : (dense ? LAYOUT_DENSE : (compact ? LAYOUT_COMPACT : LAYOUT_WIDE));
        for (int a = 0; a < 3; ++a) {
            m->lv[l].base[a] = base[a];
            m->lv[l].rmax[a] = rmax[a];
        }
        m->lv[l].nby = bytes ? ncell[1] : nbk[1];
        m->lv[l].nbz = bytes ? ncell[2] : nbk[2];
        m->lv[l].n_slots = TF;
        if (read_status()) return fail(set_error(BBS_ECUDA, "build_maps: status read"));
        cudaFreeAsync(sc.p[5], st);
        sc.p[5] = nullptr;
        if (sc.p[6]) {
            cudaFreeAsync(sc.p[6], st);
            sc.p[6] = nullptr;
        }
        m->lv[l].log2T = lf;
        m->lv[l].maxp = hs.maxp;
        m->lv[l].n_bricks = nbricks;
        m->lv[l].n_voxels = (int64_t)hs.voxels;
        m->lv[l].displaced = (int64_t)hs.displaced;
        m->arena_bytes += table_bytes;
    }
#undef TRYC
    *out = m;
    return BBS_OK;
}

int maps_keys(const bbs_maps* m, int level, int32_t* out, int64_t cap, int64_t* n)
{
    if (level < 0 || level >= m->levels) return set_error(BBS_EINVAL, "maps_keys: level %d", level);
    const int64_t nv = m->lv[level].n_voxels;
    *n = nv;
    if (cap < nv || (nv > 0 && !out)) return set_error(BBS_EINVAL, "maps_keys: capacity %lld < %lld", (long long)cap, (long long)nv);
    if (nv == 0) return BBS_OK;
    int32_t* d_out = nullptr;
    unsigned long long* d_n = nullptr;
    BBS_CUDA_TRY(cudaMalloc((void**)&d_out, sizeof(int32_t) * 3 * (size_t)nv));
    BBS_CUDA_TRY(cudaMalloc((void**)&d_n, sizeof(unsigned long long)));
    cudaMemset(d_n, 0, sizeof(unsigned long long));
    const LevelTable& t = m->lv[level];
    const int64_t T = t.n_slots;
    if (t.layout == LAYOUT_BYTES)
        bytes_keys_kernel<<<blocks_for(T), 256>>>(reinterpret_cast<const uint8_t*>(t.slots), t.rmax[0] + 2u, t.nby,
                                                  t.nbz, t.base[0], t.base[1], t.base[2], d_out, d_n, nv);
    else if (t.layout == LAYOUT_DENSE)
        dense_keys_kernel<<<blocks_for(T), 256>>>(t.slots, T, t.base[0] >> 2, t.base[1] >> 2, t.base[2] >> 2, t.nby,
                                                  t.nbz, d_out, d_n, nv);
    else if (t.layout == LAYOUT_COMPACT)
        compact_keys_kernel<<<blocks_for(T), 256>>>(t.slots, T, t.base[0] >> 2, t.base[1] >> 2, t.base[2] >> 2, d_out,
                                                    d_n, nv);
    else
        brick_keys_kernel<<<blocks_for(T), 256>>>(t.slots, T, d_out, d_n, nv);
    cudaError_t e = cudaGetLastError();
    unsigned long long got = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&got, d_n, sizeof(got), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, sizeof(int32_t) * 3 * (size_t)nv, cudaMemcpyDeviceToHost);
    cudaFree(d_out);
    cudaFree(d_n);
    if (e != cudaSuccess) return set_error(BBS_ECUDA, "maps_keys: %s", cudaGetErrorString(e));
    if ((int64_t)got != nv) return set_error(BBS_ECORRUPT, "maps_keys: %llu keys, expected %lld", got, (long long)nv);
    return BBS_OK;
}

}  // namespace bbs
