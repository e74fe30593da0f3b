// Grid construction: block activation from phi, compaction, device block
// hash, 26-neighbour table, occupancy bitmaps and surface-weight slabs.
//
// The paper stores 8^3 chunks that hold at least one inserted point, with the
// chunk position and an allocation mask cached per chunk (Sec. 2.4), and
// inserts a point iff phi > lower bound + eps (Appendix B, Listing 5).  This
// file builds the same information for B^3 blocks (B = 4 or 8) directly on
// the device: one warp scans each box block of phi, an exclusive scan
// compacts the active ones in tiled block order, an open-addressing hash
// maps block coordinates to ids, and the neighbour table is resolved once so
// that the time step never probes the hash.  Blocks are listed tile by tile
// (see BlockEnum) so that face neighbours are close in the list.
#include <math.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "sbg_internal.cuh"
#include "sbg_trace.cuh"

namespace sbg {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }
sbg_status fail(sbg_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}
sbg_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SBG_ERR_OOM : SBG_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// exclusive scan of int32 counts (flag = count > 0 when `as_flags`)
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int scan_block_exclusive(int v, int *smem_warp, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) smem_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int s = (lane < (int)(blockDim.x >> 5)) ? smem_warp[lane] : 0;
        int si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        smem_warp[lane] = si - s;  // exclusive warp offsets
        if (lane == 31) smem_warp[32] = si;
    }
    __syncthreads();
    total = smem_warp[32];
    int r = incl - v + smem_warp[warp];
    __syncthreads();
    return r;
}

__global__ void k_scan_tiles(const int32_t *in, int64_t n, bool as_flags, int32_t *out,
                             int32_t *tile_sums) {
    __shared__ int sw[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t k = base + i;
        int x = (k < n) ? in[k] : 0;
        if (as_flags) x = x > 0;
        v[i] = x;
        s += x;
    }
    int total;
    int off = scan_block_exclusive(s, sw, total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        int64_t k = base + i;
        if (k < n) out[k] = off;
        off += v[i];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_scan_sums(int32_t *sums, int64_t ntiles, int32_t *grand_total) {
    __shared__ int sw[33];
    int carry = 0;
    for (int64_t start = 0; start < ntiles; start += blockDim.x) {
        int64_t k = start + threadIdx.x;
        int v = (k < ntiles) ? sums[k] : 0;
        int total;
        int off = scan_block_exclusive(v, sw, total);
        if (k < ntiles) sums[k] = off + carry;
        carry += total;
    }
    if (threadIdx.x == 0) *grand_total = carry;
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *tile_sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const int add = tile_sums[blockIdx.x];
    for (int i = threadIdx.x; i < kScanTile; i += blockDim.x) {
        int64_t k = base + i;
        if (k < n) out[k] += add;
    }
}

// Exclusive scan of `in` (or of in > 0) into `out`; returns the total on the host.
static sbg_status exclusive_scan(const int32_t *in, int64_t n, bool as_flags, int32_t *out,
                                 int64_t *total, cudaStream_t st) {
    int64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (ntiles < 1) ntiles = 1;
    int32_t *tmp = nullptr;
    SBG_CUDA(dmalloc_async((void **)&tmp, sizeof(int32_t) * (ntiles + 1), st));
    k_scan_tiles<<<(unsigned)ntiles, kScanThreads, 0, st>>>(in, n, as_flags, out, tmp);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(tmp, ntiles, tmp + ntiles);
    k_scan_add<<<(unsigned)ntiles, 256, 0, st>>>(out, n, tmp);
    int32_t h = 0;
    SBG_CUDA(cudaMemcpyAsync(&h, tmp + ntiles, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SBG_CUDA(dfree_async(tmp, st));
    SBG_CUDA(cudaStreamSynchronize(st));
    *total = h;
    return SBG_OK;
}

// ---------------------------------------------------------------------------
// Block order.  Box blocks are enumerated tile by tile (tiles of tx x ty x tz
// blocks; tiles and the blocks inside a tile in x-fastest order), and the
// active ones are compacted in that order.
//  - SBG_ORDER_TILED: tiles of 32^3 voxels (T = 32 / B blocks per side).  All
//    six face neighbours of a block are close to it in the list, so a CTA that
//    walks a contiguous range of the list finds most halo values in L2 and
//    meets a neighbour block soon after reading its halo.
//  - SBG_ORDER_PLANES: one tile per plane of blocks (the whole x-y extent, one
//    block thick), i.e. plain x-fastest order.  CTAs that take the list's
//    groups in turn then sweep the box one plane of blocks after another: the
//    -z neighbours were read one sweep earlier and the +z ones are read one
//    sweep later, so both stay in L2.
struct BlockEnum {
    int nbx, nby, nbz, tx, ty, tz, ntx, nty, ntz;
    __host__ __device__ int64_t count() const { return (int64_t)ntx * nty * ntz * tx * ty * tz; }
    // enumeration index -> block coordinates; false when the slot is padding
    __host__ __device__ bool decode(int64_t k, int &bx, int &by, int &bz) const {
        const int64_t t3 = (int64_t)tx * ty * tz;
        const int64_t tile = k / t3;
        const int inner = (int)(k - tile * t3);
        const int ix = (int)(tile % ntx), iy = (int)((tile / ntx) % nty), iz = (int)(tile / ((int64_t)ntx * nty));
        bx = ix * tx + inner % tx;
        by = iy * ty + (inner / tx) % ty;
        bz = iz * tz + inner / (tx * ty);
        return bx < nbx && by < nby && bz < nbz;
    }
};
static BlockEnum make_enum(int64_t nx, int64_t ny, int64_t nz, int B, int order) {
    BlockEnum e;
    e.nbx = (int)((nx + B - 1) / B);
    e.nby = (int)((ny + B - 1) / B);
    e.nbz = (int)((nz + B - 1) / B);
    if (order == SBG_ORDER_PLANES) {
        e.tx = e.nbx;
        e.ty = e.nby;
        e.tz = 1;
    } else {
        e.tx = e.ty = e.tz = 32 / B;
    }
    e.ntx = (e.nbx + e.tx - 1) / e.tx;
    e.nty = (e.nby + e.ty - 1) / e.ty;
    e.ntz = (e.nbz + e.tz - 1) / e.tz;
    return e;
}

// block activation: one warp per enumerated box block counts voxels with phi > eps
template <int B>
__global__ void k_block_count(const float *__restrict__ phi, int nx, int ny, int nz, BlockEnum en,
                              int64_t nbox, float eps, int32_t *count) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nbox) return;
    int bx, by, bz;
    if (!en.decode(warp, bx, by, bz)) {
        if (lane == 0) count[warp] = 0;
        return;
    }
    int c = 0;
    for (int l = lane; l < B * B * B; l += 32) {
        int x = bx * B + l % B, y = by * B + (l / B) % B, z = bz * B + l / (B * B);
        if (x < nx && y < ny && z < nz) c += phi[((int64_t)z * ny + y) * nx + x] > eps;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) count[warp] = c;
}

__global__ void k_compact(const int32_t *count, const int32_t *pos, int64_t nbox, BlockEnum en, int geom,
                          int64_t offset, int4 *blocks) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nbox || count[k] == 0) return;
    int4 b;
    en.decode(k, b.x, b.y, b.z);
    b.w = geom;
    blocks[offset + pos[k]] = b;
}

// one warp per active block: occupancy bitmap (ballot), band flag
template <int B>
__global__ void k_block_fill(const float *__restrict__ phi, int nx, int ny, int nz,
                             const int4 *__restrict__ blocks, int64_t begin, int64_t count,
                             float eps, float band_eps, uint64_t *bitmap, int32_t *band,
                             int32_t *nact) {
    constexpr int B3 = B * B * B;
    constexpr int W = (B3 + 63) / 64;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= count) return;
    const int64_t b = begin + warp;
    const int4 bc = blocks[b];
    int c = 0, bandany = 0;
    uint32_t halfword[2 * W];
    for (int i = 0; i < 2 * W; ++i) halfword[i] = 0;
#pragma unroll
    for (int base = 0; base < B3; base += 32) {
        int l = base + lane;
        int x = bc.x * B + l % B, y = bc.y * B + (l / B) % B, z = bc.z * B + l / (B * B);
        bool act = false, inband = false;
        if (l < B3 && x < nx && y < ny && z < nz) {
            float p = phi[((int64_t)z * ny + y) * nx + x];
            act = p > eps;
            inband = act && p < band_eps;
        }
        uint32_t m = __ballot_sync(0xffffffffu, act);
        halfword[base / 32] = m;
        c += act;
        bandany |= __any_sync(0xffffffffu, inband);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if (lane == 0) {
        for (int wd = 0; wd < W; ++wd) {
            uint64_t lo = halfword[2 * wd], hi = halfword[2 * wd + 1];
            bitmap[b * W + wd] = lo | (hi << 32);
        }
        band[b] = bandany;
        nact[b] = c;
    }
}

template <int B>
__global__ void k_fill_w(const float *__restrict__ phi, int nx, int ny, int nz,
                         const int4 *__restrict__ blocks, int64_t begin, int64_t count,
                         const int32_t *__restrict__ wslab, float eps, double band_eps, float *w,
                         double *w64) {
    constexpr int B3 = B * B * B;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * B3) return;
    const int64_t b = begin + t / B3;
    const int l = (int)(t % B3);
    const int ws = wslab[b];
    if (ws < 0) return;
    const int4 bc = blocks[b];
    int x = bc.x * B + l % B, y = bc.y * B + (l / B) % B, z = bc.z * B + l / (B * B);
    double val = 0.0;
    if (x < nx && y < ny && z < nz) {
        float p = phi[((int64_t)z * ny + y) * nx + x];
        if (p > eps && (double)p < band_eps) {
            const double pi = 3.14159265358979323846;
            val = (1.0 + cos(pi * (double)p / band_eps)) / (2.0 * band_eps);
        }
    }
    w[(int64_t)ws * B3 + l] = (float)val;
    w64[(int64_t)ws * B3 + l] = val;
}

// wslab[b] = band[b] ? position among band blocks : -1
__global__ void k_select_slab(const int32_t *band, const int32_t *pos, int64_t nb, int32_t *ws) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nb) ws[i] = band[i] ? pos[i] : -1;
}

// Band rows of 4^3 blocks: a row (four x-consecutive voxels) is a band row iff
// one of its surface weights is non-zero.  count[b] = number of band rows.
__global__ void k_band_rows(const int32_t *__restrict__ wslab, const float *__restrict__ w, int64_t nb,
                            int32_t *count) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int ws = wslab[b];
    int c = 0;
    if (ws >= 0)
        for (int r = 0; r < 16; ++r) {
            const float *q = w + (int64_t)ws * 64 + r * 4;
            c += (q[0] != 0.f || q[1] != 0.f || q[2] != 0.f || q[3] != 0.f);
        }
    count[b] = c;
}

// wmeta[b] = (index of the block's first band row in wrow, mask of its band
// rows), wmeta[nb].x = the number of band rows; wrow = the rows' weights,
// copied bit for bit from the slabs.  One thread per (block, row).
__global__ void k_band_rows_fill(const int32_t *__restrict__ wslab, const float *__restrict__ w, int64_t nb,
                                 const int32_t *__restrict__ off, int2 *wmeta, float4 *wrow) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 16) return;
    const int64_t b = t >> 4;
    const int r = (int)(t & 15);
    const int ws = wslab[b];
    uint32_t mask = 0;
    if (ws >= 0)
        for (int q = 0; q < 16; ++q) {
            const float *p = w + (int64_t)ws * 64 + q * 4;
            if (p[0] != 0.f || p[1] != 0.f || p[2] != 0.f || p[3] != 0.f) mask |= 1u << q;
        }
    if (r == 0) {
        wmeta[b] = make_int2(off[b], (int)mask);
        if (b == nb - 1) wmeta[nb] = make_int2(off[b] + __popc(mask), 0);
    }
    if ((mask >> r) & 1u) {
        const float *p = w + (int64_t)ws * 64 + r * 4;
        wrow[off[b] + __popc(mask & ((1u << r) - 1u))] = make_float4(p[0], p[1], p[2], p[3]);
    }
}

// ---------------------------------------------------------------------------
// device hash: key = geometry, bz, by, bx packed in 16 bits each
__host__ __device__ __forceinline__ unsigned long long block_key(int bx, int by, int bz, int g) {
    return ((unsigned long long)(uint16_t)g << 48) | ((unsigned long long)(uint16_t)bz << 32) |
           ((unsigned long long)(uint16_t)by << 16) | (unsigned long long)(uint16_t)bx;
}
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
constexpr unsigned long long kEmpty = ~0ull;

__global__ void k_hash_insert(const int4 *blocks, int64_t nb, unsigned long long *keys,
                              int32_t *vals, int64_t cap) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb) return;
    int4 b = blocks[i];
    unsigned long long key = block_key(b.x, b.y, b.z, b.w);
    uint64_t h = mix64(key) & (uint64_t)(cap - 1);
    for (int64_t probe = 0; probe < cap; ++probe) {
        unsigned long long prev = atomicCAS(&keys[h], kEmpty, key);
        if (prev == kEmpty || prev == key) {
            vals[h] = (int32_t)i;
            return;
        }
        h = (h + 1) & (uint64_t)(cap - 1);
    }
}

__device__ __forceinline__ int32_t hash_find(const unsigned long long *keys, const int32_t *vals,
                                             int64_t cap, unsigned long long key) {
    uint64_t h = mix64(key) & (uint64_t)(cap - 1);
    for (int64_t probe = 0; probe < cap; ++probe) {
        unsigned long long k = keys[h];
        if (k == key) return vals[h];
        if (k == kEmpty) return -1;
        h = (h + 1) & (uint64_t)(cap - 1);
    }
    return -1;
}

__global__ void k_neighbours(const int4 *blocks, int64_t nb, const int32_t *gdims, int B,
                             const unsigned long long *keys, const int32_t *vals, int64_t cap,
                             int32_t *nbr, int32_t *face) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb * 26) return;
    const int64_t i = t / 26;
    const int k = (int)(t % 26);
    const int kk = k >= 13 ? k + 1 : k;
    const int dx = kk % 3 - 1, dy = (kk / 3) % 3 - 1, dz = kk / 9 - 1;
    const int4 b = blocks[i];
    const int nbx = (gdims[b.w * 4 + 0] + B - 1) / B, nby = (gdims[b.w * 4 + 1] + B - 1) / B,
              nbz = (gdims[b.w * 4 + 2] + B - 1) / B;
    const int x = b.x + dx, y = b.y + dy, z = b.z + dz;
    int32_t id = -1;
    if (x >= 0 && y >= 0 && z >= 0 && x < nbx && y < nby && z < nbz)
        id = hash_find(keys, vals, cap, block_key(x, y, z, b.w));
    nbr[i * 26 + k] = id;
    int f = -1;
    if (k == kNbrXm) f = 0;
    else if (k == kNbrXp) f = 1;
    else if (k == kNbrYm) f = 2;
    else if (k == kNbrYp) f = 3;
    else if (k == kNbrZm) f = 4;
    else if (k == kNbrZp) f = 5;
    if (f >= 0) face[i * 6 + f] = id;
}

// ---------------------------------------------------------------------------
static inline sbg_status cuda_ok(cudaError_t e, const char *what) {
    return e == cudaSuccess ? SBG_OK : cuda_fail(e, what);
}

template <typename T>
static sbg_status dalloc(sbg_grid g, T **p, size_t count) {
    size_t bytes = sizeof(T) * (count > 0 ? count : 1);
    cudaError_t e = dmalloc((void **)(void **)p, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (grid)");
    g->bytes += (int64_t)bytes;
    return SBG_OK;
}

static void grid_free(sbg_grid g) {
    if (!g) return;
    dfree(g->blocks);
    dfree(g->nbr);
    dfree(g->face_nbr);
    dfree(g->hkeys);
    dfree(g->hvals);
    dfree(g->bitmap);
    dfree(g->wslab);
    dfree(g->w);
    dfree(g->w64);
    dfree(g->gdims);
    dfree(g->partials);
    dfree(g->red_dev);
    hfree(g->red_host);
    dfree(g->err);
    dfree(g->pad);
    dfree(g->heldbits);
    dfree(g->eps ? g->eps - 64 : nullptr);  // the allocation starts with a ghost block
    dfree(g->eps64);
    dfree(g->wmeta);
    dfree(g->wrow);
    hfree(g->err_host);
    delete g;
}

template <int B>
static sbg_status build_impl(int32_t n, const float *const *phis, const int64_t *dims,
                             const sbg_build_opts *opts, cudaStream_t st, sbg_grid *out) {
    constexpr int B3 = B * B * B;
    sbg_grid g = new sbg_grid_s();
    g->B = B;
    g->n_geoms = n;
    g->eps_mask = opts->eps_mask > 0.f ? opts->eps_mask : 1.1920928955078125e-7f;
    g->band_eps = opts->band_eps > 0.f ? opts->band_eps : 1.0f;
    g->order = opts->order;
    g->dims.assign(dims, dims + 3 * (size_t)n);
    g->geom_nactive.assign(n, 0);
    g->geom_begin.assign(n, 0);
    g->geom_count.assign(n, 0);

    std::vector<float *> dphi(n, nullptr);
    std::vector<int32_t *> dcount(n, nullptr), dpos(n, nullptr);
    int32_t *band = nullptr, *nact = nullptr, *wpos = nullptr;
    sbg_status rc = SBG_OK;
    auto cleanup = [&]() {
        for (int i = 0; i < n; ++i) {
            if (!opts->phi_on_device) dfree(dphi[i]);
            dfree(dcount[i]);
            dfree(dpos[i]);
        }
        dfree(band);
        dfree(nact);
        dfree(wpos);
    };
#define TRY(x)                 \
    do {                       \
        rc = (x);              \
        if (rc != SBG_OK) {    \
            cleanup();         \
            grid_free(g);      \
            return rc;         \
        }                      \
    } while (0)
#define TRYC(call) TRY(cuda_ok((call), #call))

    // pass 1: per geometry, count active voxels per box block and scan
    int64_t total = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t nx = dims[3 * i], ny = dims[3 * i + 1], nz = dims[3 * i + 2];
        const int64_t nvox = nx * ny * nz;
        if (opts->phi_on_device) {
            dphi[i] = const_cast<float *>(phis[i]);
        } else {
            TRYC(dmalloc((void **)&dphi[i], sizeof(float) * nvox));
            TRYC(cudaMemcpyAsync(dphi[i], phis[i], sizeof(float) * nvox, cudaMemcpyHostToDevice, st));
        }
        const BlockEnum en = make_enum(nx, ny, nz, B, opts->order);
        const int64_t nbox = en.count();
        TRYC(dmalloc((void **)&dcount[i], sizeof(int32_t) * nbox));
        TRYC(dmalloc((void **)&dpos[i], sizeof(int32_t) * nbox));
        k_block_count<B><<<(unsigned)((nbox * 32 + 255) / 256), 256, 0, st>>>(
            dphi[i], (int)nx, (int)ny, (int)nz, en, nbox, g->eps_mask, dcount[i]);
        TRY(cuda_ok(cudaGetLastError(), "k_block_count"));
        int64_t nbg = 0;
        TRY(exclusive_scan(dcount[i], nbox, true, dpos[i], &nbg, st));
        g->geom_begin[i] = total;
        g->geom_count[i] = nbg;
        total += nbg;
    }
    g->nb = total;
    if (total > (int64_t)INT32_MAX / 32) TRY(fail(SBG_ERR_INVALID_ARG, "sbg_build: too many blocks"));

    // device arrays
    const int W = g->words();
    TRY(dalloc(g, &g->blocks, total));
    TRY(dalloc(g, &g->nbr, total * 26));
    TRY(dalloc(g, &g->face_nbr, total * 6));
    TRY(dalloc(g, &g->bitmap, total * W));
    TRY(dalloc(g, &g->wslab, total));
    TRY(dalloc(g, &g->gdims, 4 * (size_t)n));
    TRY(dalloc(g, &g->partials, (size_t)kRedMaxCtas * kNumRed));
    TRY(dalloc(g, &g->red_dev, (size_t)kNumRed));
    TRYC(hmalloc((void **)&g->red_host, sizeof(double) * kNumRed));
    TRY(dalloc(g, &g->err, 1));
    TRY(dalloc(g, &g->pad, 8));
    {
        const float hp[8] = {sentinel_f32(), sentinel_f32(), sentinel_f32(), sentinel_f32(), 0.f, 0.f, 0.f, 0.f};
        TRYC(cudaMemcpy(g->pad, hp, sizeof(hp), cudaMemcpyHostToDevice));
    }
    TRYC(cudaMemsetAsync(g->err, 0, sizeof(int), st));
    TRYC(hmalloc((void **)&g->err_host, sizeof(int)));
    TRYC(dmalloc((void **)&band, sizeof(int32_t) * std::max<int64_t>(total, 1)));
    TRYC(dmalloc((void **)&nact, sizeof(int32_t) * std::max<int64_t>(total, 1)));
    TRYC(dmalloc((void **)&wpos, sizeof(int32_t) * std::max<int64_t>(total, 1)));
    {
        std::vector<int32_t> hd(4 * (size_t)n, 0);
        for (int i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a) hd[4 * i + a] = (int32_t)dims[3 * i + a];
        TRYC(cudaMemcpyAsync(g->gdims, hd.data(), sizeof(int32_t) * hd.size(),
                             cudaMemcpyHostToDevice, st));
        TRYC(cudaStreamSynchronize(st));
    }

    // pass 2: compaction, bitmaps, band flags
    for (int i = 0; i < n; ++i) {
        const int64_t nx = dims[3 * i], ny = dims[3 * i + 1], nz = dims[3 * i + 2];
        const BlockEnum en = make_enum(nx, ny, nz, B, opts->order);
        const int64_t nbox = en.count();
        k_compact<<<(unsigned)((nbox + 255) / 256), 256, 0, st>>>(dcount[i], dpos[i], nbox, en, i,
                                                                 g->geom_begin[i], g->blocks);
        if (g->geom_count[i] > 0)
            k_block_fill<B><<<(unsigned)((g->geom_count[i] * 32 + 255) / 256), 256, 0, st>>>(
                dphi[i], (int)nx, (int)ny, (int)nz, g->blocks, g->geom_begin[i], g->geom_count[i],
                g->eps_mask, g->band_eps, g->bitmap, band, nact);
        TRY(cuda_ok(cudaGetLastError(), "k_block_fill"));
    }

    // active-voxel counts per geometry
    {
        std::vector<int32_t> hn(std::max<int64_t>(total, 1));
        if (total > 0)
            TRYC(cudaMemcpyAsync(hn.data(), nact, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, st));
        TRYC(cudaStreamSynchronize(st));
        for (int i = 0; i < n; ++i) {
            int64_t s = 0;
            for (int64_t b = g->geom_begin[i]; b < g->geom_begin[i] + g->geom_count[i]; ++b) s += hn[b];
            g->geom_nactive[i] = s;
            g->n_active += s;
        }
    }

    // surface-weight slabs for blocks that meet the band
    int64_t nband = 0;
    TRY(exclusive_scan(band, total, true, wpos, &nband, st));
    g->n_band = nband;
    TRY(dalloc(g, &g->w, (size_t)nband * B3));
    TRY(dalloc(g, &g->w64, (size_t)nband * B3));
    if (total > 0)
        k_select_slab<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(band, wpos, total, g->wslab);
    for (int i = 0; i < n; ++i) {
        if (g->geom_count[i] == 0) continue;
        const int64_t nx = dims[3 * i], ny = dims[3 * i + 1], nz = dims[3 * i + 2];
        k_fill_w<B><<<(unsigned)((g->geom_count[i] * B3 + 255) / 256), 256, 0, st>>>(
            dphi[i], (int)nx, (int)ny, (int)nz, g->blocks, g->geom_begin[i], g->geom_count[i],
            g->wslab, g->eps_mask, (double)g->band_eps, g->w, g->w64);
    }

    // band rows (4^3 blocks): the rows of four voxels that hold surface weight,
    // packed in list order, for the streaming step kernel
    if (B == 4) {
        TRY(dalloc(g, &g->wmeta, total + 1));
        TRYC(cudaMemsetAsync(g->wmeta, 0, sizeof(int2) * (total + 1), st));
        if (total > 0 && nband > 0) {
            int32_t *rcount = nullptr, *roff = nullptr;
            cudaError_t e1 = dmalloc_async((void **)&rcount, sizeof(int32_t) * total, st);
            cudaError_t e2 = dmalloc_async((void **)&roff, sizeof(int32_t) * total, st);
            int64_t nrows = 0;
            sbg_status r2 = (e1 == cudaSuccess && e2 == cudaSuccess) ? SBG_OK : cuda_fail(e1 != cudaSuccess ? e1 : e2, "cudaMallocAsync (band rows)");
            if (r2 == SBG_OK) {
                k_band_rows<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(g->wslab, g->w, total, rcount);
                r2 = exclusive_scan(rcount, total, false, roff, &nrows, st);
            }
            if (r2 == SBG_OK) {
                g->n_wrows = nrows;
                r2 = dalloc(g, &g->wrow, (size_t)nrows);
            }
            if (r2 == SBG_OK) {
                k_band_rows_fill<<<(unsigned)((total * 16 + 255) / 256), 256, 0, st>>>(g->wslab, g->w, total, roff,
                                                                                       g->wmeta, g->wrow);
                r2 = cuda_ok(cudaGetLastError(), "k_band_rows_fill");
            }
            dfree_async(rcount, st);
            dfree_async(roff, st);
            TRY(r2);
        }
    }

    // hash and neighbour table
    int64_t cap = 64;
    while (cap < 2 * std::max<int64_t>(total, 1)) cap <<= 1;
    g->hcap = cap;
    TRY(dalloc(g, &g->hkeys, cap));
    TRY(dalloc(g, &g->hvals, cap));
    TRYC(cudaMemsetAsync(g->hkeys, 0xff, sizeof(unsigned long long) * cap, st));
    if (total > 0) {
        k_hash_insert<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(g->blocks, total, g->hkeys,
                                                                       g->hvals, cap);
        k_neighbours<<<(unsigned)((total * 26 + 255) / 256), 256, 0, st>>>(
            g->blocks, total, g->gdims, B, g->hkeys, g->hvals, cap, g->nbr, g->face_nbr);
    }
    TRY(cuda_ok(cudaGetLastError(), "k_neighbours"));
    TRYC(cudaStreamSynchronize(st));
    cleanup();
    *out = g;
    return SBG_OK;
#undef TRY
#undef TRYC
}

static sbg_status check_build_args(int32_t n, const float *const *phis, const int64_t *dims,
                                   const sbg_build_opts *opts, sbg_grid *out) {
    if (!phis || !dims || !opts || !out || n < 1)
        return fail(SBG_ERR_INVALID_ARG, "sbg_build: null pointer or n < 1");
    if (opts->block != 4 && opts->block != 8)
        return fail(SBG_ERR_INVALID_ARG, "sbg_build: block must be 4 or 8");
    if (n > 65535) return fail(SBG_ERR_INVALID_ARG, "sbg_build: at most 65535 geometries");
    for (int i = 0; i < n; ++i) {
        if (!phis[i]) return fail(SBG_ERR_INVALID_ARG, "sbg_build: null phi");
        for (int a = 0; a < 3; ++a)
            if (dims[3 * i + a] < 1 || dims[3 * i + a] > 65535LL * opts->block)
                return fail(SBG_ERR_INVALID_ARG, "sbg_build: dims out of range");
        if (dims[3 * i] * dims[3 * i + 1] * dims[3 * i + 2] > (1LL << 40))
            return fail(SBG_ERR_INVALID_ARG, "sbg_build: box too large");
    }
    if (!(opts->eps_mask >= 0.f) || !(opts->band_eps >= 0.f))
        return fail(SBG_ERR_INVALID_ARG, "sbg_build: eps_mask and band_eps must be >= 0");
    if (opts->order != SBG_ORDER_TILED && opts->order != SBG_ORDER_PLANES)
        return fail(SBG_ERR_INVALID_ARG, "sbg_build: order must be SBG_ORDER_TILED or SBG_ORDER_PLANES");
    return SBG_OK;
}

}  // namespace sbg

using namespace sbg;

extern "C" sbg_status sbg_build_batch(int32_t n, const float *const *phis, const int64_t *dims,
                                      const sbg_build_opts *opts, void *stream, sbg_grid *out) {
    TraceRange trace_range("sbg_build_batch");
    sbg_status rc = check_build_args(n, phis, dims, opts, out);
    if (rc != SBG_OK) return rc;
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    return opts->block == 8 ? build_impl<8>(n, phis, dims, opts, st, out)
                            : build_impl<4>(n, phis, dims, opts, st, out);
}

extern "C" sbg_status sbg_build(const float *phi, const int64_t dims[3], const sbg_build_opts *opts,
                                void *stream, sbg_grid *out) {
    TraceRange trace_range("sbg_build");
    const float *phis[1] = {phi};
    return sbg_build_batch(1, phis, dims, opts, stream, out);
}

extern "C" sbg_status sbg_grid_info(sbg_grid g, sbg_grid_info_t *info) {
    if (!g || !info) return fail(SBG_ERR_INVALID_ARG, "sbg_grid_info: null pointer");
    std::memset(info, 0, sizeof(*info));
    for (int a = 0; a < 3; ++a) info->dims[a] = g->dims[a];
    info->block = g->B;
    info->n_geoms = g->n_geoms;
    info->n_blocks = g->nb;
    info->n_active = g->n_active;
    info->n_band_blocks = g->n_band;
    info->porosity = (double)g->geom_nactive[0] / (double)(g->dims[0] * g->dims[1] * g->dims[2]);
    info->device_bytes = g->bytes;
    return SBG_OK;
}

extern "C" sbg_status sbg_grid_geometry_info(sbg_grid g, int64_t *n_active, int64_t *block_begin,
                                             int64_t *block_count) {
    if (!g) return fail(SBG_ERR_INVALID_ARG, "sbg_grid_geometry_info: null grid");
    for (int i = 0; i < g->n_geoms; ++i) {
        if (n_active) n_active[i] = g->geom_nactive[i];
        if (block_begin) block_begin[i] = g->geom_begin[i];
        if (block_count) block_count[i] = g->geom_count[i];
    }
    return SBG_OK;
}

extern "C" sbg_status sbg_grid_tables(sbg_grid g, int32_t *nbr26, int32_t *blocks) {
    if (!g) return fail(SBG_ERR_INVALID_ARG, "sbg_grid_tables: null grid");
    if (g->nb == 0) return SBG_OK;
    if (nbr26) SBG_CUDA(cudaMemcpy(nbr26, g->nbr, sizeof(int32_t) * 26 * g->nb, cudaMemcpyDeviceToHost));
    if (blocks) SBG_CUDA(cudaMemcpy(blocks, g->blocks, sizeof(int4) * g->nb, cudaMemcpyDeviceToHost));
    return SBG_OK;
}

extern "C" void sbg_grid_destroy(sbg_grid g) { grid_free(g); }

extern "C" const char *sbg_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *sbg_status_string(sbg_status s) {
    switch (s) {
        case SBG_OK: return "ok";
        case SBG_ERR_INVALID_ARG: return "invalid argument";
        case SBG_ERR_OOM: return "out of memory";
        case SBG_ERR_CUDA: return "CUDA error";
        case SBG_ERR_UNSTABLE_DT: return "time step above the explicit stability limit";
        case SBG_ERR_NONFINITE: return "non-finite value in the state";
        case SBG_ERR_TIMEOUT: return "bounded device wait timed out";
        case SBG_ERR_NOT_CONVERGED: return "not converged";
        case SBG_ERR_BOUNDS: return "index outside its table (debug build)";
    }
    return "unknown status";
}

extern "C" int32_t sbg_abi_version(void) { return 2; }
