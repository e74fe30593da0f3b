// Slab decomposition along x (the domain decomposition with one ghost layer
// that the paper's runs use across GPUs, Sec. 2.4 and the scaling results of
// Sec. 3.6).  Each rank holds the sub-box of its slab of x planes plus one
// ghost plane on every side where a neighbour slab lies; the ghost planes are
// held (not updated) by the rank's steps and overwritten after every step by
// the neighbour's first or last owned plane.  A 7-point step needs nothing
// else, so every owned voxel gets exactly the update it gets in the whole box.
//
// This file holds the pieces of that scheme inside the library:
//  - sbg_slab_partition: x bounds (multiples of the block edge) that balance
//    the active blocks between the slabs;
//  - sbg_state_get_xplane / sbg_state_set_xplane: one x plane of a species
//    between the block layout and a dense [Nz][Ny] buffer (the exchanged
//    ghost layer).
// The exchange itself (who sends which plane where) is host logic above the
// ABI (slab.py), with the transport a communicator provides.
#include <algorithm>
#include <vector>

#include "sbg_internal.cuh"
#include "sbg_trace.cuh"

namespace sbg {

// one thread per (block, y, z) of the blocks whose x range holds plane x
template <typename T, int B, bool TO_STATE>
__global__ void k_xplane(T *__restrict__ val, const int4 *__restrict__ blocks, const uint64_t *__restrict__ bitmap,
                         int64_t begin, int64_t count, int x, int ny, int nz, T *__restrict__ plane) {
    constexpr int B3 = B * B * B;
    constexpr int W = (B3 + 63) / 64;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * B * B) return;
    const int64_t b = begin + t / (B * B);
    const int r = (int)(t % (B * B));
    const int4 bc = blocks[b];
    if (bc.x != x / B) return;
    const int ly = r % B, lz = r / B;
    const int gy = bc.y * B + ly, gz = bc.z * B + lz;
    if (gy >= ny || gz >= nz) return;
    const int l = (lz * B + ly) * B + (x - bc.x * B);
    const bool act = (bitmap[b * W + l / 64] >> (l % 64)) & 1ull;
    const int64_t slot = b * B3 + l;
    const int64_t pi = (int64_t)gz * ny + gy;
    if (TO_STATE) {
        if (act) val[slot] = plane[pi];
    } else {
        plane[pi] = act ? val[slot] : T(0);
    }
}

template <typename T>
static void launch_xplane(sbg_grid g, T *val, int geom, int x, T *plane, bool to_state, cudaStream_t s) {
    const int64_t begin = g->geom_begin[geom], count = g->geom_count[geom];
    const int ny = (int)g->dims[3 * geom + 1], nz = (int)g->dims[3 * geom + 2];
    const int B = g->B;
    const unsigned grid = (unsigned)((count * B * B + 255) / 256);
    if (count == 0) return;
    if (B == 8) {
        if (to_state) k_xplane<T, 8, true><<<grid, 256, 0, s>>>(val, g->blocks, g->bitmap, begin, count, x, ny, nz, plane);
        else k_xplane<T, 8, false><<<grid, 256, 0, s>>>(val, g->blocks, g->bitmap, begin, count, x, ny, nz, plane);
    } else {
        if (to_state) k_xplane<T, 4, true><<<grid, 256, 0, s>>>(val, g->blocks, g->bitmap, begin, count, x, ny, nz, plane);
        else k_xplane<T, 4, false><<<grid, 256, 0, s>>>(val, g->blocks, g->bitmap, begin, count, x, ny, nz, plane);
    }
}

static sbg_status xplane_io(sbg_grid g, sbg_state st, int32_t geom, int32_t species, int64_t x, void *plane,
                            int32_t plane_dtype, int32_t on_device, bool to_state, void *stream) {
    const char *who = to_state ? "sbg_state_set_xplane" : "sbg_state_get_xplane";
    if (!g || !st || !plane) return fail(SBG_ERR_INVALID_ARG, std::string(who) + ": null pointer");
    if (st->grid != g) return fail(SBG_ERR_INVALID_ARG, std::string(who) + ": state of another grid");
    if (geom < 0 || geom >= g->n_geoms) return fail(SBG_ERR_INVALID_ARG, std::string(who) + ": bad geometry");
    if (species < 0 || species >= st->ns) return fail(SBG_ERR_INVALID_ARG, std::string(who) + ": bad species");
    if (x < 0 || x >= g->dims[3 * geom]) return fail(SBG_ERR_INVALID_ARG, std::string(who) + ": x outside the box");
    if (st->dtype != SBG_F32 && st->dtype != SBG_F64)
        return fail(SBG_ERR_INVALID_ARG, std::string(who) + ": SBG_F32 or SBG_F64 states only");
    const int want = st->dtype == SBG_F64 ? SBG_F64 : SBG_F32;
    if (plane_dtype != want)
        return fail(SBG_ERR_INVALID_ARG, std::string(who) + ": the plane's dtype must be the state's");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)g->dims[3 * geom + 1] * (size_t)g->dims[3 * geom + 2] * st->elem();
    void *dplane = plane;
    if (!on_device) {
        SBG_CUDA(dmalloc_async(&dplane, bytes, s));
        if (to_state) {
            cudaError_t e = cudaMemcpyAsync(dplane, plane, bytes, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                dfree_async(dplane, s);
                return cuda_fail(e, who);
            }
        }
    }
    if (st->dtype == SBG_F64)
        launch_xplane<double>(g, (double *)st->val[st->cur][species], geom, (int)x, (double *)dplane, to_state, s);
    else
        launch_xplane<float>(g, (float *)st->val[st->cur][species], geom, (int)x, (float *)dplane, to_state, s);
    cudaError_t e = cudaGetLastError();
    if (!on_device) {
        if (e == cudaSuccess && !to_state) e = cudaMemcpyAsync(plane, dplane, bytes, cudaMemcpyDeviceToHost, s);
        dfree_async(dplane, s);
        cudaError_t se = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = se;
    }
    if (e != cudaSuccess) return cuda_fail(e, who);
    return SBG_OK;
}

}  // namespace sbg

using namespace sbg;

extern "C" sbg_status sbg_slab_partition(const float *phi, const int64_t dims[3], int32_t block, float eps_mask,
                                         int32_t nparts, int64_t *x_bounds) {
    if (!phi || !dims || !x_bounds) return fail(SBG_ERR_INVALID_ARG, "sbg_slab_partition: null pointer");
    if (block != 4 && block != 8) return fail(SBG_ERR_INVALID_ARG, "sbg_slab_partition: block must be 4 or 8");
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    if (nx < 1 || ny < 1 || nz < 1) return fail(SBG_ERR_INVALID_ARG, "sbg_slab_partition: dims >= 1");
    const int64_t nbx = (nx + block - 1) / block;
    if (nparts < 1 || nparts > nbx)
        return fail(SBG_ERR_INVALID_ARG, "sbg_slab_partition: 1 <= nparts <= number of block columns along x");
    const float eps = eps_mask > 0.f ? eps_mask : 1.1920928955078125e-7f;
    const int64_t nby = (ny + block - 1) / block, nbz = (nz + block - 1) / block;
    // active blocks per block column along x
    std::vector<int64_t> col(nbx, 0);
    std::vector<unsigned char> act((size_t)(nby * nbz));
    for (int64_t bx = 0; bx < nbx; ++bx) {
        std::fill(act.begin(), act.end(), 0);
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = bx * block; x < std::min(nx, (bx + 1) * block); ++x)
                    if (phi[(z * ny + y) * nx + x] > eps) act[(size_t)((z / block) * nby + y / block)] = 1;
        for (unsigned char a : act) col[bx] += a;
    }
    // cut k (k = 1 .. nparts - 1) after the first block column e at which the running
    // count reaches k / nparts of the total, each slab keeping at least one column
    std::vector<int64_t> pre(nbx + 1, 0);
    for (int64_t c = 0; c < nbx; ++c) pre[c + 1] = pre[c] + col[c];
    const int64_t total = pre[nbx];
    x_bounds[0] = 0;
    int64_t prev = 0;
    for (int32_t k = 1; k < nparts; ++k) {
        int64_t e = prev + 1;
        while (e < nbx && (double)pre[e] * nparts < (double)total * k) ++e;
        e = std::min<int64_t>(std::max<int64_t>(e, prev + 1), nbx - (nparts - k));
        x_bounds[k] = e * block;
        prev = e;
    }
    x_bounds[nparts] = nx;
    return SBG_OK;
}

extern "C" sbg_status sbg_state_get_xplane(sbg_grid g, sbg_state st, int32_t geom, int32_t species, int64_t x,
                                           void *plane, int32_t plane_dtype, int32_t on_device, void *stream) {
    TraceRange trace_range("sbg_state_get_xplane");
    return xplane_io(g, st, geom, species, x, plane, plane_dtype, on_device, false, stream);
}

extern "C" sbg_status sbg_state_set_xplane(sbg_grid g, sbg_state st, int32_t geom, int32_t species, int64_t x,
                                           const void *plane, int32_t plane_dtype, int32_t on_device, void *stream) {
    TraceRange trace_range("sbg_state_set_xplane");
    return xplane_io(g, st, geom, species, x, const_cast<void *>(plane), plane_dtype, on_device, true, stream);
}
