// Per-voxel diffusivity factor for inhomogeneous diffusion: the factor eps of
// Eq. 6 (D_smooth as a function of phi), stored in block layout beside the
// grid so that the step reads it with the state (the paper's functor reads
// the diffusion coefficient at the centre and its six neighbours, Appendix B
// Listing 6).  Inactive voxels hold 0, a finite value: their faces carry no
// flux because the no-flux rule zeroes the difference of u across them.
#include <math.h>

#include <cstring>
#include <string>

#include "sbg_internal.cuh"
#include "sbg_trace.cuh"

namespace sbg {

// One thread per voxel slot of geometry `geom`'s blocks: from a dense array
// (MODE 0) or from phi by Eq. 6 (MODE 1).  Writes both copies and folds the
// largest value (FP32 bits of a non-negative float order like integers) and
// a flag for negative or non-finite values into `stat` ([0]: max bits, [1]: bad).
template <typename Tin, int MODE, int B>
__global__ void k_set_eps(const Tin *__restrict__ dense, int nx, int ny, int nz, const int4 *__restrict__ blocks,
                          const uint64_t *__restrict__ bitmap, int64_t begin, int64_t count, double d_min,
                          double d_max, double g1, double g2, float *__restrict__ eps,
                          double *__restrict__ eps64, unsigned int *stat) {
    constexpr int B3 = B * B * B;
    constexpr int W = (B3 + 63) / 64;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * B3) return;
    const int64_t b = begin + t / B3;
    const int l = (int)(t % B3);
    const int64_t slot = b * B3 + l;
    const bool act = (bitmap[b * W + l / 64] >> (l % 64)) & 1ull;
    if (!act) {
        eps[slot] = 0.f;
        eps64[slot] = 0.0;
        return;
    }
    const int4 bc = blocks[b];
    const int x = bc.x * B + l % B, y = bc.y * B + (l / B) % B, z = bc.z * B + l / (B * B);
    const double v0 = (double)dense[((int64_t)z * ny + y) * nx + x];
    const double v = MODE == 0 ? v0 : d_min + d_max / (1.0 + exp(-(g1 + g2 * v0)));
    if (!(v >= 0.0) || !isfinite(v)) {
        atomicOr(&stat[1], 1u);
        eps[slot] = 0.f;
        eps64[slot] = 0.0;
        return;
    }
    const float f = (float)v;
    eps[slot] = f;
    eps64[slot] = v;
    atomicMax(&stat[0], __float_as_uint(f));
}

static sbg_status set_eps(sbg_grid g, int geom, const void *dense, int dense_dtype, int on_device, int mode,
                          double d_min, double d_max, double g1, double g2, cudaStream_t s) {
    if (!g || !dense) return fail(SBG_ERR_INVALID_ARG, "diffusivity factor: null pointer");
    if (geom < 0 || geom >= g->n_geoms) return fail(SBG_ERR_INVALID_ARG, "diffusivity factor: bad geometry");
    if (dense_dtype != SBG_F32 && dense_dtype != SBG_F64)
        return fail(SBG_ERR_INVALID_ARG, "diffusivity factor: dense dtype must be SBG_F32 or SBG_F64");
    const int64_t slots = g->nb * g->b3();
    if (!g->eps) {
        // the FP32 factor is preceded by a ghost block of zeros (block id -1, the factor of an absent
        // neighbour block for the streaming kernel; any finite value gives the same result there)
        float *base = nullptr;
        cudaError_t e = dmalloc((void **)&base, sizeof(float) * (64 + (slots > 0 ? slots : 1)));
        if (e == cudaSuccess) g->eps = base + 64;
        if (e == cudaSuccess) e = dmalloc((void **)&g->eps64, sizeof(double) * (slots > 0 ? slots : 1));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (diffusivity factor)");
        g->bytes += (int64_t)(12 * slots + 256);
        SBG_CUDA(cudaMemsetAsync(base, 0, sizeof(float) * (64 + (slots > 0 ? slots : 1)), s));
        SBG_CUDA(cudaMemsetAsync(g->eps64, 0, sizeof(double) * (slots > 0 ? slots : 1), s));
    }
    const int64_t nx = g->dims[3 * geom], ny = g->dims[3 * geom + 1], nz = g->dims[3 * geom + 2];
    const int64_t begin = g->geom_begin[geom], count = g->geom_count[geom];
    const size_t ebytes = dense_dtype == SBG_F64 ? 8 : 4;
    const size_t bytes = (size_t)(nx * ny * nz) * ebytes;
    void *d = const_cast<void *>(dense);
    unsigned int *stat = nullptr;
    {
        // on failure, free what this call allocated before returning
        cudaError_t e = cudaSuccess;
        if (!on_device) {
            e = dmalloc_async((void **)&d, bytes, s);
            if (e != cudaSuccess) d = nullptr;
            if (e == cudaSuccess) e = cudaMemcpyAsync(d, dense, bytes, cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess) e = dmalloc_async((void **)(void **)&stat, 2 * sizeof(unsigned int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(stat, 0, 2 * sizeof(unsigned int), s);
        if (e != cudaSuccess) {
            if (!on_device && d) dfree_async(d, s);
            if (stat) dfree_async(stat, s);
            cudaStreamSynchronize(s);
            return cuda_fail(e, "staging buffers");
        }
    }
    if (count > 0) {
        const unsigned grid = (unsigned)((count * g->b3() + 255) / 256);
#define EPS_LAUNCH(TIN, MODE_, B_)                                                                          \
    k_set_eps<TIN, MODE_, B_><<<grid, 256, 0, s>>>((const TIN *)d, (int)nx, (int)ny, (int)nz, g->blocks,      \
                                                   g->bitmap, begin, count, d_min, d_max, g1, g2, g->eps,   \
                                                   g->eps64, stat)
        const bool f64 = dense_dtype == SBG_F64;
        if (g->B == 8) {
            if (mode == 0) { if (f64) EPS_LAUNCH(double, 0, 8); else EPS_LAUNCH(float, 0, 8); }
            else EPS_LAUNCH(float, 1, 8);
        } else {
            if (mode == 0) { if (f64) EPS_LAUNCH(double, 0, 4); else EPS_LAUNCH(float, 0, 4); }
            else EPS_LAUNCH(float, 1, 4);
        }
#undef EPS_LAUNCH
    }
    cudaError_t le = cudaGetLastError();
    unsigned int host[2] = {0u, 0u};
    cudaError_t ce = cudaMemcpyAsync(host, stat, sizeof(host), cudaMemcpyDeviceToHost, s);
    dfree_async(stat, s);
    if (!on_device) dfree_async(d, s);
    cudaError_t se = cudaStreamSynchronize(s);
    if (le != cudaSuccess) return cuda_fail(le, "diffusivity factor kernel launch");
    if (ce != cudaSuccess) return cuda_fail(ce, "diffusivity factor statistics copy");
    if (se != cudaSuccess) return cuda_fail(se, "diffusivity factor");
    if (host[1]) {
        g->has_eps = false;
        g->eps_max = 0.f;
        ++g->eps_version;
        return fail(SBG_ERR_INVALID_ARG, "diffusivity factor: negative or non-finite value on an active voxel");
    }
    float m;
    std::memcpy(&m, &host[0], sizeof(m));
    if (!g->has_eps || m > g->eps_max) g->eps_max = m;
    g->has_eps = true;
    ++g->eps_version;
    return SBG_OK;
}

}  // namespace sbg

using namespace sbg;

extern "C" sbg_status sbg_grid_set_diffusivity(sbg_grid g, int32_t geom, const void *dense, int32_t dense_dtype,
                                               int32_t on_device, void *stream) {
    TraceRange trace_range("sbg_grid_set_diffusivity");
    return set_eps(g, geom, dense, dense_dtype, on_device, 0, 0.0, 0.0, 0.0, 0.0, (cudaStream_t)stream);
}

extern "C" sbg_status sbg_grid_set_diffusivity_sigmoid(sbg_grid g, int32_t geom, const float *phi,
                                                       int32_t phi_on_device, double d_min, double d_max,
                                                       double gamma1, double gamma2, void *stream) {
    TraceRange trace_range("sbg_grid_set_diffusivity_sigmoid");
    if (!(d_min >= 0.0) || !(d_max >= 0.0) || !isfinite(d_min) || !isfinite(d_max) || !isfinite(gamma1) ||
        !isfinite(gamma2))
        return fail(SBG_ERR_INVALID_ARG, "sbg_grid_set_diffusivity_sigmoid: d_min, d_max >= 0 and finite parameters");
    return set_eps(g, geom, phi, SBG_F32, phi_on_device, 1, d_min, d_max, gamma1, gamma2, (cudaStream_t)stream);
}

extern "C" sbg_status sbg_grid_clear_diffusivity(sbg_grid g) {
    if (!g) return fail(SBG_ERR_INVALID_ARG, "sbg_grid_clear_diffusivity: null grid");
    g->has_eps = false;
    g->eps_max = 0.f;
    ++g->eps_version;
    return SBG_OK;
}
