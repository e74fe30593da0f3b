// External space-time source of the reaction term (Eq. 1 with f depending on
// x and t): f_s(x, t_n) = a_n S_s(x), the spatial part S_s stored per slot
// beside the state and one factor a_n per step.  This is the hook the
// method of manufactured solutions needs (Sec. 3.1 and the appendix's
// manufactured source, whose time dependence is the factor exp(-B t)).
#include <math.h>

#include <string>

#include "sbg_internal.cuh"
#include "sbg_trace.cuh"

namespace sbg {

// One thread per slot of geometry `geom`'s blocks; inactive voxels hold 0.
template <typename Tin, typename Tst, int B>
__global__ void k_set_source(const Tin *__restrict__ dense, int nx, int ny, int nz, const int4 *__restrict__ blocks,
                             const uint64_t *__restrict__ bitmap, int64_t begin, int64_t count,
                             Tst *__restrict__ out, unsigned int *bad) {
    constexpr int B3 = B * B * B;
    constexpr int W = (B3 + 63) / 64;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * B3) return;
    const int64_t b = begin + t / B3;
    const int l = (int)(t % B3);
    const int64_t slot = b * B3 + l;
    const bool act = (bitmap[b * W + l / 64] >> (l % 64)) & 1ull;
    if (!act) {
        out[slot] = Tst(0);
        return;
    }
    const int4 bc = blocks[b];
    const int x = bc.x * B + l % B, y = bc.y * B + (l / B) % B, z = bc.z * B + l / (B * B);
    const double v = (double)dense[((int64_t)z * ny + y) * nx + x];
    if (!isfinite(v)) {
        atomicOr(bad, 1u);
        out[slot] = Tst(0);
        return;
    }
    out[slot] = (Tst)v;
}

}  // namespace sbg

using namespace sbg;

extern "C" sbg_status sbg_state_set_source(sbg_grid g, sbg_state st, int32_t geom, int32_t species,
                                           const void *dense, int32_t dense_dtype, int32_t on_device, void *stream) {
    TraceRange trace_range("sbg_state_set_source");
    if (!g || !st || !dense) return fail(SBG_ERR_INVALID_ARG, "sbg_state_set_source: null pointer");
    if (st->grid != g) return fail(SBG_ERR_INVALID_ARG, "sbg_state_set_source: state of another grid");
    if (geom < 0 || geom >= g->n_geoms) return fail(SBG_ERR_INVALID_ARG, "sbg_state_set_source: bad geometry");
    if (species < 0 || species >= st->ns) return fail(SBG_ERR_INVALID_ARG, "sbg_state_set_source: bad species");
    if (st->dtype != SBG_F32 && st->dtype != SBG_F64)
        return fail(SBG_ERR_INVALID_ARG, "sbg_state_set_source: SBG_F32 or SBG_F64 states only");
    if (dense_dtype != SBG_F32 && dense_dtype != SBG_F64)
        return fail(SBG_ERR_INVALID_ARG, "sbg_state_set_source: dense dtype must be SBG_F32 or SBG_F64");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t elem = st->elem();
    const int64_t slots = st->nslots > 0 ? st->nslots : 1;
    if (!st->ext[species]) {
        cudaError_t e = dmalloc((void **)&st->ext[species], elem * (size_t)slots);
        if (e != cudaSuccess) {
            st->ext[species] = nullptr;
            return cuda_fail(e, "cudaMalloc (external source)");
        }
        st->bytes += (int64_t)(elem * (size_t)slots);
        SBG_CUDA(cudaMemsetAsync(st->ext[species], 0, elem * (size_t)slots, s));
    }
    const int64_t nx = g->dims[3 * geom], ny = g->dims[3 * geom + 1], nz = g->dims[3 * geom + 2];
    const int64_t begin = g->geom_begin[geom], count = g->geom_count[geom];
    const size_t bytes = (size_t)(nx * ny * nz) * (dense_dtype == SBG_F64 ? 8 : 4);
    void *d = const_cast<void *>(dense);
    unsigned int *bad = nullptr;
    {
        // on failure, free what this call allocated before returning
        cudaError_t e = cudaSuccess;
        if (!on_device) {
            e = dmalloc_async((void **)&d, bytes, s);
            if (e != cudaSuccess) d = nullptr;
            if (e == cudaSuccess) e = cudaMemcpyAsync(d, dense, bytes, cudaMemcpyHostToDevice, s);
        }
        if (e == cudaSuccess) e = dmalloc_async((void **)(void **)&bad, sizeof(unsigned int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(unsigned int), s);
        if (e != cudaSuccess) {
            if (!on_device && d) dfree_async(d, s);
            if (bad) dfree_async(bad, s);
            cudaStreamSynchronize(s);
            return cuda_fail(e, "staging buffers");
        }
    }
    if (count > 0) {
        const unsigned grid = (unsigned)((count * g->b3() + 255) / 256);
#define SRC_LAUNCH(TIN, TST)                                                                                 \
    do {                                                                                                     \
        if (g->B == 8)                                                                                       \
            k_set_source<TIN, TST, 8><<<grid, 256, 0, s>>>((const TIN *)d, (int)nx, (int)ny, (int)nz,        \
                                                           g->blocks, g->bitmap, begin, count,               \
                                                           (TST *)st->ext[species], bad);                    \
        else                                                                                                 \
            k_set_source<TIN, TST, 4><<<grid, 256, 0, s>>>((const TIN *)d, (int)nx, (int)ny, (int)nz,        \
                                                           g->blocks, g->bitmap, begin, count,               \
                                                           (TST *)st->ext[species], bad);                    \
    } while (0)
        const bool in64 = dense_dtype == SBG_F64;
        if (st->dtype == SBG_F64) {
            if (in64) SRC_LAUNCH(double, double);
            else SRC_LAUNCH(float, double);
        } else {
            if (in64) SRC_LAUNCH(double, float);
            else SRC_LAUNCH(float, float);
        }
#undef SRC_LAUNCH
    }
    cudaError_t le = cudaGetLastError();
    unsigned int host_bad = 0;
    cudaError_t ce = cudaMemcpyAsync(&host_bad, bad, sizeof(host_bad), cudaMemcpyDeviceToHost, s);
    dfree_async(bad, s);
    if (!on_device) dfree_async(d, s);
    cudaError_t se = cudaStreamSynchronize(s);
    if (le != cudaSuccess) return cuda_fail(le, "external source kernel launch");
    if (ce != cudaSuccess) return cuda_fail(ce, "external source flag copy");
    if (se != cudaSuccess) return cuda_fail(se, "sbg_state_set_source");
    if (host_bad) return fail(SBG_ERR_INVALID_ARG, "sbg_state_set_source: non-finite value on an active voxel");
    return SBG_OK;
}

extern "C" sbg_status sbg_state_clear_source(sbg_state st) {
    if (!st) return fail(SBG_ERR_INVALID_ARG, "sbg_state_clear_source: null state");
    for (int s = 0; s < 2; ++s) {
        if (st->ext[s]) {
            dfree(st->ext[s]);
            st->bytes -= (int64_t)(st->elem() * (size_t)(st->nslots > 0 ? st->nslots : 1));
            st->ext[s] = nullptr;
        }
    }
    return SBG_OK;
}

extern "C" sbg_status sbg_step_source(sbg_grid g, sbg_state st, const sbg_params *p, int64_t nsteps,
                                      const double *factors, void *stream) {
    TraceRange trace_range("sbg_step_source");
    if (!g || !st || !p) return fail(SBG_ERR_INVALID_ARG, "sbg_step_source: null pointer");
    if (st->grid != g) return fail(SBG_ERR_INVALID_ARG, "sbg_step_source: state of another grid");
    if (nsteps < 0) return fail(SBG_ERR_INVALID_ARG, "sbg_step_source: nsteps < 0");
    if (nsteps > 0 && !factors) return fail(SBG_ERR_INVALID_ARG, "sbg_step_source: null factors");
    if (st->dtype != SBG_F32 && st->dtype != SBG_F64)
        return fail(SBG_ERR_INVALID_ARG, "sbg_step_source: SBG_F32 or SBG_F64 states only");
    if (g->has_eps)
        return fail(SBG_ERR_INVALID_ARG, "sbg_step_source: not with a diffusivity factor");
    for (int64_t n = 0; n < nsteps; ++n)
        if (!isfinite(factors[n])) return fail(SBG_ERR_INVALID_ARG, "sbg_step_source: non-finite factor");
    sbg_status rc = validate_params(g, p, st->ns);
    if (rc != SBG_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    rc = prepare_held_bits(g, p, s);
    if (rc != SBG_OK) return rc;
    for (int64_t n = 0; n < nsteps; ++n) {
        rc = launch_step_ext(g, st, p, st->cur, factors[n], s);
        if (rc != SBG_OK) return rc;
        st->cur = 1 - st->cur;
    }
    return SBG_OK;
}
