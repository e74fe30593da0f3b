// Species state in block layout: u[s][block * B^3 + (z*B + y)*B + x], two
// buffers (read one, write the other each step, like the two concentration
// properties of Appendix B Listing 7).  Inactive voxels of active blocks hold
// the NaN sentinel; the step kernel reads that as "outside Omega".
#include <math.h>

#include <cstring>
#include <vector>

#include "sbg_internal.cuh"
#include "sbg_trace.cuh"

namespace sbg {

// corr (SBG_F32R states): the correction array, set to 0 (active) or the sentinel
template <typename Tin, typename Tst, bool X2, int B>
__global__ void k_scatter(const Tin *__restrict__ dense, int nx, int ny, int nz,
                          const int4 *__restrict__ blocks, const uint64_t *__restrict__ bitmap,
                          int64_t begin, int64_t count, Tst *__restrict__ val, float *__restrict__ lo,
                          float *__restrict__ corr) {
    constexpr int B3 = B * B * B;
    constexpr int W = (B3 + 63) / 64;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * B3) return;
    const int64_t b = begin + t / B3;
    const int l = (int)(t % B3);
    const int4 bc = blocks[b];
    const bool act = (bitmap[b * W + l / 64] >> (l % 64)) & 1ull;
    const int64_t slot = b * B3 + l;
    if (!act) {
        val[slot] = sentinel<Tst>();
        if (X2) lo[slot] = 0.f;
        if (corr) corr[slot] = sentinel_f32();
        return;
    }
    if (corr) corr[slot] = 0.f;
    const int x = bc.x * B + l % B, y = bc.y * B + (l / B) % B, z = bc.z * B + l / (B * B);
    double v = (double)dense[((int64_t)z * ny + y) * nx + x];
    if (isnan(v)) v = __longlong_as_double(0x7fffffffffffffffll);  // canonical NaN, not the sentinel
    if (X2) {
        float h = (float)v;
        if (isnan(v)) h = __uint_as_float(0x7fffffffu);
        val[slot] = (Tst)h;
        lo[slot] = isfinite(v) ? (float)(v - (double)h) : 0.f;
    } else {
        Tst s = (Tst)v;
        if (isnan(v)) s = (Tst)__longlong_as_double(0x7fffffffffffffffll);
        val[slot] = s;
    }
}

// The same for FP32 input and an FP32-based state, one thread per x-row of
// four slots: one 16-byte load of the dense row (when the row lies inside the
// box and the dense array allows it) and 16-byte stores.  X2: also the low
// part (0 for FP32 input) and, with corr, the SBG_F32R correction.
template <bool X2, int B>
__global__ void k_scatter_rows(const float *__restrict__ dense, int nx, int ny, int nz,
                               const int4 *__restrict__ blocks, const uint64_t *__restrict__ bitmap, int64_t begin,
                               int64_t count, bool vec_ok, float *__restrict__ val, float *__restrict__ lo,
                               float *__restrict__ corr) {
    constexpr int B3 = B * B * B;
    constexpr int W = (B3 + 63) / 64;
    constexpr int RPB = B3 / 4;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * RPB) return;
    const int64_t b = begin + t / RPB;
    const int l0 = (int)(t % RPB) * 4;
    const uint32_t bits = (uint32_t)(bitmap[b * W + l0 / 64] >> (l0 % 64)) & 0xFu;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (bits) {
        const int4 bc = blocks[b];
        const int x = bc.x * B + l0 % B, y = bc.y * B + (l0 / B) % B, z = bc.z * B + l0 / (B * B);
        const int64_t di = ((int64_t)z * ny + y) * nx + x;
        if (vec_ok && x + 3 < nx) {
            const float4 q = *reinterpret_cast<const float4 *>(dense + di);
            v[0] = q.x;
            v[1] = q.y;
            v[2] = q.z;
            v[3] = q.w;
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((bits >> i) & 1u) v[i] = dense[di + i];  // active voxels lie inside the box
        }
    }
    const float SENT = sentinel_f32();
    float o[4], cr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool act = (bits >> i) & 1u;
        const float h = isnan(v[i]) ? __uint_as_float(0x7fffffffu) : v[i];  // canonical NaN, not the sentinel
        o[i] = act ? h : SENT;
        cr[i] = act ? 0.f : SENT;
    }
    const int64_t slot = b * B3 + l0;
    *reinterpret_cast<float4 *>(val + slot) = make_float4(o[0], o[1], o[2], o[3]);
    if (X2) *reinterpret_cast<float4 *>(lo + slot) = make_float4(0.f, 0.f, 0.f, 0.f);
    if (corr) *reinterpret_cast<float4 *>(corr + slot) = make_float4(cr[0], cr[1], cr[2], cr[3]);
}

template <typename Tout, typename Tst, bool X2, int B>
__global__ void k_gather(Tout *__restrict__ dense, int nx, int ny, int nz,
                         const int4 *__restrict__ blocks, int64_t begin, int64_t count,
                         const Tst *__restrict__ val, const float *__restrict__ lo,
                         const float *__restrict__ corr) {
    constexpr int B3 = B * B * B;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * B3) return;
    const int64_t b = begin + t / B3;
    const int l = (int)(t % B3);
    const int4 bc = blocks[b];
    const int x = bc.x * B + l % B, y = bc.y * B + (l / B) % B, z = bc.z * B + l / (B * B);
    if (x >= nx || y >= ny || z >= nz) return;
    const int64_t slot = b * B3 + l;
    Tst v = val[slot];
    if (is_sent(v)) return;  // dense output was zeroed
    double d = (double)v;
    if (X2) d += (double)lo[slot];
    if (corr) d += (double)corr[slot];
    dense[((int64_t)z * ny + y) * nx + x] = (Tout)d;
}

template <int B>
static sbg_status scatter_gather(sbg_grid g, sbg_state st, int geom, int species, void *ddense,
                                 int dense_dtype, bool to_state, cudaStream_t s) {
    const int64_t nx = g->dims[3 * geom], ny = g->dims[3 * geom + 1], nz = g->dims[3 * geom + 2];
    const int64_t begin = g->geom_begin[geom], count = g->geom_count[geom];
    if (count == 0) return SBG_OK;
    const unsigned grid = (unsigned)((count * B * B * B + 255) / 256);
    void *val = st->val[st->cur][species];
    float *lo = st->lo[st->cur][species];
    float *corr = nullptr;
    if (st->dtype == SBG_F32R) {  // the base pair takes the value, the correction is zeroed
        corr = (float *)val;
        val = st->bh;
        lo = st->bl;
        if (to_state) st->r_valid = false;
    }
#define SG_LAUNCH(TIN, TST, X2)                                                                   \
    do {                                                                                         \
        if (to_state)                                                                            \
            k_scatter<TIN, TST, X2, B><<<grid, 256, 0, s>>>((const TIN *)ddense, (int)nx, (int)ny, \
                                                          (int)nz, g->blocks, g->bitmap, begin,  \
                                                          count, (TST *)val, lo, corr);          \
        else                                                                                     \
            k_gather<TIN, TST, X2, B><<<grid, 256, 0, s>>>((TIN *)ddense, (int)nx, (int)ny,       \
                                                         (int)nz, g->blocks, begin, count,       \
                                                         (const TST *)val, lo, corr);            \
    } while (0)
    const bool in64 = dense_dtype == SBG_F64;
    if (to_state && !in64 && st->dtype != SBG_F64) {
        // FP32 input into an FP32-based state: the row kernel (16-byte loads where the dense
        // array's base and row length allow them)
        const bool vec_ok = (nx % 4 == 0) && ((reinterpret_cast<uintptr_t>(ddense) & 15) == 0);
        const unsigned rgrid = (unsigned)((count * (B * B * B / 4) + 255) / 256);
        if (st->dtype == SBG_F32)
            k_scatter_rows<false, B><<<rgrid, 256, 0, s>>>((const float *)ddense, (int)nx, (int)ny, (int)nz,
                                                           g->blocks, g->bitmap, begin, count, vec_ok,
                                                           (float *)val, lo, corr);
        else
            k_scatter_rows<true, B><<<rgrid, 256, 0, s>>>((const float *)ddense, (int)nx, (int)ny, (int)nz,
                                                          g->blocks, g->bitmap, begin, count, vec_ok,
                                                          (float *)val, lo, corr);
        SBG_LAUNCH_CHECK("state scatter");
        return SBG_OK;
    }
    if (st->dtype == SBG_F64) {
        if (in64) SG_LAUNCH(double, double, false);
        else SG_LAUNCH(float, double, false);
    } else if (st->dtype == SBG_F32) {
        if (in64) SG_LAUNCH(double, float, false);
        else SG_LAUNCH(float, float, false);
    } else {
        if (in64) SG_LAUNCH(double, float, true);
        else SG_LAUNCH(float, float, true);
    }
#undef SG_LAUNCH
    SBG_LAUNCH_CHECK("state scatter/gather");
    return SBG_OK;
}

static sbg_status dense_io(sbg_grid g, sbg_state st, int32_t geom, int32_t species, void *dense,
                           int32_t dense_dtype, int32_t on_device, bool to_state, void *stream) {
    if (!g || !st || !dense) return fail(SBG_ERR_INVALID_ARG, "sbg_state_set/get: null pointer");
    if (st->grid != g) return fail(SBG_ERR_INVALID_ARG, "sbg_state_set/get: state of another grid");
    if (geom < 0 || geom >= g->n_geoms) return fail(SBG_ERR_INVALID_ARG, "sbg_state_set/get: bad geometry");
    if (species < 0 || species >= st->ns) return fail(SBG_ERR_INVALID_ARG, "sbg_state_set/get: bad species");
    if (dense_dtype != SBG_F32 && dense_dtype != SBG_F64)
        return fail(SBG_ERR_INVALID_ARG, "sbg_state_set/get: dense dtype must be SBG_F32 or SBG_F64");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nvox = g->dims[3 * geom] * g->dims[3 * geom + 1] * g->dims[3 * geom + 2];
    const size_t bytes = (size_t)nvox * (dense_dtype == SBG_F64 ? 8 : 4);
    void *ddense = dense;
    if (!on_device) {
        SBG_CUDA(dmalloc_async((void **)&ddense, bytes, s));
        if (to_state) SBG_CUDA(cudaMemcpyAsync(ddense, dense, bytes, cudaMemcpyHostToDevice, s));
    }
    if (!to_state) SBG_CUDA(cudaMemsetAsync(ddense, 0, bytes, s));
    sbg_status rc = g->B == 8 ? scatter_gather<8>(g, st, geom, species, ddense, dense_dtype, to_state, s)
                              : scatter_gather<4>(g, st, geom, species, ddense, dense_dtype, to_state, s);
    if (!on_device) {
        if (rc == SBG_OK && !to_state)
            SBG_CUDA(cudaMemcpyAsync(dense, ddense, bytes, cudaMemcpyDeviceToHost, s));
        SBG_CUDA(dfree_async(ddense, s));
        SBG_CUDA(cudaStreamSynchronize(s));
    }
    return rc;
}

}  // namespace sbg

using namespace sbg;

extern "C" sbg_status sbg_state_create(sbg_grid g, int32_t nspecies, sbg_dtype dtype, sbg_state *out) {
    if (!g || !out) return fail(SBG_ERR_INVALID_ARG, "sbg_state_create: null pointer");
    if (nspecies < 1 || nspecies > 2) return fail(SBG_ERR_INVALID_ARG, "sbg_state_create: nspecies must be 1 or 2");
    if (dtype != SBG_F32 && dtype != SBG_F64 && dtype != SBG_F32X2 && dtype != SBG_F32R)
        return fail(SBG_ERR_INVALID_ARG, "sbg_state_create: bad dtype");
    if (dtype == SBG_F32R && nspecies != 1)
        return fail(SBG_ERR_INVALID_ARG, "sbg_state_create: SBG_F32R states hold one species");
    *out = nullptr;
    sbg_state st = new sbg_state_s();
    st->grid = g;
    st->ns = nspecies;
    st->dtype = dtype;
    st->nslots = g->nb * (int64_t)g->b3();
    const size_t per = (size_t)st->nslots * st->elem();
    // each species array is preceded by one ghost block of sentinels (block id -1, the id the
    // face table gives an absent neighbour), which the streaming step kernel reads for an absent
    // neighbour block; 256-byte multiples keep every array 256-byte aligned
    const size_t ghost = ((size_t)g->b3() * st->elem() + 255) / 256 * 256;
    const size_t perlo = dtype == SBG_F32X2 ? (size_t)st->nslots * 4 : 0;
    const size_t extra = dtype == SBG_F32R ? 3 * (size_t)st->nslots * 4 : 0;  // base hi, lo and source
    const size_t total = 2 * (size_t)nspecies * (per + ghost + perlo) + extra;
    cudaError_t e = dmalloc((void **)&st->base, total > 0 ? total : 16);
    if (e != cudaSuccess) {
        delete st;
        return cuda_fail(e, "cudaMalloc (state)");
    }
    st->bytes = (int64_t)total;
    char *p = (char *)st->base;
    for (int b = 0; b < 2; ++b)
        for (int s = 0; s < nspecies; ++s) {
            st->val[b][s] = p + ghost;
            p += ghost + per;
            if (perlo) {
                st->lo[b][s] = (float *)p;
                p += perlo;
            }
        }
    if (extra) {
        st->bh = (float *)p;
        st->bl = st->bh + st->nslots;
        st->rsrc = st->bl + st->nslots;
    }
    // every slot starts as the sentinel until sbg_state_set (0xff.. bytes: a NaN, not the sentinel,
    // so an unset state is reported as non-finite)
    e = cudaMemset(st->base, 0xff, total > 0 ? total : 16);
    if (e == cudaSuccess) {
        // the ghost blocks hold the sentinel for good (no kernel writes block -1)
        std::vector<unsigned char> gh(ghost);
        for (size_t i = 0; i < ghost; i += st->elem()) {
            if (st->elem() == 8) {
                const double v = sentinel_f64();
                std::memcpy(&gh[i], &v, 8);
            } else {
                const float v = sentinel_f32();
                std::memcpy(&gh[i], &v, 4);
            }
        }
        for (int b = 0; b < 2 && e == cudaSuccess; ++b)
            for (int s = 0; s < nspecies && e == cudaSuccess; ++s)
                e = cudaMemcpy((char *)st->val[b][s] - ghost, gh.data(), ghost, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        dfree(st->base);
        delete st;
        return cuda_fail(e, "cudaMemset (state)");
    }
    st->has_ghost = true;
    *out = st;
    return SBG_OK;
}

extern "C" sbg_status sbg_state_set(sbg_grid g, sbg_state st, int32_t geom, int32_t species,
                                    const void *dense, int32_t dense_dtype, int32_t on_device,
                                    void *stream) {
    TraceRange trace_range("sbg_state_set");
    return dense_io(g, st, geom, species, const_cast<void *>(dense), dense_dtype, on_device, true, stream);
}

extern "C" sbg_status sbg_state_get(sbg_grid g, sbg_state st, int32_t geom, int32_t species,
                                    void *dense, int32_t dense_dtype, int32_t on_device, void *stream) {
    TraceRange trace_range("sbg_state_get");
    return dense_io(g, st, geom, species, dense, dense_dtype, on_device, false, stream);
}

extern "C" sbg_status sbg_state_copy(sbg_state dst, sbg_state src, void *stream) {
    if (!dst || !src) return fail(SBG_ERR_INVALID_ARG, "sbg_state_copy: null pointer");
    if (dst->grid != src->grid || dst->dtype != src->dtype || dst->ns != src->ns)
        return fail(SBG_ERR_INVALID_ARG, "sbg_state_copy: grid, dtype or species differ");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t per = (size_t)src->nslots * src->elem();
    for (int sp = 0; sp < src->ns; ++sp) {
        SBG_CUDA(cudaMemcpyAsync(dst->val[dst->cur][sp], src->val[src->cur][sp], per,
                                 cudaMemcpyDeviceToDevice, s));
        if (src->dtype == SBG_F32X2)
            SBG_CUDA(cudaMemcpyAsync(dst->lo[dst->cur][sp], src->lo[src->cur][sp],
                                     (size_t)src->nslots * 4, cudaMemcpyDeviceToDevice, s));
    }
    if (src->dtype == SBG_F32R) {  // base hi, lo and source are contiguous
        SBG_CUDA(cudaMemcpyAsync(dst->bh, src->bh, 3 * (size_t)src->nslots * 4, cudaMemcpyDeviceToDevice, s));
        dst->r_valid = src->r_valid;
        dst->since_refresh = src->since_refresh;
    }
    return SBG_OK;
}

extern "C" void sbg_state_destroy(sbg_state st) {
    if (!st) return;
    if (st->graph) cudaGraphExecDestroy(st->graph);
    wave_destroy(st);
    dfree(st->ext[0]);
    dfree(st->ext[1]);
    dfree(st->base);
    delete st;
}
