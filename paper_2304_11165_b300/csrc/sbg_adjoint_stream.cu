// Streaming adjoint step: lambda^n = M^T lambda^{n+1} for one FP32 species on
// 4^3 blocks (the checkpointed adjoint of the forward-Euler step of Eq. 1,
// transposed masked stencil and surface sink), with the gradient terms
// dt lambda g(u^n) (dL/dD) and dt w u^n (0 - lambda) (dL/dk) summed on the
// way.  The structure of the streaming step kernel (sbg_step_stream.cu): CTAs
// of 256 threads take groups of 16 blocks in turn, one x-row of four voxels
// per thread, every row it needs (its own and the y/z neighbour rows, the two
// x neighbour values) read from global memory through L1, for lambda^{n+1}
// (the state) and u^n (a tape buffer) at the same offsets; an absent
// neighbour block is the ghost block of sentinels both arrays start with.
// The per-row arithmetic is row_adjoint1, the ring kernel's, so lambda is
// bitwise the ring kernel's and the gradients differ only in the order of
// their double-float additions: per thread and warp in double-float, per CTA
// in FP64, added to the CTA's own slot (fixed order for a fixed grid).
#include <algorithm>

#include "sbg_adj_row.cuh"
#include "sbg_row.cuh"

namespace sbg {

constexpr int kAdjStreamThreads = 256;  // 16 blocks x 16 rows

template <bool REACT, bool HELD, int MINB>
__global__ void __launch_bounds__(kAdjStreamThreads, MINB)
k_adjoint_stream(const StepArgs a, const float *__restrict__ lam_in, const float *__restrict__ u_in,
                 float *__restrict__ lam_out, double *gsum, float i0, float i1, float i2,
                 const int2 *__restrict__ wmeta, const float4 *__restrict__ wrow, int *err, int n_wrows) {
    const int t = threadIdx.x;
    const int j = t >> 4, rr = t & 15, y = rr & 3, z = rr >> 2;
    const int nb = (int)a.nb;  // the launcher guarantees (nb + 2) * 64 < 2^31
    const int ngroups = (nb + 15) >> 4;
    const int G = (int)gridDim.x;
    const float *gl = lam_in - 64;  // block f at (f + 1) * 64, an absent one (f = -1) at the ghost block
    const float *gu = u_in - 64;
    const int oxm = 64 + rr * 4 + 3, oxp = 64 + rr * 4;
    const int oym = 64 + rr * 4 + 12, oyp = 64 + rr * 4 - 12;
    const int ozm = 64 + rr * 4 + 48, ozp = 64 + rr * 4 - 48;
    struct Meta {
        int f[4];
        int woff;
        uint32_t wmask, held;
    };
    auto load_meta = [&](int gi, Meta &m) {
        const int b = gi * 16 + j;
        if (gi < ngroups && b < nb) {
            const int32_t *fp = a.face + (int64_t)b * 6;
            m.f[0] = __ldg(fp + 0);
            m.f[1] = __ldg(fp + 1);
            m.f[2] = (y == 0) ? __ldg(fp + 2) : (y == 3) ? __ldg(fp + 3) : -1;
            m.f[3] = (z == 0) ? __ldg(fp + 4) : (z == 3) ? __ldg(fp + 5) : -1;
            if (REACT) {
                const int2 wm = __ldg(wmeta + b);
                m.woff = wm.x;
                m.wmask = (uint32_t)wm.y;
            } else {
                m.woff = 0;
                m.wmask = 0;
            }
            m.held = HELD ? (uint32_t)(__ldg(a.heldbits + b) >> (rr * 4)) & 0xFu : 0u;
#if SBG_DEBUG
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (m.f[k] < -1 || m.f[k] >= nb) {
                    atomicExch(err, (int)SBG_ERR_BOUNDS);
                    m.f[k] = -1;
                }
#endif
        } else {
            m.f[0] = m.f[1] = m.f[2] = m.f[3] = -1;
            m.woff = 0;
            m.wmask = 0;
            m.held = 0;
        }
    };
    (void)err;
    (void)n_wrows;
    float gh[2] = {0.f, 0.f}, glo[2] = {0.f, 0.f};  // this thread's dL/dD and dL/dk, double-float
    Meta cur, nxt;
    load_meta(blockIdx.x, cur);
    for (int gi = blockIdx.x; gi < ngroups; gi += G) {
        const int *f = cur.f;
        const int b = gi * 16 + j;
        const bool valid = b < nb;
        const int row = valid ? (b + 1) * 64 + rr * 4 : rr * 4;
        const int o_xm = f[0] * 64 + oxm;
        const int o_xp = f[1] * 64 + oxp;
        const int o_ym = y > 0 ? row - 4 : f[2] * 64 + oym;
        const int o_yp = y < 3 ? row + 4 : f[2] * 64 + oyp;
        const int o_zm = z > 0 ? row - 16 : f[3] * 64 + ozm;
        const int o_zp = z < 3 ? row + 16 : f[3] * 64 + ozp;
        float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (REACT && valid && ((cur.wmask >> rr) & 1u)) {
            const int wi = cur.woff + __popc(cur.wmask & ((1u << rr) - 1u));
#if SBG_DEBUG
            if (wi < 0 || wi >= n_wrows) atomicExch(err, (int)SBG_ERR_BOUNDS);
            else
#endif
                w4 = __ldg(wrow + wi);
        }
        RowVals v0, v1;  // lambda^{n+1}, u^n
        v0.u = ldg4(gl + row);
        v0.ym = ldg4(gl + o_ym);
        v0.yp = ldg4(gl + o_yp);
        v0.zm = ldg4(gl + o_zm);
        v0.zp = ldg4(gl + o_zp);
        v0.xm = __ldg(gl + o_xm);
        v0.xp = __ldg(gl + o_xp);
        v1.u = ldg4(gu + row);
        v1.ym = ldg4(gu + o_ym);
        v1.yp = ldg4(gu + o_yp);
        v1.zm = ldg4(gu + o_zm);
        v1.zp = ldg4(gu + o_zp);
        v1.xm = __ldg(gu + o_xm);
        v1.xp = __ldg(gu + o_xp);
        const uint32_t held = cur.held;
        load_meta(gi + G, nxt);  // the next group's tables, in flight while this one computes
        float qd = 0.f, qk = 0.f;
        const float4 r = row_adjoint1<REACT>(v0, v1, w4, held, a.cf, i0, i1, i2, qd, qk);
        if (valid) *reinterpret_cast<float4 *>(lam_out + (row - 64)) = r;
        df_add(gh[0], glo[0], qd, 0.f);
        if (REACT) df_add(gh[1], glo[1], qk, 0.f);
        cur = nxt;
    }
    // CTA sums: double-float across the warp, FP64 across the warps, added to the CTA's own
    // slots (dL/dD_0 and dL/dk)
    __shared__ double red[kAdjStreamThreads / 32][2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_down_sync(0xffffffffu, gh[q], o);
            const float l2 = __shfl_down_sync(0xffffffffu, glo[q], o);
            df_add(gh[q], glo[q], h2, l2);
        }
        if ((t & 31) == 0) red[t >> 5][q] = (double)gh[q] + (double)glo[q];
    }
    __syncthreads();
    if (t < 2) {
        double v = 0.0;
        for (int w = 0; w < kAdjStreamThreads / 32; ++w) v += red[w][t];
        gsum[(int64_t)blockIdx.x * 3 + (t == 0 ? 0 : 2)] += v;
    }
}

template <bool REACT, bool HELD>
static cudaError_t launch_adj_stream_t(const StepArgs &a, const float *lam_in, const float *u_in, float *lam_out,
                                       double *gsum, const float inv2[3], sbg_grid g, int max_ctas,
                                       cudaStream_t s) {
    constexpr int MINB = 3;
    auto kern = k_adjoint_stream<REACT, HELD, MINB>;
    static int occ = -1, nsm = 0;
    if (occ < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0);  // all of it as L1
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kAdjStreamThreads, 0);
        if (occ < 1) occ = 1;
    }
    const int64_t ngroups = (a.nb + 15) / 16;
    int64_t grid = (int64_t)nsm * occ;
    if (grid > ngroups) grid = ngroups;
    if (grid > max_ctas) grid = max_ctas;
    if (grid < 1) return cudaSuccess;
    const int nw = (int)std::min<int64_t>(g->n_wrows, INT32_MAX);
    kern<<<(unsigned)grid, kAdjStreamThreads, 0, s>>>(a, lam_in, u_in, lam_out, gsum, inv2[0], inv2[1], inv2[2],
                                                     g->wmeta, g->wrow, g->err, nw);
    return cudaGetLastError();
}

bool adjoint_stream_applies(sbg_grid g, sbg_state lam) {
    return lam->dtype == SBG_F32 && lam->ns == 1 && lam->has_ghost && g->B == 4 && !g->has_eps &&
           g->wmeta != nullptr && (g->nb + 2) * 64 < (int64_t(1) << 31);
}

cudaError_t launch_adjoint_stream(const StepArgs &a, const float *lam_in, const float *u_in, float *lam_out,
                                  double *gsum, const float inv2[3], sbg_grid g, bool react, int max_ctas,
                                  cudaStream_t s) {
    const bool held = a.held_mask != 0;
    if (react) return held ? launch_adj_stream_t<true, true>(a, lam_in, u_in, lam_out, gsum, inv2, g, max_ctas, s)
                           : launch_adj_stream_t<true, false>(a, lam_in, u_in, lam_out, gsum, inv2, g, max_ctas, s);
    return held ? launch_adj_stream_t<false, true>(a, lam_in, u_in, lam_out, gsum, inv2, g, max_ctas, s)
                : launch_adj_stream_t<false, false>(a, lam_in, u_in, lam_out, gsum, inv2, g, max_ctas, s);
}

}  // namespace sbg
