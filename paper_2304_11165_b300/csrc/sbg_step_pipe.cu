// Pipelined persistent step kernel for FP32 and compensated-FP32 states.
//
// Why: one thread per voxel with one 4-byte load each keeps only ~8 KB in
// flight per SM, far below what HBM3e needs (~40 KB per SM at ~800 ns), and a
// 7-point stencil on B300 has a budget of only ~40 issued instructions per
// FP32 voxel update before the SM, not HBM, is the limit.  So:
//  - persistent CTAs (several per SM) each walk a contiguous range of
//    "groups" of the block list (a group = 512 voxels: one 8^3 block or eight
//    4^3 blocks, contiguous in memory);
//  - one thread streams groups into an S-stage shared-memory ring with 1-D
//    bulk copies (cp.async.bulk, TMA engine) completing on per-stage
//    mbarriers, S groups ahead of the compute; only that thread waits on the
//    barrier, the others sleep in __syncthreads;
//  - each thread updates four x-consecutive voxels: its row and the rows
//    above/below/in front/behind come from shared memory as 16-byte loads;
//  - the one-voxel face halos come from the neighbouring blocks (mostly L2
//    hits): face ids are prefetched two groups ahead and halo values one
//    group ahead into registers (two alternating register sets, no copies),
//    so their latency overlaps the current group's compute;
//  - results leave as one 16-byte store per thread and array.
// Every wait on an mbarrier is bounded: on time-out the CTA sets the grid's
// error word (reported as SBG_ERR_TIMEOUT), waits (bounded) for its copies in
// flight and exits.
#include "sbg_ptx.cuh"
#include "sbg_step.cuh"

namespace sbg {

constexpr int kPipeThreads = 128;
constexpr int kGroupVox = 512;

__device__ __forceinline__ float f4get(const float4 &v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

template <bool X2, int B, int NS, bool REACT, int S>
__global__ void __launch_bounds__(kPipeThreads) k_step_pipe(const StepArgs a, int *err) {
    constexpr int B3 = B * B * B;
    constexpr int G = kGroupVox / B3;
    constexpr int NA = X2 ? 2 : NS;  // arrays streamed per group
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *stages = reinterpret_cast<float *>(smem_raw);  // [S][NA][512]
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + (size_t)S * NA * kGroupVox * sizeof(float));

    const int tid = threadIdx.x;
    const int64_t ngroups = (a.nb + G - 1) / G;
    const int64_t g0 = ngroups * blockIdx.x / gridDim.x;
    const int64_t g1 = ngroups * (blockIdx.x + 1) / gridDim.x;
    if (g0 >= g1) return;  // uniform over the CTA

    const float *src[NA];
    float *dst[NA];
    if (X2) {
        src[0] = (const float *)a.in[0];
        src[NA - 1] = a.in_lo[0];
        dst[0] = (float *)a.out[0];
        dst[NA - 1] = a.out_lo[0];
    } else {
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            src[k] = (const float *)a.in[k];
            dst[k] = (float *)a.out[k];
        }
    }

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();

    auto issue = [&](int64_t gi, int s) {
        const int64_t b0 = gi * G;
        const int64_t nblk = (a.nb - b0 < G) ? (a.nb - b0) : G;
        const uint32_t bytes = (uint32_t)(nblk * B3 * sizeof(float));
        mbar_arrive_expect_tx(&full[s], bytes * NA);
#pragma unroll
        for (int k = 0; k < NA; ++k)
            bulk_g2s(stages + ((size_t)s * NA + k) * kGroupVox, src[k] + b0 * B3, bytes, &full[s]);
    };
    if (tid == 0)
        for (int s = 0; s < S && g0 + s < g1; ++s) issue(g0 + s, s);

    // this thread's voxels: v0 .. v0 + 3 (x0 .. x0 + 3 of one row) in block j of the group
    const int v0 = 4 * tid;
    const int j = v0 / B3;
    const int l0 = v0 - j * B3;
    const int x0 = l0 % B, y = (l0 / B) % B, z = l0 / (B * B);
    const bool dxm = (x0 == 0), dxp = (x0 + 3 == B - 1);  // x-halo duties
    const int fy = (y == 0) ? 2 : (y == B - 1) ? 3 : -1;
    const int fz = (z == 0) ? 4 : (z == B - 1) ? 5 : -1;
    const int oxm = l0 + (B - 1), oxp = l0 + 3 - (B - 1);
    const int oy = (fy == 2) ? l0 + (B - 1) * B : l0 - (B - 1) * B;
    const int oz = (fz == 4) ? l0 + (B - 1) * B * B : l0 - (B - 1) * B * B;
    const float SENT = sentinel_f32();

    struct Ids {
        int xm, xp, y, z, ws;
    };
    struct Halo {
        float hxm[NA], hxp[NA];
        float4 hy[NA], hz[NA];
        float4 w;
        int4 bc;
    };
    auto load_ids = [&](int64_t gi) {
        Ids r{-1, -1, -1, -1, -1};
        const int64_t b = gi * G + j;
        if (gi < g1 && b < a.nb) {
            const int32_t *f = a.face + b * 6;
            if (dxm) r.xm = __ldg(f + 0);
            if (dxp) r.xp = __ldg(f + 1);
            if (fy >= 0) r.y = __ldg(f + fy);
            if (fz >= 0) r.z = __ldg(f + fz);
            if (REACT) r.ws = __ldg(a.wslab + b);
        }
        return r;
    };
    auto load_halo = [&](int64_t gi, const Ids &id, Halo &h) {
        const int64_t b = gi * G + j;
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const float absent = (X2 && k == 1) ? 0.f : SENT;
            h.hxm[k] = (id.xm >= 0) ? __ldg(src[k] + (int64_t)id.xm * B3 + oxm) : absent;
            h.hxp[k] = (id.xp >= 0) ? __ldg(src[k] + (int64_t)id.xp * B3 + oxp) : absent;
            h.hy[k] = (id.y >= 0) ? __ldg(reinterpret_cast<const float4 *>(src[k] + (int64_t)id.y * B3 + oy))
                                  : make_float4(absent, absent, absent, absent);
            h.hz[k] = (id.z >= 0) ? __ldg(reinterpret_cast<const float4 *>(src[k] + (int64_t)id.z * B3 + oz))
                                  : make_float4(absent, absent, absent, absent);
        }
        h.w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (REACT && id.ws >= 0) h.w = __ldg(reinterpret_cast<const float4 *>(a.w + (int64_t)id.ws * B3 + l0));
        h.bc = make_int4(0, 0, 0, 0);
        if (a.held_mask && gi < g1 && b < a.nb) h.bc = __ldg(a.blocks + b);
    };

    auto body = [&](int64_t gi, int it, const Halo &cur, Halo &nxt, const Ids &id1, Ids &id2) -> bool {
        const int s = it % S;
        const uint32_t par = (uint32_t)((it / S) & 1);
        id2 = load_ids(gi + 2);
        load_halo(gi + 1, id1, nxt);

        bool ok = true;
        if (tid == 0) ok = mbar_wait_bounded(&full[s], par);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(err, (int)SBG_ERR_TIMEOUT);
                for (int q = it; q < it + S && g0 + q < g1; ++q)
                    mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1), 1ll << 28);
            }
            return false;
        }
        mbar_try_wait(&full[s], par);  // completed: gives this thread the acquire of the copied data
        // every thread has finished the previous group: refill its stage
        if (tid == 0 && it >= 1 && gi - 1 + S < g1) issue(gi - 1 + S, (it - 1) % S);

        const int64_t b = gi * G + j;
        if (b >= a.nb) return true;
        const float *sb = stages + (size_t)s * NA * kGroupVox;

        // Dirichlet-held voxels
        bool held[4] = {false, false, false, false};
        if (a.held_mask) {
            const int4 bc = cur.bc;
            const int nx = __ldg(a.gdims + bc.w * 4 + 0), ny = __ldg(a.gdims + bc.w * 4 + 1),
                      nz = __ldg(a.gdims + bc.w * 4 + 2);
            const int gx = bc.x * B + x0, gy = bc.y * B + y, gz = bc.z * B + z;
#pragma unroll
            for (int i = 0; i < 4; ++i) held[i] = is_held(a.held_mask, gx + i, gy, gz, nx, ny, nz);
        }

        float4 uc[NA], ym[NA], yp[NA], zm[NA], zp[NA];
        float xm[NA], xp[NA];
#pragma unroll
        for (int k = 0; k < NA; ++k) {
            const float *t = sb + k * kGroupVox;
            uc[k] = *reinterpret_cast<const float4 *>(t + v0);
            xm[k] = dxm ? cur.hxm[k] : t[v0 - 1];
            xp[k] = dxp ? cur.hxp[k] : t[v0 + 4];
            ym[k] = (y > 0) ? *reinterpret_cast<const float4 *>(t + v0 - B) : cur.hy[k];
            yp[k] = (y < B - 1) ? *reinterpret_cast<const float4 *>(t + v0 + B) : cur.hy[k];
            zm[k] = (z > 0) ? *reinterpret_cast<const float4 *>(t + v0 - B * B) : cur.hz[k];
            zp[k] = (z < B - 1) ? *reinterpret_cast<const float4 *>(t + v0 + B * B) : cur.hz[k];
        }
        const StepCoef<float> &kc = a.cf;
        float res[NA][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (X2) {
                const float hc = f4get(uc[0], i), lc = f4get(uc[NA - 1], i);
                res[0][i] = hc;
                res[NA - 1][i] = lc;
                if (!is_sent(hc) && !held[i]) {
                    const float hv[6] = {i == 0 ? xm[0] : f4get(uc[0], i - 1), i == 3 ? xp[0] : f4get(uc[0], i + 1),
                                         f4get(ym[0], i), f4get(yp[0], i), f4get(zm[0], i), f4get(zp[0], i)};
                    const float lv[6] = {i == 0 ? xm[NA - 1] : f4get(uc[NA - 1], i - 1),
                                         i == 3 ? xp[NA - 1] : f4get(uc[NA - 1], i + 1),
                                         f4get(ym[NA - 1], i), f4get(yp[NA - 1], i),
                                         f4get(zm[NA - 1], i), f4get(zp[NA - 1], i)};
                    float nh[6], nl[6];
#pragma unroll
                    for (int f = 0; f < 6; ++f) {
                        const bool m = is_sent(hv[f]);
                        nh[f] = m ? hc : hv[f];
                        nl[f] = m ? lc : lv[f];
                    }
                    float rate = kc.decay[0];
                    if (REACT) rate = __fmaf_rn(kc.k, f4get(cur.w, i), rate);
                    fused_update_x2(hc, lc, nh, nl, kc.c[0], kc.dt, rate, res[0][i], res[NA - 1][i]);
                }
            } else {
                const float ua = f4get(uc[0], i);
                const float t = REACT ? __fmul_rn(__fmul_rn(kc.k, f4get(cur.w, i)), ua) : 0.f;
#pragma unroll
                for (int k = 0; k < NA; ++k) {
                    const float c = f4get(uc[k], i);
                    res[k][i] = c;
                    if (!is_sent(c) && !held[i]) {
                        const float vxm = i == 0 ? xm[k] : f4get(uc[k], i - 1);
                        const float vxp = i == 3 ? xp[k] : f4get(uc[k], i + 1);
                        res[k][i] = fused_update(c, mirror(vxm, c), mirror(vxp, c), mirror(f4get(ym[k], i), c),
                                                 mirror(f4get(yp[k], i), c), mirror(f4get(zm[k], i), c),
                                                 mirror(f4get(zp[k], i), c), kc.c[k], kc.dt, kc.decay[k],
                                                 k == 0 ? -t : t);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NA; ++k)
            *reinterpret_cast<float4 *>(dst[k] + b * B3 + l0) = make_float4(res[k][0], res[k][1], res[k][2], res[k][3]);
        return true;
    };

    Ids idA = load_ids(g0), idB;
    Halo hA, hB;
    load_halo(g0, idA, hA);
    idA = load_ids(g0 + 1);
    int it = 0;
    for (int64_t gi = g0; gi < g1; gi += 2, it += 2) {
        if (!body(gi, it, hA, hB, idA, idB)) return;
        if (gi + 1 >= g1) break;
        if (!body(gi + 1, it + 1, hB, hA, idB, idA)) return;
    }
}

template <bool X2, int B, int NS, bool REACT>
static cudaError_t launch_pipe_t(const StepArgs &a, int ctas_per_sm, int *err, cudaStream_t s) {
    constexpr int S = 8;
    constexpr int NA = X2 ? 2 : NS;
    constexpr size_t smem = (size_t)S * NA * kGroupVox * sizeof(float) + S * sizeof(uint64_t);
    auto kern = k_step_pipe<X2, B, NS, REACT, S>;
    static int occ = -1, nsm = 0;
    if (occ < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kPipeThreads, smem);
        if (occ < 1) occ = 1;
    }
    const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
    constexpr int G = kGroupVox / (B * B * B);
    const int64_t ngroups = (a.nb + G - 1) / G;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > ngroups) grid = ngroups;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, kPipeThreads, smem, s>>>(a, err);
    return cudaGetLastError();
}

bool launch_step_pipe(const StepArgs &a, sbg_dtype dtype, int ns, int B, bool react, int ctas_per_sm,
                      int *err_flag, cudaStream_t s, cudaError_t *launch_err) {
    cudaError_t e = cudaSuccess;
    if (dtype == SBG_F32X2 && ns == 1) {
        if (B == 8) e = react ? launch_pipe_t<true, 8, 1, true>(a, ctas_per_sm, err_flag, s)
                              : launch_pipe_t<true, 8, 1, false>(a, ctas_per_sm, err_flag, s);
        else e = react ? launch_pipe_t<true, 4, 1, true>(a, ctas_per_sm, err_flag, s)
                       : launch_pipe_t<true, 4, 1, false>(a, ctas_per_sm, err_flag, s);
    } else if (dtype == SBG_F32 && ns == 1) {
        if (B == 8) e = react ? launch_pipe_t<false, 8, 1, true>(a, ctas_per_sm, err_flag, s)
                              : launch_pipe_t<false, 8, 1, false>(a, ctas_per_sm, err_flag, s);
        else e = react ? launch_pipe_t<false, 4, 1, true>(a, ctas_per_sm, err_flag, s)
                       : launch_pipe_t<false, 4, 1, false>(a, ctas_per_sm, err_flag, s);
    } else if (dtype == SBG_F32 && ns == 2) {
        if (B == 8) e = react ? launch_pipe_t<false, 8, 2, true>(a, ctas_per_sm, err_flag, s)
                              : launch_pipe_t<false, 8, 2, false>(a, ctas_per_sm, err_flag, s);
        else e = react ? launch_pipe_t<false, 4, 2, true>(a, ctas_per_sm, err_flag, s)
                       : launch_pipe_t<false, 4, 2, false>(a, ctas_per_sm, err_flag, s);
    } else {
        return false;
    }
    *launch_err = e;
    return true;
}

}  // namespace sbg
