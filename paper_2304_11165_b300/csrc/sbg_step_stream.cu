// Streaming step kernel: the forward-Euler FTCS step of Eq. 1 (Sec. 2.3, the
// no-flux rule of Appendix B Listing 6, the surface sink of Sec. 3.5) for
// FP32 states of one or two species on 4^3 blocks.
//
// Why this form: the step moves 8 B per species and voxel and does ~12 FP32
// operations for it, so on B300 it is bound by HBM bytes and by how many of
// them are in flight, not by arithmetic.  The ring-buffer kernels
// (sbg_step_pipe.cu) stage every group through shared memory and fetch the
// face halos of each group with extra copies; with two species they fit only
// a few CTAs per SM and stay latency-bound.  Here:
//  - CTAs of 16 threads per block take groups of consecutive blocks of the
//    list in turn (16 blocks; 12 for two species, in CTAs of 192 threads, four
//    per SM, which measured 1% faster than 16 blocks at three per SM; group g
//    goes to CTA g mod gridDim), so at any moment the whole GPU
//    works on one window of the list.  On a grid built in plane order
//    (SBG_ORDER_PLANES: x fastest, z slowest) that window sweeps the box plane
//    by plane, and the face neighbours of every block (in the same plane, one
//    plane below or one above) were read less than one sweep ago or are read
//    within one sweep: they come from L2, never again from HBM;
//  - one thread per x-row of four voxels: its own row, the four y/z
//    neighbour rows and the two x neighbour values are read straight from
//    global memory (16-byte loads through L1; rows of the same block are read
//    by the same half-warp).  An absent neighbour block reads the state's
//    ghost block (block id -1, all sentinels), so no pointer selects;
//  - the +x neighbour values a group reads sit in the blocks of the next
//    groups, so every sweep pulls the rows of the sweep after it into L2 as a
//    side effect; beyond that, only a per-thread L2 prefetch of its own row
//    of the next group (one sweep ahead) for two species and SBG_F32R states,
//    the cases where it measured faster (bulk L2 prefetches a few sweeps
//    ahead measured 12-29% slower on the 512^3 two-species run: they compete
//    for L2 with the sweep in flight);
//  - the face ids, band-row metadata and held bits of the next group are
//    loaded while the current group computes.
// The per-voxel arithmetic is the plain kernel's (sbg_step.cu) with every
// rounding pinned: the x differences of a row are formed once and shared by
// neighbouring voxels (the same values), and an inactive neighbour (sentinel)
// is mirrored.  States are bitwise equal to the plain kernel's (tested).
// There is no wait on another thread or CTA in this kernel.
#include <algorithm>

#include "sbg_row.cuh"

namespace sbg {

constexpr int kStreamThreads = 256;  // 16 blocks x 16 rows of 4 voxels

// SRC: the correction d of an SBG_F32R state (one species, no surface
// reaction): the stored source r = L_h b of the row takes the place of the
// transfer term, d' = d + dt (L_h d - decay d + r), as in the plain kernel.
// WL: the groups are the spans of a work list (a.items: first block, blocks;
// at most 16 blocks each, within one geometry) instead of consecutive groups of
// the list: the batch solver's steps over its unconverged geometries.
// GB: blocks per group (16 threads each); 16 with a work list.
template <int NS, bool REACT, bool HELD, int MINB, bool SRC = false, bool WL = false, int GB = 16>
__global__ void __launch_bounds__(16 * GB, MINB)
k_step_stream(const StepArgs a, const int2 *__restrict__ wmeta, const float4 *__restrict__ wrow, float negzero, int *err,
              int n_wrows) {
    const int t = threadIdx.x;
    const int j = t >> 4, rr = t & 15, y = rr & 3, z = rr >> 2;
    const int nb = (int)a.nb;  // the launcher guarantees (nb + 2) * 64 < 2^31
    const int ngroups = WL ? (int)a.nitems : (nb + GB - 1) / GB;
    const int G = (int)gridDim.x;
    // this thread's block in group gi (-1: none)
    auto block_of = [&](int gi) -> int {
        if (gi >= ngroups) return -1;
        if (WL) {
            const int first = (int)__ldg(a.items + 2 * (int64_t)gi);
            const int count = (int)__ldg(a.items + 2 * (int64_t)gi + 1);
            return j < count ? first + j : -1;
        }
        const int b = gi * GB + j;
        return b < nb ? b : -1;
    };
    // every species array is preceded by a ghost block of sentinels, block id -1: offsets
    // below are taken from that block's start, so block f sits at (f + 1) * 64 and an
    // absent neighbour (f = -1) at 0
    const float *gb[NS];
    float *out[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        gb[s] = (const float *)a.in[s] - 64;
        out[s] = (float *)a.out[s];
    }
    // neighbour rows of this thread's row inside the neighbour block
    const int oxm = 64 + rr * 4 + 3, oxp = 64 + rr * 4;
    const int oym = 64 + rr * 4 + 12, oyp = 64 + rr * 4 - 12;
    const int ozm = 64 + rr * 4 + 48, ozp = 64 + rr * 4 - 48;

    // per thread: the face neighbours of its block it reads (-x, +x, the y side, the z side),
    // its block's band rows and its row's held bits
    struct Meta {
        int b;  // the block (-1: none)
        int f[4];
        int woff;
        uint32_t wmask, held;
    };
    auto load_meta = [&](int gi, Meta &m) {
        const int b = block_of(gi);
        m.b = b;
        if (b >= 0) {
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

    Meta cur, nxt;
    load_meta(blockIdx.x, cur);
    for (int gi = blockIdx.x; gi < ngroups; gi += G) {
        const int *f = cur.f;
        const int woff = cur.woff;
        const uint32_t wmask = cur.wmask, held = cur.held;
        const int b = cur.b;
        const bool valid = b >= 0;
        // offsets from the ghost block's start of every value this row reads (a thread past the
        // end of the list reads the ghost block and stores nothing)
        const int row = valid ? (b + 1) * 64 + rr * 4 : rr * 4;
        const int o_xm = f[0] * 64 + oxm;
        const int o_xp = f[1] * 64 + oxp;
        const int o_ym = y > 0 ? row - 4 : f[2] * 64 + oym;
        const int o_yp = y < 3 ? row + 4 : f[2] * 64 + oyp;
        const int o_zm = z > 0 ? row - 16 : f[3] * 64 + ozm;
        const int o_zp = z < 3 ? row + 16 : f[3] * 64 + ozp;
        float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (REACT && valid && ((wmask >> rr) & 1u)) {
            const int wi = woff + __popc(wmask & ((1u << rr) - 1u));
#if SBG_DEBUG
            if (wi < 0 || wi >= n_wrows) atomicExch(err, (int)SBG_ERR_BOUNDS);
            else
#endif
                w4 = __ldg(wrow + wi);
        }
        load_meta(gi + G, nxt);  // the next group's tables, in flight while this one computes
        if (NS == 2 || SRC) {  // this thread's row of the next group, one sweep ahead (measured: 1.3% faster on
                               // the 512^3 two-species run, 1.8% for SBG_F32R on grf256; slower for the others)
            const int bn = nxt.b;
            if (bn >= 0) {
#pragma unroll
                for (int s = 0; s < NS; ++s) prefetch_l2(gb[s] + (bn + 1) * 64 + rr * 4);
            }
        }
        uint32_t keep[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) keep[i] = ((held >> i) & 1u) ? ~0u : 0u;
        f32x2 tr01 = 0ull, tr23 = 0ull;  // the surface transfer k w u_A, from species A's pass
        if (SRC) {
            const float4 r4 = valid ? ldg4(a.src_term + (row - 64)) : make_float4(0.f, 0.f, 0.f, 0.f);
            tr01 = pk(r4.x, r4.y);
            tr23 = pk(r4.z, r4.w);
        }
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const float *q = gb[s];
            const float4 c = ldg4(q + row);
            const float4 ym = ldg4(q + o_ym), yp = ldg4(q + o_yp);
            const float4 zm = ldg4(q + o_zm), zp = ldg4(q + o_zp);
            const float xm = __ldg(q + o_xm), xp = __ldg(q + o_xp);
            if (s == 0 && REACT) {
                const f32x2 k2 = pk(a.cf.k, a.cf.k);
                tr01 = mul2(mul2(k2, pk(w4.x, w4.y)), pk(c.x, c.y));
                tr23 = mul2(mul2(k2, pk(w4.z, w4.w)), pk(c.z, c.w));
            }
            float ta, tb, tc, td;
            upk(tr01, ta, tb);
            upk(tr23, tc, td);
            // species A loses the transfer, B gains it (the plain kernel's -/+ of the same product;
            // without a surface reaction the product is +0 and A's term is -0).  That -0 comes in
            // as a kernel argument: an addend the compiler knows to be -0 would let it turn the
            // packed fma of the decay term into a product and fuse it with the add that follows,
            // which rounds once where the plain kernel rounds twice
            const f32x2 t01 = SRC ? tr01 : s == 0 ? (REACT ? pk(-ta, -tb) : pk(negzero, negzero)) : tr01;
            const f32x2 t23 = SRC ? tr23 : s == 0 ? (REACT ? pk(-tc, -td) : pk(negzero, negzero)) : tr23;
            const float4 r = row_update(c, xm, xp, ym, yp, zm, zp, a.cf.c[s], a.cf.dt, a.cf.decay[s], t01, t23, keep);
            if (valid) *reinterpret_cast<float4 *>(out[s] + (row - 64)) = r;
        }
        cur = nxt;
    }
}

// Inhomogeneous diffusion (the functor of Appendix B Listing 6 with the Eq. 6
// factor, one FP32 species): the same group walk and row reads, for the state
// u and for the diffusivity factor eps at the same offsets (an absent
// neighbour block reads the ghost blocks: sentinels for u, zeros for eps).
// Per voxel the plain kernel's inh_update: face fluxes with the mean of the
// two factors, a neighbour outside Omega (sentinel u) giving a zero
// difference; the x differences of a row are formed once and shared.
template <bool HELD, int MINB>
__global__ void __launch_bounds__(kStreamThreads, MINB)
k_step_stream_inh(const StepArgs a, int *err) {
    const int t = threadIdx.x;
    const int j = t >> 4, rr = t & 15, y = rr & 3, z = rr >> 2;
    const int nb = (int)a.nb;  // the launcher guarantees (nb + 2) * 64 < 2^31
    const int ngroups = (nb + 15) >> 4;
    const int G = (int)gridDim.x;
    const float *gu = (const float *)a.in[0] - 64;
    const float *ge = a.eps - 64;
    float *out = (float *)a.out[0];
    const int oxm = 64 + rr * 4 + 3, oxp = 64 + rr * 4;
    const int oym = 64 + rr * 4 + 12, oyp = 64 + rr * 4 - 12;
    const int ozm = 64 + rr * 4 + 48, ozp = 64 + rr * 4 - 48;
    struct Meta {
        int f[4];
        uint32_t held;
    };
    auto load_meta = [&](int gi, Meta &m) {
        const int b = gi * 16 + j;
        if (gi < ngroups && b < nb) {
            const int32_t *fp = a.face + (int64_t)b * 6;
            m.f[0] = __ldg(fp + 0);
            m.f[1] = __ldg(fp + 1);
            m.f[2] = (y == 0) ? __ldg(fp + 2) : (y == 3) ? __ldg(fp + 3) : -1;
            m.f[3] = (z == 0) ? __ldg(fp + 4) : (z == 3) ? __ldg(fp + 5) : -1;
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
            m.held = 0;
        }
    };
    (void)err;
    Meta cur, nxt;
    load_meta(blockIdx.x, cur);
    for (int gi = blockIdx.x; gi < ngroups; gi += G) {
        const int *f = cur.f;
        const uint32_t held = cur.held;
        const int b = gi * 16 + j;
        const bool valid = b < nb;
        const int row = valid ? (b + 1) * 64 + rr * 4 : rr * 4;
        const int o_xm = f[0] * 64 + oxm;
        const int o_xp = f[1] * 64 + oxp;
        const int o_ym = y > 0 ? row - 4 : f[2] * 64 + oym;
        const int o_yp = y < 3 ? row + 4 : f[2] * 64 + oyp;
        const int o_zm = z > 0 ? row - 16 : f[3] * 64 + ozm;
        const int o_zp = z < 3 ? row + 16 : f[3] * 64 + ozp;
        const float4 c = ldg4(gu + row);
        const float4 ym = ldg4(gu + o_ym), yp = ldg4(gu + o_yp);
        const float4 zm = ldg4(gu + o_zm), zp = ldg4(gu + o_zp);
        const float xm = __ldg(gu + o_xm), xp = __ldg(gu + o_xp);
        const float4 ec = ldg4(ge + row);
        const float4 eym = ldg4(ge + o_ym), eyp = ldg4(ge + o_yp);
        const float4 ezm = ldg4(ge + o_zm), ezp = ldg4(ge + o_zp);
        const float exm = __ldg(ge + o_xm), exp_ = __ldg(ge + o_xp);
        load_meta(gi + G, nxt);  // the next group's tables, in flight while this one computes
        const float R[6] = {xm, c.x, c.y, c.z, c.w, xp};
        const float E[6] = {exm, ec.x, ec.y, ec.z, ec.w, exp_};
        bool act[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) act[i] = !is_sent(R[i]);
        float D[5];  // x differences R[i+1] - R[i], shared by neighbouring voxels
#pragma unroll
        for (int i = 0; i < 5; ++i) D[i] = __fsub_rn(R[i + 1], R[i]);
        float res[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float u = R[i + 1];
            const float nym = f4at(ym, i), nyp = f4at(yp, i), nzm = f4at(zm, i), nzp = f4at(zp, i);
            const float vym = is_sent(nym) ? u : nym, vyp = is_sent(nyp) ? u : nyp;
            const float vzm = is_sent(nzm) ? u : nzm, vzp = is_sent(nzp) ? u : nzp;
            const float dp[3] = {act[i + 2] ? D[i + 1] : 0.f, __fsub_rn(vyp, u), __fsub_rn(vzp, u)};
            const float dm[3] = {act[i] ? D[i] : 0.f, __fsub_rn(u, vym), __fsub_rn(u, vzm)};
            const float en[6] = {E[i], E[i + 2], f4at(eym, i), f4at(eyp, i), f4at(ezm, i), f4at(ezp, i)};
            const float nr = inh_update(u, dp, dm, E[i + 1], en, a.cf.c[0], a.cf.dt, a.cf.decay[0]);
            res[i] = (act[i + 1] && !((held >> i) & 1u)) ? nr : u;
        }
        if (valid) *reinterpret_cast<float4 *>(out + (row - 64)) = make_float4(res[0], res[1], res[2], res[3]);
        cur = nxt;
    }
}

// Compensated FP32 state (SBG_F32X2, value = hi + lo, one species): hi and lo
// rows read at the same offsets, a neighbour outside Omega (sentinel hi)
// taking the centre's hi and lo, and per voxel the plain kernel's
// fused_update_x2 (error-free products and sums, the increment added with a
// two-sum).  The lo array follows the hi array in the state's allocation, so
// the 64 values before it (an absent neighbour's lo, never used: the mirror
// replaces it) are the hi array's last block.
template <bool REACT, bool HELD, int MINB>
__global__ void __launch_bounds__(kStreamThreads, MINB)
k_step_stream_x2(const StepArgs a, const int2 *__restrict__ wmeta, const float4 *__restrict__ wrow, int *err,
                 int n_wrows) {
    const int t = threadIdx.x;
    const int j = t >> 4, rr = t & 15, y = rr & 3, z = rr >> 2;
    const int nb = (int)a.nb;  // the launcher guarantees (nb + 2) * 64 < 2^31
    const int ngroups = (nb + 15) >> 4;
    const int G = (int)gridDim.x;
    const float *gh = (const float *)a.in[0] - 64;
    const float *gl = a.in_lo[0] - 64;
    float *oh = (float *)a.out[0];
    float *ol = a.out_lo[0];
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
    Meta cur, nxt;
    load_meta(blockIdx.x, cur);
    for (int gi = blockIdx.x; gi < ngroups; gi += G) {
        const int *f = cur.f;
        const uint32_t held = cur.held;
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
        const float4 hc = ldg4(gh + row), lc = ldg4(gl + row);
        const float4 hym = ldg4(gh + o_ym), hyp = ldg4(gh + o_yp), hzm = ldg4(gh + o_zm), hzp = ldg4(gh + o_zp);
        const float4 lym = ldg4(gl + o_ym), lyp = ldg4(gl + o_yp), lzm = ldg4(gl + o_zm), lzp = ldg4(gl + o_zp);
        const float hxm = __ldg(gh + o_xm), hxp = __ldg(gh + o_xp);
        const float lxm = __ldg(gl + o_xm), lxp = __ldg(gl + o_xp);
        load_meta(gi + G, nxt);  // the next group's tables, in flight while this one computes
        const float H[6] = {hxm, hc.x, hc.y, hc.z, hc.w, hxp};
        const float L[6] = {lxm, lc.x, lc.y, lc.z, lc.w, lxp};
        float rh[4], rl[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float c0 = H[i + 1], c1 = L[i + 1];
            const float h[6] = {H[i], H[i + 2], f4at(hym, i), f4at(hyp, i), f4at(hzm, i), f4at(hzp, i)};
            const float l[6] = {L[i], L[i + 2], f4at(lym, i), f4at(lyp, i), f4at(lzm, i), f4at(lzp, i)};
            float nh[6], nl[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const bool out = is_sent(h[q]);
                nh[q] = out ? c0 : h[q];
                nl[q] = out ? c1 : l[q];
            }
            float rate = a.cf.decay[0];
            if (REACT) rate = __fmaf_rn(a.cf.k, f4at(w4, i), rate);
            float vh, vl;
            fused_update_x2(c0, c1, nh, nl, a.cf.c[0], a.cf.dt, rate, vh, vl);
            const bool upd = !is_sent(c0) && !((held >> i) & 1u);
            rh[i] = upd ? vh : c0;
            rl[i] = upd ? vl : c1;
        }
        if (valid) {
            *reinterpret_cast<float4 *>(oh + (row - 64)) = make_float4(rh[0], rh[1], rh[2], rh[3]);
            *reinterpret_cast<float4 *>(ol + (row - 64)) = make_float4(rl[0], rl[1], rl[2], rl[3]);
        }
        cur = nxt;
    }
}

template <bool REACT, bool HELD>
static cudaError_t launch_stream_x2_t(const StepArgs &a, const int2 *wmeta, const float4 *wrow, int ctas_per_sm,
                                      int *err, int n_wrows, cudaStream_t s) {
    constexpr int MINB = 3;
    auto kern = k_step_stream_x2<REACT, HELD, MINB>;
    static int occ = -1, nsm = 0;
    if (occ < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0);  // all of it as L1
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kStreamThreads, 0);
        if (occ < 1) occ = 1;
    }
    const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
    const int64_t ngroups = (a.nb + 15) / 16;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > ngroups) grid = ngroups;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, kStreamThreads, 0, s>>>(a, wmeta, wrow, err, n_wrows);
    return cudaGetLastError();
}

bool stream_x2_applies(sbg_grid g, sbg_state st) {
    return st->dtype == SBG_F32X2 && st->ns == 1 && g->B == 4 && st->has_ghost && !g->has_eps &&
           g->wmeta != nullptr && (g->nb + 2) * 64 < (int64_t(1) << 31) &&
           st->lo[0][0] == (float *)st->val[0][0] + st->nslots && st->lo[1][0] == (float *)st->val[1][0] + st->nslots;
}

cudaError_t launch_step_stream_x2(const StepArgs &a, sbg_grid g, bool react, int ctas_per_sm, cudaStream_t s) {
    const bool held = a.held_mask != 0;
    const int nw = (int)std::min<int64_t>(g->n_wrows, INT32_MAX);
    if (react) return held ? launch_stream_x2_t<true, true>(a, g->wmeta, g->wrow, ctas_per_sm, g->err, nw, s)
                           : launch_stream_x2_t<true, false>(a, g->wmeta, g->wrow, ctas_per_sm, g->err, nw, s);
    return held ? launch_stream_x2_t<false, true>(a, g->wmeta, g->wrow, ctas_per_sm, g->err, nw, s)
                : launch_stream_x2_t<false, false>(a, g->wmeta, g->wrow, ctas_per_sm, g->err, nw, s);
}

template <bool HELD>
static cudaError_t launch_stream_inh_t(const StepArgs &a, int ctas_per_sm, int *err, cudaStream_t s) {
    constexpr int MINB = 3;
    auto kern = k_step_stream_inh<HELD, MINB>;
    static int occ = -1, nsm = 0;
    if (occ < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0);  // all of it as L1
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kStreamThreads, 0);
        if (occ < 1) occ = 1;
    }
    const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
    const int64_t ngroups = (a.nb + 15) / 16;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > ngroups) grid = ngroups;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, kStreamThreads, 0, s>>>(a, err);
    return cudaGetLastError();
}

bool stream_inh_applies(sbg_grid g, sbg_state st) {
    return st->dtype == SBG_F32 && st->ns == 1 && g->B == 4 && st->has_ghost && g->has_eps && g->eps != nullptr &&
           (g->nb + 2) * 64 < (int64_t(1) << 31);
}

cudaError_t launch_step_stream_inh(const StepArgs &a, sbg_grid g, int ctas_per_sm, cudaStream_t s) {
    return a.held_mask ? launch_stream_inh_t<true>(a, ctas_per_sm, g->err, s)
                       : launch_stream_inh_t<false>(a, ctas_per_sm, g->err, s);
}

template <int NS, bool REACT, bool HELD, bool SRC = false, bool WL = false>
static cudaError_t launch_stream_t(const StepArgs &a, const int2 *wmeta, const float4 *wrow, int ctas_per_sm,
                                   int *err, int n_wrows, cudaStream_t s) {
    // two species: groups of 12 blocks, 4 CTAs of 192 threads per SM (80 registers); otherwise 16
    // blocks, 256 threads, at least 3 CTAs per SM
    constexpr int GB = (NS == 2 && !WL) ? 12 : 16;
    constexpr int MINB = GB == 12 ? 4 : 3;
    constexpr int kThreads = 16 * GB;
    auto kern = k_step_stream<NS, REACT, HELD, MINB, SRC, WL, GB>;
    static int occ = -1, nsm = 0;
    if (occ < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0);  // all of it as L1
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kThreads, 0);
        if (occ < 1) occ = 1;
    }
    const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
    const int64_t ngroups = WL ? a.nitems : (a.nb + GB - 1) / GB;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > ngroups) grid = ngroups;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, kThreads, 0, s>>>(a, wmeta, wrow, -0.0f, err, n_wrows);
    return cudaGetLastError();
}

bool stream_kernel_applies(sbg_grid g, sbg_state st) {
    const bool kind = (st->dtype == SBG_F32 && (st->ns == 1 || st->ns == 2)) || (st->dtype == SBG_F32R && st->ns == 1);
    return kind && g->B == 4 && st->has_ghost && !g->has_eps && g->wmeta != nullptr &&
           (g->nb + 2) * 64 < (int64_t(1) << 31);
}

// WL: a.items holds a work list (spans of at most 16 blocks)
template <bool WL>
static cudaError_t launch_step_stream_t(const StepArgs &a, sbg_grid g, int ns, bool react, int ctas_per_sm,
                                       cudaStream_t s) {
    const bool held = a.held_mask != 0;
    const int2 *wm = g->wmeta;
    const float4 *wr = g->wrow;
    int *err = g->err;
    const int nw = (int)std::min<int64_t>(g->n_wrows, INT32_MAX);
    if (a.src_term) {  // SBG_F32R correction (the caller excludes a surface reaction)
        return held ? launch_stream_t<1, false, true, true, WL>(a, wm, wr, ctas_per_sm, err, nw, s)
                    : launch_stream_t<1, false, false, true, WL>(a, wm, wr, ctas_per_sm, err, nw, s);
    }
    if (ns == 1) {
        if (react) return held ? launch_stream_t<1, true, true, false, WL>(a, wm, wr, ctas_per_sm, err, nw, s)
                               : launch_stream_t<1, true, false, false, WL>(a, wm, wr, ctas_per_sm, err, nw, s);
        return held ? launch_stream_t<1, false, true, false, WL>(a, wm, wr, ctas_per_sm, err, nw, s)
                    : launch_stream_t<1, false, false, false, WL>(a, wm, wr, ctas_per_sm, err, nw, s);
    }
    if (react) return held ? launch_stream_t<2, true, true, false, WL>(a, wm, wr, ctas_per_sm, err, nw, s)
                           : launch_stream_t<2, true, false, false, WL>(a, wm, wr, ctas_per_sm, err, nw, s);
    return held ? launch_stream_t<2, false, true, false, WL>(a, wm, wr, ctas_per_sm, err, nw, s)
                : launch_stream_t<2, false, false, false, WL>(a, wm, wr, ctas_per_sm, err, nw, s);
}

cudaError_t launch_step_stream(const StepArgs &a, sbg_grid g, int ns, bool react, int ctas_per_sm,
                               cudaStream_t s) {
    if (a.items) return launch_step_stream_t<true>(a, g, ns, react, ctas_per_sm, s);
    return launch_step_stream_t<false>(a, g, ns, react, ctas_per_sm, s);
}


}  // namespace sbg
