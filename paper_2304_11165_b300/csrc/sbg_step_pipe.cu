// Pipelined persistent kernels for FP32 arrays: the forward step of FP32 and
// compensated-FP32 states, and the adjoint step.
//
// Why: one thread per voxel with one 4-byte load each keeps only ~8 KB in
// flight per SM, far below what HBM3e needs (~40 KB per SM at ~800 ns), and a
// 7-point stencil on B300 has a budget of only ~40 issued instructions per
// FP32 voxel update before the SM, not HBM, is the limit.  So:
//  - persistent CTAs (several per SM) each walk a contiguous range of
//    "groups" of the block list (a group = 512 voxels: one 8^3 block or eight
//    4^3 blocks, contiguous in memory; 1024 for the two-row kernel below);
//  - one thread streams groups into an S-stage shared-memory ring with 1-D
//    bulk copies (cp.async.bulk, TMA engine) completing on per-stage
//    mbarriers, S groups ahead of the compute; only that thread waits on the
//    barrier, the others sleep in __syncthreads;
//  - each thread updates four x-consecutive voxels;
//  - the one-voxel face halos come from the neighbouring blocks (mostly L2
//    hits): each thread fetches the halo values of its own row into its own
//    slots of a halo buffer, so that every neighbour of its row is at a
//    per-thread constant offset from either the stage's tile or the halo
//    buffer (16-byte shared loads, no position-dependent selects of values);
//    a thread reads back only the slots it wrote itself, so the halo needs no
//    CTA barrier.  Halo variants (HV): 0 loads a group's halo into registers
//    when the group comes up and parks it after the stage wait; 1 prefetches
//    it one group ahead in registers; 2 copies it one group ahead with
//    per-thread cp.async into the other half of a double halo buffer and
//    waits for its own copies (cp.async.wait_group) before the stage barrier;
//  - results leave as one 16-byte store per thread and array.
// Every wait on an mbarrier is bounded: on time-out the CTA sets the grid's
// error word (reported as SBG_ERR_TIMEOUT), waits (bounded) for its copies in
// flight and exits.
//
// Modes (the arrays streamed per group, in order):
//  kFwd  NS species u_s                        -> u_s'           (FP32 state)
//  kX2   hi, lo                                -> hi', lo'       (compensated state)
//  kAdj  lambda_s^{n+1} (NS), u_s^n (NS)       -> lambda_s^n     (adjoint step)
//  kSrc  d, r (r without halo)                 -> d'             (SBG_F32R correction)
//  kInh  u, eps                                -> u'             (inhomogeneous diffusion)
// The per-voxel arithmetic is that of the plain kernels (sbg_step.cu), with
// the rounding of every operation pinned, so both give bitwise equal states.
#include <cstring>

#include "sbg_ptx.cuh"
#include "sbg_adj_row.cuh"
#include "sbg_step.cuh"

namespace sbg {

constexpr int kPipeThreads = 128;
constexpr int kGroupVox = 512;

enum PipeMode : int { kFwd = 0, kX2 = 1, kAdj = 2, kSrc = 3, kInh = 4 };

template <int MODE, int NS>
struct PipeShape {
    static constexpr int NA = MODE == kFwd ? NS : MODE == kAdj ? 2 * NS : 2;  // arrays streamed
    static constexpr int NH = MODE == kSrc ? 1 : NA;                          // the first NH have halos
    static constexpr int NO = MODE == kX2 ? 2 : (MODE == kSrc || MODE == kInh) ? 1 : NS;  // arrays written
};

__device__ __forceinline__ float f4get(const float4 &v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Shared memory of one CTA: an S-stage ring of groups (NA arrays of 512
// voxels each, written by the bulk copies) and one halo buffer with a B x B
// face per block of the group and face direction, per array (written by the
// threads: each thread writes the halo values of its own row into its own
// halo slots and reads them back itself, so they need no extra barrier; one
// buffer serves every stage because a thread parks a group's halo values only
// after it finished its previous group).  One more CTA per SM fits than with
// a halo buffer per stage, which measured faster than the saved selects.
template <int B>
struct PipeLayout {
    static constexpr int B3 = B * B * B;
    static constexpr int G = kGroupVox / B3;
    static constexpr int kHalo = G * 6 * B * B;  // floats per array
    __host__ __device__ static constexpr int face(int j, int f) { return (j * 6 + f) * B * B; }
};

template <int MODE, int B, int NS, bool REACT, int HV>
struct PipeSmem {
    static constexpr int NA = PipeShape<MODE, NS>::NA;
    static constexpr int NH = PipeShape<MODE, NS>::NH;
    static constexpr int G = kGroupVox / (B * B * B);
    static constexpr int kHaloBufs = HV == 2 ? 2 : 1;
    // floats after the stage ring: halo buffer(s), then (HV 2) the row weights [2][512]
    static constexpr int kHaloFloats = kHaloBufs * NH * PipeLayout<B>::kHalo;
    static constexpr int kWFloats = (HV == 2 && REACT) ? 2 * kGroupVox : 0;
    __host__ __device__ static constexpr size_t floats(int S) {
        return (size_t)S * NA * kGroupVox + kHaloFloats + kWFloats;
    }
    __host__ __device__ static constexpr size_t bytes(int S) { return floats(S) * sizeof(float) + S * sizeof(uint64_t); }
};

template <int MODE, int B, int NS, bool REACT, int S, int MINB, int HV>
__global__ void __launch_bounds__(kPipeThreads, MINB) k_step_pipe(const StepArgs a, const PipeIO io, int *err) {
    constexpr bool PF = HV == 1;
    using SM = PipeSmem<MODE, B, NS, REACT, HV>;
    using L = PipeLayout<B>;
    constexpr int B3 = L::B3;
    constexpr int G = L::G;
    constexpr int NA = PipeShape<MODE, NS>::NA;
    constexpr int NH = PipeShape<MODE, NS>::NH;
    constexpr int NO = PipeShape<MODE, NS>::NO;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *stages = reinterpret_cast<float *>(smem_raw);                // [S][NA][512]
    float *halo = stages + (size_t)S * NA * kGroupVox;                  // [bufs][NH][kHalo]
    float *wbuf = halo + SM::kHaloFloats;                               // HV 2, REACT: [2][512]
    uint64_t *full = reinterpret_cast<uint64_t *>(stages + SM::floats(S));

    const int tid = threadIdx.x;
    // work items: consecutive groups of the block list, or an explicit list
    // of (first block, block count) spans (the batch solver's active set)
    // (the launcher guarantees nb * B^3 < 2^31, so block ids, group indices
    // and voxel slots fit 32-bit ints)
    const int nb = (int)a.nb;
    const int ngroups = a.items ? (int)a.nitems : (nb + G - 1) / G;
    const int g0 = (int)((int64_t)ngroups * blockIdx.x / gridDim.x);
    const int g1 = (int)((int64_t)ngroups * (blockIdx.x + 1) / gridDim.x);
    if (g0 >= g1) return;  // uniform over the CTA
    auto span = [&](int gi, int &b0, int &nblk) {
        if (a.items) {
            b0 = (int)__ldg(a.items + 2 * gi);
            nblk = (int)__ldg(a.items + 2 * gi + 1);
        } else {
            b0 = gi * G;
            nblk = (nb - b0 < G) ? (nb - b0) : G;
        }
    };

    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();

    auto issue = [&](int gi, int s) {
        if (gi == a.stall_group) return;  // test hook: this stage never completes
        int b0, nblk;
        span(gi, b0, nblk);
        const uint32_t bytes = (uint32_t)(nblk * B3 * sizeof(float));
        mbar_arrive_expect_tx(&full[s], bytes * NA);
#pragma unroll
        for (int k = 0; k < NA; ++k)
            bulk_g2s(stages + ((size_t)s * NA + k) * kGroupVox, io.src[k] + b0 * B3, bytes, &full[s]);
    };
    if (tid == 0)
        for (int s = 0; s < S && g0 + s < g1; ++s) issue(g0 + s, s);

    // this thread's voxels: v0 .. v0 + 3 (x0 .. x0 + 3 of one row) in block j of the group
    const int v0 = 4 * tid;
    const int j = v0 / B3;
    const int l0 = v0 - j * B3;
    const int x0 = (B == 4) ? 0 : l0 % B;  // a B = 4 row is the whole x extent of its block
    const int y = (l0 / B) % B, z = l0 / (B * B);
    const bool hxm = (x0 == 0), hxp = (x0 + 3 == B - 1);  // which neighbours are halo values
    const bool hym = (y == 0), hyp = (y == B - 1), hzm = (z == 0), hzp = (z == B - 1);
    // where, in the neighbouring block, this thread's halo values are
    const int oxm = l0 + (B - 1), oxp = l0 + 3 - (B - 1);
    const int oy = hym ? l0 + (B - 1) * B : l0 - (B - 1) * B;
    const int oz = hzm ? l0 + (B - 1) * B * B : l0 - (B - 1) * B * B;
    const int fyy = hym ? 2 : 3, fzz = hzm ? 4 : 5;
    // neighbour offsets: in the halo buffer when the neighbour is a halo
    // value, else in the stage's tile
    const int sxm = hxm ? L::face(j, 0) + z * B + y : v0 - 1;
    const int sxp = hxp ? L::face(j, 1) + z * B + y : v0 + 4;
    const int sym = hym ? L::face(j, 2) + z * B + x0 : v0 - B;
    const int syp = hyp ? L::face(j, 3) + z * B + x0 : v0 + B;
    const int szm = hzm ? L::face(j, 4) + y * B + x0 : v0 - B * B;
    const int szp = hzp ? L::face(j, 5) + y * B + x0 : v0 + B * B;
    const int shy = hym ? sym : syp;
    const int shz = hzm ? szm : szp;
    const bool dy = hym || hyp, dz = hzm || hzp;
    // one haloed array: the four halo base pointers of this thread, once
    const float *hp[4] = {io.src[0] + oxm, io.src[0] + oxp, io.src[0] + oy, io.src[0] + oz};

    struct Ids {
        int xm, xp, y, z, ws;
        uint32_t hb;  // held bits of this thread's four voxels (Dirichlet faces)
    };
    struct Halo {
        float vxm[NH], vxp[NH];
        float4 vy[NH], vz[NH];
        float4 w;
        int ixm, ixp;  // x neighbour inside the group: its offset in the stage tile, else -1
        uint32_t hb;   // held bits of the row
    };
    auto load_ids = [&](int gi) {
        Ids r{-1, -1, -1, -1, -1, 0u};
        if (gi >= g1) return r;
        int b0, nblk;
        span(gi, b0, nblk);
        const int b = b0 + j;
        if (j < nblk) {
            const int32_t *f = a.face + 6 * b;
            if (hxm) r.xm = __ldg(f + 0);
            if (hxp) r.xp = __ldg(f + 1);
            if (dy) r.y = __ldg(f + fyy);
            if (dz) r.z = __ldg(f + fzz);
            if (REACT) r.ws = __ldg(a.wslab + b);
            if (a.held_mask) {
                constexpr int W = (B3 + 63) / 64;
                const uint64_t word = __ldg(reinterpret_cast<const unsigned long long *>(a.heldbits) + b * W + (l0 >> 6));
                r.hb = (uint32_t)(word >> (l0 & 63)) & 0xFu;
            }
        }
        return r;
    };
    // halo values of this thread's row, its surface weights and block coordinates
    auto load_halo = [&](int gi, const Ids &id, Halo &h) {
        // an x neighbour in the same group (the list is in tiled, x-fastest
        // order, so most are) is read from the stage tile instead
        int b0 = 0, nblk = 0;
        if (gi < g1) span(gi, b0, nblk);
        h.ixm = (hxm && (unsigned)(id.xm - b0) < (unsigned)nblk) ? (id.xm - b0) * B3 + oxm : -1;
        h.ixp = (hxp && (unsigned)(id.xp - b0) < (unsigned)nblk) ? (id.xp - b0) * B3 + oxp : -1;
        const float SENT = sentinel_f32();
#pragma unroll
        for (int k = 0; k < NH; ++k) {
            // the compensated lo part and the diffusivity factor of an absent block read 0
            const float absent = ((MODE == kX2 || MODE == kInh) && k == 1) ? 0.f : SENT;
            // this thread's halo addresses are fixed offsets from neighbour block
            // starts: one wide multiply-add per load
            const float *pxm = (NH == 1 ? hp[0] : io.src[k] + oxm), *pxp = (NH == 1 ? hp[1] : io.src[k] + oxp);
            const float *py = (NH == 1 ? hp[2] : io.src[k] + oy), *pz = (NH == 1 ? hp[3] : io.src[k] + oz);
            h.vxm[k] = (id.xm >= 0 && h.ixm < 0) ? __ldg(pxm + id.xm * B3) : absent;
            h.vxp[k] = (id.xp >= 0 && h.ixp < 0) ? __ldg(pxp + id.xp * B3) : absent;
            h.vy[k] = (id.y >= 0) ? __ldg(reinterpret_cast<const float4 *>(py + id.y * B3))
                                  : make_float4(absent, absent, absent, absent);
            h.vz[k] = (id.z >= 0) ? __ldg(reinterpret_cast<const float4 *>(pz + id.z * B3))
                                  : make_float4(absent, absent, absent, absent);
        }
        h.w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (REACT && id.ws >= 0) h.w = __ldg(reinterpret_cast<const float4 *>(a.w + (int64_t)id.ws * B3 + l0));
        h.hb = id.hb;
    };
    // park this thread's halo values in its own slots of the halo buffer
    auto park = [&](const Halo &h) {
#pragma unroll
        for (int k = 0; k < NH; ++k) {
            float *hb = halo + k * L::kHalo;
            if (hxm && h.ixm < 0) hb[sxm] = h.vxm[k];
            if (hxp && h.ixp < 0) hb[sxp] = h.vxp[k];
            if (dy) *reinterpret_cast<float4 *>(hb + shy) = h.vy[k];
            if (dz) *reinterpret_cast<float4 *>(hb + shz) = h.vz[k];
        }
    };

    // HV 2: cp.async copies of group gi's halo values (ids `id`), row weights
    // and block coordinates into buffer `buf`, as one commit group per call
    // (an empty group past the end, so every group has one)
    uint32_t hbq0 = 0u, hbq1 = 0u;  // HV 2: held bits of the groups in the two halo buffers
    auto issue_async = [&](int gi, const Ids &id, int buf) {
        if (HV != 2) return;
        if (buf) hbq1 = id.hb;
        else hbq0 = id.hb;
        if (gi < g1) {
            int b0, nblk;
            span(gi, b0, nblk);
            if (j < nblk) {
                const float SENT = sentinel_f32();
#pragma unroll
                for (int k = 0; k < NH; ++k) {
                    const float absent = ((MODE == kX2 || MODE == kInh) && k == 1) ? 0.f : SENT;
                    const float *sk = io.src[k];
                    float *hb = halo + ((size_t)buf * NH + k) * L::kHalo;
                    if (hxm) {
                        if (id.xm >= 0) cp_async4(hb + sxm, sk + (int64_t)id.xm * B3 + oxm);
                        else hb[sxm] = absent;
                    }
                    if (hxp) {
                        if (id.xp >= 0) cp_async4(hb + sxp, sk + (int64_t)id.xp * B3 + oxp);
                        else hb[sxp] = absent;
                    }
                    if (dy) {
                        if (id.y >= 0) cp_async16(hb + shy, sk + (int64_t)id.y * B3 + oy);
                        else *reinterpret_cast<float4 *>(hb + shy) = make_float4(absent, absent, absent, absent);
                    }
                    if (dz) {
                        if (id.z >= 0) cp_async16(hb + shz, sk + (int64_t)id.z * B3 + oz);
                        else *reinterpret_cast<float4 *>(hb + shz) = make_float4(absent, absent, absent, absent);
                    }
                }
                if (REACT) {
                    float *wb = wbuf + buf * kGroupVox + v0;
                    if (id.ws >= 0) cp_async16(wb, a.w + (int64_t)id.ws * B3 + l0);
                    else *reinterpret_cast<float4 *>(wb) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
        }
        cp_async_commit();
    };

    // adjoint: this thread's gradient sums, double-float (hi, lo) per quantity
    float gh[3] = {0.f, 0.f, 0.f}, gl[3] = {0.f, 0.f, 0.f};

    // One group.  PF: park this group's halo values (prefetched during the
    // previous group), prefetch the next group's (ids read a group earlier).
    // !PF: load this group's halo values now (ids read during the previous
    // group) and park them after the stage wait, relying on the other CTAs of
    // the SM to hide their latency.  The loop below is unrolled by two with
    // the register sets swapped, so no prefetched value is copied (a copy
    // would wait for the load every group).
    auto body = [&](int gi, int it, Halo &cur, Halo &nxt, const Ids &id1, Ids &id2) -> bool {
        const int s = it % S;
        const uint32_t par = (uint32_t)((it / S) & 1);
        int b0, nblk;
        span(gi, b0, nblk);
        const int b = b0 + j;
        const bool valid = j < nblk;
        if (HV == 2) {
            // the next group's halo into the other buffer (ids read a group
            // earlier), ids two groups ahead, then this group's own copies
            issue_async(gi + 1, id1, (it + 1) & 1);
            id2 = load_ids(gi + 2);
            cp_async_wait_group<1>();
        } else if (PF) {
            if (valid) park(cur);
            id2 = load_ids(gi + 2);
            load_halo(gi + 1, id1, nxt);
        } else {
            load_halo(gi, id1, cur);
            id2 = load_ids(gi + 1);
        }

        bool ok = true;
        if (tid == 0) ok = mbar_wait_bounded(&full[s], par, a.wait_cycles);
        if (__syncthreads_or(!ok)) {
            if (HV == 2) cp_async_wait_all();
            if (tid == 0) {
                atomicExch(err, (int)SBG_ERR_TIMEOUT);
                for (int q = it; q < it + S && g0 + q < g1; ++q)
                    mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1), min(a.wait_cycles, 1ll << 28));
            }
            return false;
        }
        mbar_try_wait(&full[s], par);  // completed: gives this thread the acquire of the copied data
        // every thread has finished the previous group: refill its stage
        if (tid == 0 && it >= 1 && gi - 1 + S < g1) issue(gi - 1 + S, (it - 1) % S);
        if (!valid) return true;
        if (HV == 0) park(cur);

        // Dirichlet-held voxels of this row (bits prepared per block for the
        // current Dirichlet faces)
        const uint32_t hbits = HV == 2 ? ((it & 1) ? hbq1 : hbq0) : cur.hb;
        bool held[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) held[i] = (hbits >> i) & 1u;
        const float4 w4 = (HV == 2 && REACT) ? *reinterpret_cast<const float4 *>(wbuf + (it & 1) * kGroupVox + v0)
                                             : cur.w;

        float4 uc[NA], ym[NH], yp[NH], zm[NH], zp[NH];
        float xm[NH], xp[NH];
#pragma unroll
        for (int k = 0; k < NA; ++k)
            uc[k] = *reinterpret_cast<const float4 *>(stages + ((size_t)s * NA + k) * kGroupVox + v0);
#pragma unroll
        for (int k = 0; k < NH; ++k) {
            const float *t = stages + ((size_t)s * NA + k) * kGroupVox;
            const float *h = halo + ((size_t)(HV == 2 ? (it & 1) : 0) * NH + k) * L::kHalo;
            const int ixm = HV == 2 ? -1 : cur.ixm, ixp = HV == 2 ? -1 : cur.ixp;
            xm[k] = ixm >= 0 ? t[ixm] : (hxm ? h : t)[sxm];
            xp[k] = ixp >= 0 ? t[ixp] : (hxp ? h : t)[sxp];
            ym[k] = *reinterpret_cast<const float4 *>((hym ? h : t) + sym);
            yp[k] = *reinterpret_cast<const float4 *>((hyp ? h : t) + syp);
            zm[k] = *reinterpret_cast<const float4 *>((hzm ? h : t) + szm);
            zp[k] = *reinterpret_cast<const float4 *>((hzp ? h : t) + szp);
        }
        const StepCoef<float> &kc = a.cf;
        float res[NO][4];
        float q[3] = {0.f, 0.f, 0.f};  // adjoint: this group's gradient terms
        // With one haloed array every voxel of the row is computed (an inactive
        // one from sentinels) and the result selected, so the row takes no
        // divergent branches; with more arrays the four interleaved updates
        // would not fit the register budget, and inactive or held voxels
        // branch around the update instead.
        constexpr bool kBranchFree = NH == 1;
        // x differences along the row, shared by neighbouring voxels (all modes
        // but the compensated one): with R = (xm, the row's four values, xp),
        // Dx[k][j] = R[j+1] - R[j]; voxel i takes (x_{i+1} - u_i) = Dx[k][i+1]
        // and (u_i - x_{i-1}) = Dx[k][i], each replaced by 0 when that
        // neighbour is outside Omega: the values the per-voxel form computes
        // from mirrored neighbours, so results stay bitwise the same.
        bool actx[6];
        float Dx[NH][5];
        if (MODE != kX2) {
            actx[0] = !is_sent(xm[0]);
            actx[5] = !is_sent(xp[0]);
#pragma unroll
            for (int i = 0; i < 4; ++i) actx[i + 1] = !is_sent(f4get(uc[0], i));
#pragma unroll
            for (int k = 0; k < NH; ++k) {
                const float R[6] = {xm[k], uc[k].x, uc[k].y, uc[k].z, uc[k].w, xp[k]};
#pragma unroll
                for (int jj = 0; jj < 5; ++jj) Dx[k][jj] = __fsub_rn(R[jj + 1], R[jj]);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            // neighbours of voxel i in array 0 decide the no-flux mirror for every array
            const float n0[6] = {i == 0 ? xm[0] : f4get(uc[0], i - 1), i == 3 ? xp[0] : f4get(uc[0], i + 1),
                                 f4get(ym[0], i), f4get(yp[0], i), f4get(zm[0], i), f4get(zp[0], i)};
            bool out[6];
#pragma unroll
            for (int f = (MODE == kX2 ? 0 : 2); f < 6; ++f) out[f] = is_sent(n0[f]);
            const float c0 = f4get(uc[0], i);
            const bool act = !is_sent(c0);
            const bool upd = act && !held[i];
            if (!kBranchFree && !upd) {
#pragma unroll
                for (int k = 0; k < NO; ++k) res[k][i] = (MODE == kAdj && act) ? 0.f : f4get(uc[k], i);
                continue;
            }
            float nv[NH][6];  // mirrored neighbours (x entries only for the compensated mode)
            float dxs[NH];    // x second differences (other modes)
#pragma unroll
            for (int k = 0; k < NH; ++k) {
                const float c = f4get(uc[k], i);
                const float raw[6] = {i == 0 ? xm[k] : f4get(uc[k], i - 1), i == 3 ? xp[k] : f4get(uc[k], i + 1),
                                      f4get(ym[k], i), f4get(yp[k], i), f4get(zm[k], i), f4get(zp[k], i)};
#pragma unroll
                for (int f = (MODE == kX2 ? 0 : 2); f < 6; ++f) nv[k][f] = out[f] ? c : raw[f];
                if (MODE != kX2) {
                    const float dp = actx[i + 2] ? Dx[k][i + 1] : 0.f;
                    const float dm = actx[i] ? Dx[k][i] : 0.f;
                    nv[k][0] = dm;  // kept for the adjoint's g(u): (x_{i-1} - u) = -dm
                    nv[k][1] = dp;
                    dxs[k] = __fsub_rn(dp, dm);
                }
            }
            float nr[NO];
            if (MODE == kX2) {
                float rate = kc.decay[0];
                if (REACT) rate = __fmaf_rn(kc.k, f4get(w4, i), rate);
                fused_update_x2(c0, f4get(uc[1], i), nv[0], nv[1], kc.c[0], kc.dt, rate, nr[0], nr[NO - 1]);
            } else if (MODE == kSrc) {
                // correction d of an SBG_F32R state: the source r = L_h b replaces
                // the base's part of the update
                float rate = kc.decay[0];
                if (REACT) rate = __fmaf_rn(kc.k, f4get(w4, i), rate);
                nr[0] = fused_update_dx(c0, dxs[0], nv[0][2], nv[0][3], nv[0][4], nv[0][5], kc.c[0], kc.dt, rate,
                                        f4get(uc[1], i));
            } else if (MODE == kInh) {
                // inhomogeneous diffusion: one-sided differences of u (0 towards
                // a neighbour outside Omega) and the raw neighbour factors
                const float dp[3] = {nv[0][1], __fsub_rn(nv[0][3], c0), __fsub_rn(nv[0][5], c0)};
                const float dm[3] = {nv[0][0], __fsub_rn(c0, nv[0][2]), __fsub_rn(c0, nv[0][4])};
                const float en[6] = {i == 0 ? xm[1] : f4get(uc[1], i - 1), i == 3 ? xp[1] : f4get(uc[1], i + 1),
                                     f4get(ym[1], i), f4get(yp[1], i), f4get(zm[1], i), f4get(zp[1], i)};
                nr[0] = inh_update(c0, dp, dm, f4get(uc[1], i), en, kc.c[0], kc.dt, kc.decay[0]);
            } else if (MODE == kFwd) {
                const float t = REACT ? __fmul_rn(__fmul_rn(kc.k, f4get(w4, i)), c0) : 0.f;
#pragma unroll
                for (int k = 0; k < NS; ++k)
                    nr[k] = fused_update_dx(f4get(uc[k], i), dxs[k], nv[k][2], nv[k][3], nv[k][4], nv[k][5],
                                            kc.c[k], kc.dt, kc.decay[k], k == 0 ? -t : t);
            } else {
                // lambda^n = M^T lambda^{n+1}: the forward stencil on lambda (held
                // voxels hold lambda = 0), with the A -> B transfer transposed
                const float kw = REACT ? __fmul_rn(kc.k, f4get(w4, i)) : 0.f;
                const float lamB = NS == 2 ? f4get(uc[1], i) : 0.f;
#pragma unroll
                for (int sp = 0; sp < NS; ++sp) {
                    const float rate = (sp == 0 && REACT) ? __fadd_rn(kc.decay[0], kw) : kc.decay[sp];
                    const float t = (sp == 0 && NS == 2 && REACT) ? __fmul_rn(kw, lamB) : 0.f;
                    nr[sp] = fused_update_dx(f4get(uc[sp], i), dxs[sp], nv[sp][2], nv[sp][3], nv[sp][4],
                                             nv[sp][5], kc.c[sp], kc.dt, rate, t);
                    // dL/dD_s += lambda_s dt g_s(u^n), g = sum_a [(u~+ - u) + (u~- - u)] / dx_a^2
                    const float u = f4get(uc[NS + sp], i);
                    const float *nu = nv[NS + sp];
                    // x part: (x_{i-1} - u) + (x_{i+1} - u) = -dm + dp (nu[0] = dm, nu[1] = dp)
                    float g = __fmul_rn(io.inv2[0], __fadd_rn(-nu[0], nu[1]));
                    g = __fmaf_rn(io.inv2[1], __fadd_rn(__fsub_rn(nu[2], u), __fsub_rn(nu[3], u)), g);
                    g = __fmaf_rn(io.inv2[2], __fadd_rn(__fsub_rn(nu[4], u), __fsub_rn(nu[5], u)), g);
                    const float term = __fmul_rn(__fmul_rn(f4get(uc[sp], i), kc.dt), g);
                    q[sp] = __fadd_rn(q[sp], upd ? term : 0.f);
                }
                if (REACT) {
                    // dL/dk += dt w u_A (lambda_B - lambda_A)
                    const float uA = f4get(uc[NS], i);
                    const float term = __fmul_rn(__fmul_rn(__fmul_rn(kc.dt, f4get(w4, i)), uA), __fsub_rn(lamB, c0));
                    q[2] = __fadd_rn(q[2], upd ? term : 0.f);
                }
            }
#pragma unroll
            for (int k = 0; k < NO; ++k)
                res[k][i] = upd ? nr[k] : ((MODE == kAdj && act) ? 0.f : f4get(uc[k], i));
        }
        if (MODE == kAdj) {
#pragma unroll
            for (int qq = 0; qq < 3; ++qq) df_add(gh[qq], gl[qq], q[qq], 0.f);
        }
#pragma unroll
        for (int k = 0; k < NO; ++k)
            *reinterpret_cast<float4 *>(io.dst[k] + b * B3 + l0) =
                make_float4(res[k][0], res[k][1], res[k][2], res[k][3]);
        return true;
    };

    Ids idA = load_ids(g0), idB;
    Halo hA, hB;
    if (PF) {
        load_halo(g0, idA, hA);
        idA = load_ids(g0 + 1);
    } else if (HV == 2) {
        issue_async(g0, idA, 0);
        idA = load_ids(g0 + 1);
    }
    int it = 0;
    bool ok = true;
    for (int gi = g0; gi < g1; gi += 2, it += 2) {
        if (!body(gi, it, hA, hB, idA, idB)) {
            ok = false;
            break;
        }
        if (gi + 1 >= g1) break;
        if (!body(gi + 1, it + 1, hB, hA, idB, idA)) {
            ok = false;
            break;
        }
    }
    if (HV == 2) cp_async_wait_all();  // no copy may land after the CTA's shared memory is gone
    if (MODE == kAdj && ok) {
        // CTA sums: double-float across the warp, FP64 across the warps; each
        // CTA adds to its own slot, so the order of additions is fixed
        __shared__ double red[kPipeThreads / 32][3];
#pragma unroll
        for (int qq = 0; qq < 3; ++qq) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float h2 = __shfl_down_sync(0xffffffffu, gh[qq], o);
                const float l2 = __shfl_down_sync(0xffffffffu, gl[qq], o);
                df_add(gh[qq], gl[qq], h2, l2);
            }
            if ((tid & 31) == 0) red[tid >> 5][qq] = (double)gh[qq] + (double)gl[qq];
        }
        __syncthreads();
        if (tid < 3) {
            double v = 0.0;
            for (int w = 0; w < kPipeThreads / 32; ++w) v += red[w][tid];
            io.gsum[(int64_t)blockIdx.x * 3 + tid] += v;
        }
    }
}

// ---------------------------------------------------------------------------
// Two rows per thread, for the modes with one haloed array (FP32 one species,
// SBG_F32R correction) and, with cp.async halos, two (species A and B; u and
// the diffusivity factor; the compensated hi and lo parts; the one-species
// adjoint's lambda and u^n).  Groups of 1024 voxels (sixteen 4^3 blocks or two 8^3
// blocks); each thread updates the rows (y, z0) and (y, z0 + B/2) of four
// voxels, so the per-group work (face ids, Dirichlet bits, the stage barrier,
// spans) is shared by eight voxels, and a quarter-warp's row loads cover
// consecutive rows (no shared-memory bank conflicts).  The per-voxel
// arithmetic is the same as above (bitwise).
constexpr int kGroup2 = 1024;

template <int B>
struct Rows2Layout {
    static constexpr int B3 = B * B * B;
    static constexpr int G = kGroup2 / B3;       // blocks per group
    static constexpr int TPB = B3 / 8;           // threads per block
    static constexpr int kHalo = G * 6 * B * B;  // a B x B face per block and direction
    __host__ __device__ static constexpr int face(int j, int f) { return (j * 6 + f) * B * B; }
};

// New values of one row of four voxels (u), given its mirrored-or-not
// neighbours; hb: held bits of the row; src: the SBG_F32R source r.
template <int MODE, bool REACT>
__device__ __forceinline__ float4 row_update(const float4 u, float xm, float xp, const float4 ym, const float4 yp,
                                             const float4 zm, const float4 zp, const float4 src, const float4 w4,
                                             uint32_t hb, const StepCoef<float> &kc) {
    bool actx[6];
    actx[0] = !is_sent(xm);
    actx[5] = !is_sent(xp);
#pragma unroll
    for (int i = 0; i < 4; ++i) actx[i + 1] = !is_sent(f4get(u, i));
    const float R[6] = {xm, u.x, u.y, u.z, u.w, xp};
    float Dx[5];
#pragma unroll
    for (int jj = 0; jj < 5; ++jj) Dx[jj] = __fsub_rn(R[jj + 1], R[jj]);
    float res[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float c = f4get(u, i);
        const float yv[4] = {f4get(ym, i), f4get(yp, i), f4get(zm, i), f4get(zp, i)};
        float nv[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) nv[f] = is_sent(yv[f]) ? c : yv[f];
        const float dp = actx[i + 2] ? Dx[i + 1] : 0.f;
        const float dm = actx[i] ? Dx[i] : 0.f;
        const float dxs = __fsub_rn(dp, dm);
        float nr;
        if (MODE == kSrc) {
            float rate = kc.decay[0];
            if (REACT) rate = __fmaf_rn(kc.k, f4get(w4, i), rate);
            nr = fused_update_dx(c, dxs, nv[0], nv[1], nv[2], nv[3], kc.c[0], kc.dt, rate, f4get(src, i));
        } else {
            const float t = REACT ? __fmul_rn(__fmul_rn(kc.k, f4get(w4, i)), c) : 0.f;
            nr = fused_update_dx(c, dxs, nv[0], nv[1], nv[2], nv[3], kc.c[0], kc.dt, kc.decay[0], -t);
        }
        const bool upd = actx[i + 1] && !((hb >> i) & 1u);
        res[i] = upd ? nr : c;
    }
    return make_float4(res[0], res[1], res[2], res[3]);
}

// One row of one array with its neighbour values as read (sentinels where a
// neighbour is outside Omega or its block is absent).
// Two species A (v0) and B (v1) with the surface transfer k w A: A loses it,
// B gains it.  Which neighbours are outside Omega is read from species A for
// both species, as in the one-row kernel.
template <bool REACT>
__device__ __forceinline__ void row_update_fwd2(const RowVals &v0, const RowVals &v1, const float4 w4, uint32_t hb,
                                                const StepCoef<float> &kc, float4 &o0, float4 &o1) {
    bool actx[6];
    actx[0] = !is_sent(v0.xm);
    actx[5] = !is_sent(v0.xp);
#pragma unroll
    for (int i = 0; i < 4; ++i) actx[i + 1] = !is_sent(f4get(v0.u, i));
    float D0[5], D1[5];
    row_dx(v0, D0);
    row_dx(v1, D1);
    float r0[4], r1[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float c0 = f4get(v0.u, i), c1 = f4get(v1.u, i);
        const float y0[4] = {f4get(v0.ym, i), f4get(v0.yp, i), f4get(v0.zm, i), f4get(v0.zp, i)};
        const float y1[4] = {f4get(v1.ym, i), f4get(v1.yp, i), f4get(v1.zm, i), f4get(v1.zp, i)};
        float n0[4], n1[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const bool out = is_sent(y0[f]);
            n0[f] = out ? c0 : y0[f];
            n1[f] = out ? c1 : y1[f];
        }
        const float dxs0 = __fsub_rn(actx[i + 2] ? D0[i + 1] : 0.f, actx[i] ? D0[i] : 0.f);
        const float dxs1 = __fsub_rn(actx[i + 2] ? D1[i + 1] : 0.f, actx[i] ? D1[i] : 0.f);
        const float t = REACT ? __fmul_rn(__fmul_rn(kc.k, f4get(w4, i)), c0) : 0.f;
        const float nr0 = fused_update_dx(c0, dxs0, n0[0], n0[1], n0[2], n0[3], kc.c[0], kc.dt, kc.decay[0], -t);
        const float nr1 = fused_update_dx(c1, dxs1, n1[0], n1[1], n1[2], n1[3], kc.c[1], kc.dt, kc.decay[1], t);
        const bool upd = actx[i + 1] && !((hb >> i) & 1u);
        r0[i] = upd ? nr0 : c0;
        r1[i] = upd ? nr1 : c1;
    }
    o0 = make_float4(r0[0], r0[1], r0[2], r0[3]);
    o1 = make_float4(r1[0], r1[1], r1[2], r1[3]);
}

// Compensated state (hi: v0, lo: v1): every neighbour outside Omega (read from
// hi, x included) mirrored in both parts, the update of fused_update_x2.
template <bool REACT>
__device__ __forceinline__ void row_update_x2(const RowVals &v0, const RowVals &v1, const float4 w4, uint32_t hb,
                                              const StepCoef<float> &kc, float4 &o0, float4 &o1) {
    float r0[4], r1[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float c0 = f4get(v0.u, i), c1 = f4get(v1.u, i);
        const float h[6] = {i == 0 ? v0.xm : f4get(v0.u, i - 1), i == 3 ? v0.xp : f4get(v0.u, i + 1),
                            f4get(v0.ym, i), f4get(v0.yp, i), f4get(v0.zm, i), f4get(v0.zp, i)};
        const float l[6] = {i == 0 ? v1.xm : f4get(v1.u, i - 1), i == 3 ? v1.xp : f4get(v1.u, i + 1),
                            f4get(v1.ym, i), f4get(v1.yp, i), f4get(v1.zm, i), f4get(v1.zp, i)};
        float nh[6], nl[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const bool out = is_sent(h[f]);
            nh[f] = out ? c0 : h[f];
            nl[f] = out ? c1 : l[f];
        }
        float rate = kc.decay[0];
        if (REACT) rate = __fmaf_rn(kc.k, f4get(w4, i), rate);
        float rh, rl;
        fused_update_x2(c0, c1, nh, nl, kc.c[0], kc.dt, rate, rh, rl);
        const bool upd = !is_sent(c0) && !((hb >> i) & 1u);
        r0[i] = upd ? rh : c0;
        r1[i] = upd ? rl : c1;
    }
    o0 = make_float4(r0[0], r0[1], r0[2], r0[3]);
    o1 = make_float4(r1[0], r1[1], r1[2], r1[3]);
}

// Inhomogeneous diffusion (Eq. 6 factor e, v1): one-sided differences of u
// (v0; 0 towards a neighbour outside Omega) and the neighbours' raw factors.
__device__ __forceinline__ float4 row_update_inh(const RowVals &v0, const RowVals &v1, uint32_t hb,
                                                 const StepCoef<float> &kc) {
    bool actx[6];
    actx[0] = !is_sent(v0.xm);
    actx[5] = !is_sent(v0.xp);
#pragma unroll
    for (int i = 0; i < 4; ++i) actx[i + 1] = !is_sent(f4get(v0.u, i));
    float D0[5];
    row_dx(v0, D0);
    float res[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float c = f4get(v0.u, i);
        const float yv[4] = {f4get(v0.ym, i), f4get(v0.yp, i), f4get(v0.zm, i), f4get(v0.zp, i)};
        float nv[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) nv[f] = is_sent(yv[f]) ? c : yv[f];
        const float dp[3] = {actx[i + 2] ? D0[i + 1] : 0.f, __fsub_rn(nv[1], c), __fsub_rn(nv[3], c)};
        const float dm[3] = {actx[i] ? D0[i] : 0.f, __fsub_rn(c, nv[0]), __fsub_rn(c, nv[2])};
        const float en[6] = {i == 0 ? v1.xm : f4get(v1.u, i - 1), i == 3 ? v1.xp : f4get(v1.u, i + 1),
                             f4get(v1.ym, i), f4get(v1.yp, i), f4get(v1.zm, i), f4get(v1.zp, i)};
        const float nr = inh_update(c, dp, dm, f4get(v1.u, i), en, kc.c[0], kc.dt, kc.decay[0]);
        const bool upd = actx[i + 1] && !((hb >> i) & 1u);
        res[i] = upd ? nr : c;
    }
    return make_float4(res[0], res[1], res[2], res[3]);
}

// AH: halo values copied one group ahead with per-thread cp.async into the
// other half of a double halo buffer (no registers held across the group).
// WL: the groups come from a work list (a separate instance, so that the
// plain walk over the block list keeps its registers).
// NH: arrays streamed, each with halos: 1 (u, or the SBG_F32R correction d,
// whose source r is read per row from global memory) or 2 (species A and B,
// u and the diffusivity factor, hi and lo, or the adjoint's lambda and u^n).  With two arrays the surface weights are read
// per row from global memory too: without a weight buffer one more CTA fits
// in an SM's shared memory.
template <int MODE, int NH, int B, bool REACT, int S, int MINB, bool AH, bool WL>
__global__ void __launch_bounds__(kPipeThreads, MINB) k_step_rows2(const StepArgs a, const PipeIO io, int *err) {
    using L = Rows2Layout<B>;
    constexpr int B3 = L::B3;
    constexpr int G = L::G;
    constexpr int TPB = L::TPB;
    constexpr int NA = NH;
    constexpr bool WSM = AH && REACT && NH == 1;  // row weights staged in shared memory by cp.async
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *stages = reinterpret_cast<float *>(smem_raw);  // [S][NA][1024]
    float *halo = stages + (size_t)S * NA * kGroup2;      // [AH ? 2 : 1][NH][kHalo]
    float *wbuf = halo + (AH ? 2 : 1) * NH * L::kHalo;    // WSM: [2][1024] row weights
    uint64_t *full = reinterpret_cast<uint64_t *>(wbuf + (WSM ? 2 * kGroup2 : 0));

    const int tid = threadIdx.x;
    // (the launcher guarantees nb * B^3 < 2^31: 32-bit block ids and slots)
    const int nb = (int)a.nb;
    // groups: consecutive G-block spans of the block list, or an explicit list of
    // (first block, block count <= G) spans (the batch solver's active set)
    const int ngroups = WL ? (int)a.nitems : (nb + G - 1) / G;
    const int g0 = (int)((int64_t)ngroups * blockIdx.x / gridDim.x);
    const int g1 = (int)((int64_t)ngroups * (blockIdx.x + 1) / gridDim.x);
    if (g0 >= g1) return;  // uniform over the CTA
    auto span = [&](int gi, int &b0, int &nblk) {
        if (WL) {
            b0 = (int)__ldg(a.items + 2 * gi);
            nblk = (int)__ldg(a.items + 2 * gi + 1);
        } else {
            b0 = gi * G;
            nblk = (nb - b0 < G) ? (nb - b0) : G;
        }
    };
    if (tid == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        fence_barrier_init();
    }
    __syncthreads();
    auto issue = [&](int gi, int s) {
        if (gi == a.stall_group) return;  // test hook: this stage never completes
        int b0, nblk;
        span(gi, b0, nblk);
        const uint32_t bytes = (uint32_t)(nblk * B3 * sizeof(float));
        mbar_arrive_expect_tx(&full[s], bytes * NA);
#pragma unroll
        for (int k = 0; k < NA; ++k)
            bulk_g2s(stages + ((size_t)s * NA + k) * kGroup2, io.src[k] + b0 * B3, bytes, &full[s]);
    };
    if (tid == 0)
        for (int s = 0; s < S && g0 + s < g1; ++s) issue(g0 + s, s);

    // this thread's rows: a = (y, z0) and b = (y, z0 + B/2), x0 .. x0 + 3, of block j.  With
    // z0 < B/2 the eight threads of a quarter-warp hold eight consecutive rows, so each
    // 16-byte row load from the stage tile touches every shared-memory bank once.
    constexpr int ZB = (B / 2) * B * B;  // row b = row a + ZB in the block
    constexpr int HB = (B / 2) * B;      // row b's slot = row a's + HB in the x and y halo faces
    const int j = tid / TPB, r = tid % TPB;
    const int x0 = (B == 4) ? 0 : (r & 1) * 4;
    const int rr = (B == 4) ? r : (r >> 1);
    const int y = rr % B, z0 = rr / B;
    const int la = (z0 * B + y) * B + x0;  // row a in its block
    const int va = j * B3 + la;            // row a in the group tile
    const bool hxm = (x0 == 0), hxp = (x0 + 3 == B - 1);
    const bool hym = (y == 0), hyp = (y == B - 1);             // both rows
    const bool hzm = (z0 == 0), hzp = (z0 + B / 2 == B - 1);  // row a below, row b above
    // offsets of this thread's halo values in the neighbour blocks (row a; row b at + ZB)
    const int oxm = la + (B - 1), oxp = la + 3 - (B - 1);
    const int oym = la + (B - 1) * B;           // y- neighbour row (y = B - 1)
    const int oyp = la - (B - 1) * B;           // y+ neighbour row (y = 0)
    const int ozm = la + (B - 1) * B * B;       // row a's z- neighbour row (z = B - 1)
    const int ozp = la + ZB - (B - 1) * B * B;  // row b's z+ neighbour row (z = 0)
    // halo slots: x faces indexed z*B + y, y faces z*B + x, z faces y*B + x
    const int sxm = L::face(j, 0) + z0 * B + y, sxp = L::face(j, 1) + z0 * B + y;
    const int sym = L::face(j, 2) + z0 * B + x0, syp = L::face(j, 3) + z0 * B + x0;
    const int szm = L::face(j, 4) + y * B + x0, szp = L::face(j, 5) + y * B + x0;

    struct Ids {
        int xm, xp, ym, yp, zm, zp, ws;
        uint32_t hb;  // held bits: row a in bits 0-3, row b in bits 4-7
    };
    struct Halo {
        float vxm[NH][2], vxp[NH][2];
        float4 vym[NH][2], vyp[NH][2], vzm[NH], vzp[NH];
        float4 w[2];
        int ixm, ixp;  // x neighbour inside the group: row a's offset in the stage tile, else -1
        uint32_t hb;
    };
    auto load_ids = [&](int gi) {
        Ids q{-1, -1, -1, -1, -1, -1, -1, 0u};
        if (gi >= g1) return q;
        int b0, nblk;
        span(gi, b0, nblk);
        const int b = b0 + j;
        if (j < nblk) {
            const int32_t *f = a.face + 6 * b;
            if (hxm) q.xm = __ldg(f + 0);
            if (hxp) q.xp = __ldg(f + 1);
            if (hym) q.ym = __ldg(f + 2);
            if (hyp) q.yp = __ldg(f + 3);
            if (hzm) q.zm = __ldg(f + 4);
            if (hzp) q.zp = __ldg(f + 5);
            if (REACT) q.ws = __ldg(a.wslab + b);
            if (a.held_mask) {
                constexpr int W = (B3 + 63) / 64;
                const unsigned long long *hw = reinterpret_cast<const unsigned long long *>(a.heldbits) + b * W;
                const uint64_t wa = __ldg(hw + (la >> 6));
                const uint64_t wb = (B == 4) ? wa : __ldg(hw + ((la + ZB) >> 6));
                q.hb = ((uint32_t)(wa >> (la & 63)) & 0xFu) | (((uint32_t)(wb >> ((la + ZB) & 63)) & 0xFu) << 4);
            }
        }
        return q;
    };
    auto load_halo = [&](int gi, const Ids &id, Halo &h) {
        int b0 = 0, nblk = 0;
        if (gi < g1) span(gi, b0, nblk);
        h.ixm = (hxm && (unsigned)(id.xm - b0) < (unsigned)nblk) ? (id.xm - b0) * B3 + oxm : -1;
        h.ixp = (hxp && (unsigned)(id.xp - b0) < (unsigned)nblk) ? (id.xp - b0) * B3 + oxp : -1;
#pragma unroll
        for (int k = 0; k < NH; ++k) {
            const float *sk = io.src[k];
            // the diffusivity factor and the compensated lo part of an absent block read 0
            const float ab = ((MODE == kInh || MODE == kX2) && k == 1) ? 0.f : sentinel_f32();
            const float4 ab4 = make_float4(ab, ab, ab, ab);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                h.vxm[k][q] = (id.xm >= 0 && h.ixm < 0) ? __ldg(sk + id.xm * B3 + oxm + q * ZB) : ab;
                h.vxp[k][q] = (id.xp >= 0 && h.ixp < 0) ? __ldg(sk + id.xp * B3 + oxp + q * ZB) : ab;
                h.vym[k][q] = (id.ym >= 0) ? __ldg(reinterpret_cast<const float4 *>(sk + id.ym * B3 + oym + q * ZB)) : ab4;
                h.vyp[k][q] = (id.yp >= 0) ? __ldg(reinterpret_cast<const float4 *>(sk + id.yp * B3 + oyp + q * ZB)) : ab4;
            }
            h.vzm[k] = (id.zm >= 0) ? __ldg(reinterpret_cast<const float4 *>(sk + id.zm * B3 + ozm)) : ab4;
            h.vzp[k] = (id.zp >= 0) ? __ldg(reinterpret_cast<const float4 *>(sk + id.zp * B3 + ozp)) : ab4;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            h.w[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (REACT && id.ws >= 0) h.w[q] = __ldg(reinterpret_cast<const float4 *>(a.w + id.ws * B3 + la + q * ZB));
        }
        h.hb = id.hb;
    };
    auto park = [&](const Halo &h) {
#pragma unroll
        for (int k = 0; k < NH; ++k) {
            float *hk = halo + k * L::kHalo;
            if (hxm && h.ixm < 0) {
                hk[sxm] = h.vxm[k][0];
                hk[sxm + HB] = h.vxm[k][1];
            }
            if (hxp && h.ixp < 0) {
                hk[sxp] = h.vxp[k][0];
                hk[sxp + HB] = h.vxp[k][1];
            }
            if (hym) {
                *reinterpret_cast<float4 *>(hk + sym) = h.vym[k][0];
                *reinterpret_cast<float4 *>(hk + sym + HB) = h.vym[k][1];
            }
            if (hyp) {
                *reinterpret_cast<float4 *>(hk + syp) = h.vyp[k][0];
                *reinterpret_cast<float4 *>(hk + syp + HB) = h.vyp[k][1];
            }
            if (hzm) *reinterpret_cast<float4 *>(hk + szm) = h.vzm[k];
            if (hzp) *reinterpret_cast<float4 *>(hk + szp) = h.vzp[k];
        }
    };

    // AH: per halo buffer, the row's x offsets inside the group, held bits and
    // (two arrays) the group's weight slab
    int aixm0 = -1, aixm1 = -1, aixp0 = -1, aixp1 = -1, aws0 = -1, aws1 = -1;
    uint32_t ahb0 = 0u, ahb1 = 0u;
    auto issue_async = [&](int gi, const Ids &id, int buf) {
        if (!AH) return;
        int ixm = -1, ixp = -1;
        if (gi < g1) {
            int b0, nblk;
            span(gi, b0, nblk);
            if (j < nblk) {
                ixm = (hxm && (unsigned)(id.xm - b0) < (unsigned)nblk) ? (id.xm - b0) * B3 + oxm : -1;
                ixp = (hxp && (unsigned)(id.xp - b0) < (unsigned)nblk) ? (id.xp - b0) * B3 + oxp : -1;
#pragma unroll
                for (int k = 0; k < NH; ++k) {
                    const float *sk = io.src[k];
                    const float ab = ((MODE == kInh || MODE == kX2) && k == 1) ? 0.f : sentinel_f32();
                    const float4 ab4 = make_float4(ab, ab, ab, ab);
                    float *hb = halo + (buf * NH + k) * L::kHalo;
                    if (hxm && ixm < 0) {
                        if (id.xm >= 0) {
                            cp_async4(hb + sxm, sk + id.xm * B3 + oxm);
                            cp_async4(hb + sxm + HB, sk + id.xm * B3 + oxm + ZB);
                        } else {
                            hb[sxm] = ab;
                            hb[sxm + HB] = ab;
                        }
                    }
                    if (hxp && ixp < 0) {
                        if (id.xp >= 0) {
                            cp_async4(hb + sxp, sk + id.xp * B3 + oxp);
                            cp_async4(hb + sxp + HB, sk + id.xp * B3 + oxp + ZB);
                        } else {
                            hb[sxp] = ab;
                            hb[sxp + HB] = ab;
                        }
                    }
                    if (hzm) {
                        if (id.zm >= 0) cp_async16(hb + szm, sk + id.zm * B3 + ozm);
                        else *reinterpret_cast<float4 *>(hb + szm) = ab4;
                    }
                    if (hzp) {
                        if (id.zp >= 0) cp_async16(hb + szp, sk + id.zp * B3 + ozp);
                        else *reinterpret_cast<float4 *>(hb + szp) = ab4;
                    }
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        if (hym) {
                            if (id.ym >= 0) cp_async16(hb + sym + q * HB, sk + id.ym * B3 + oym + q * ZB);
                            else *reinterpret_cast<float4 *>(hb + sym + q * HB) = ab4;
                        }
                        if (hyp) {
                            if (id.yp >= 0) cp_async16(hb + syp + q * HB, sk + id.yp * B3 + oyp + q * ZB);
                            else *reinterpret_cast<float4 *>(hb + syp + q * HB) = ab4;
                        }
                        if (WSM && k == 0) {
                            float *wb = wbuf + buf * kGroup2 + va + q * ZB;
                            if (id.ws >= 0) cp_async16(wb, a.w + id.ws * B3 + la + q * ZB);
                            else *reinterpret_cast<float4 *>(wb) = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    }
                }
            }
        }
        if (buf) {
            aixm1 = ixm;
            aixp1 = ixp;
            ahb1 = id.hb;
            aws1 = id.ws;
        } else {
            aixm0 = ixm;
            aixp0 = ixp;
            ahb0 = id.hb;
            aws0 = id.ws;
        }
        cp_async_commit();
    };

    // adjoint: this thread's sums of dL/dD and dL/dk, double-float (hi, lo)
    float gh[2] = {0.f, 0.f}, gl[2] = {0.f, 0.f};

    // AH: id1 holds the ids of group gi + 1 and id2 receives those of gi + 2;
    // otherwise id1 holds this group's ids and id2 receives the next group's.
    auto body = [&](int gi, int it, Halo &cur, const Ids &id1, Ids &id2) -> bool {
        const int s = it % S;
        const uint32_t par = (uint32_t)((it / S) & 1);
        int b0, nblk;
        span(gi, b0, nblk);
        const int b = b0 + j;
        const bool valid = j < nblk;
        // SBG_F32R: this row pair's source values (read now, used after the stage barrier)
        float4 ra = make_float4(0.f, 0.f, 0.f, 0.f), rb = ra;
        if (MODE == kSrc && valid) {
            ra = __ldg(reinterpret_cast<const float4 *>(io.src[1] + b * B3 + la));
            rb = __ldg(reinterpret_cast<const float4 *>(io.src[1] + b * B3 + la + ZB));
        }
        // two arrays, cp.async halos: this row pair's surface weights (read now, used after the barrier)
        float4 wga = make_float4(0.f, 0.f, 0.f, 0.f), wgb = wga;
        if (REACT && AH && !WSM && valid) {
            const int ws = (it & 1) ? aws1 : aws0;
            if (ws >= 0) {
                wga = __ldg(reinterpret_cast<const float4 *>(a.w + ws * B3 + la));
                wgb = __ldg(reinterpret_cast<const float4 *>(a.w + ws * B3 + la + ZB));
            }
        }
        if (AH) {
            issue_async(gi + 1, id1, (it + 1) & 1);
            id2 = load_ids(gi + 2);
            cp_async_wait_group<1>();  // this group's halo copies (issued a group ago) have landed
        } else {
            load_halo(gi, id1, cur);
            id2 = load_ids(gi + 1);
        }
        bool ok = true;
        if (tid == 0) ok = mbar_wait_bounded(&full[s], par, a.wait_cycles);
        if (__syncthreads_or(!ok)) {
            if (AH) cp_async_wait_all();
            if (tid == 0) {
                atomicExch(err, (int)SBG_ERR_TIMEOUT);
                for (int q = it; q < it + S && g0 + q < g1; ++q)
                    mbar_wait_bounded(&full[q % S], (uint32_t)((q / S) & 1), min(a.wait_cycles, 1ll << 28));
            }
            return false;
        }
        mbar_try_wait(&full[s], par);  // completed: gives this thread the acquire of the copied data
        if (tid == 0 && it >= 1 && gi - 1 + S < g1) issue(gi - 1 + S, (it - 1) % S);
        if (!valid) return true;
        if (!AH) park(cur);
        const int buf = AH ? (it & 1) : 0;
        const float *hbase = halo + buf * NH * L::kHalo;
        const int ixm = AH ? (buf ? aixm1 : aixm0) : cur.ixm;
        const int ixp = AH ? (buf ? aixp1 : aixp0) : cur.ixp;
        const uint32_t hbits = AH ? (buf ? ahb1 : ahb0) : cur.hb;
        float4 w0 = make_float4(0.f, 0.f, 0.f, 0.f), w1 = w0;
        if (REACT) {
            w0 = WSM ? *reinterpret_cast<const float4 *>(wbuf + buf * kGroup2 + va) : AH ? wga : cur.w[0];
            w1 = WSM ? *reinterpret_cast<const float4 *>(wbuf + buf * kGroup2 + va + ZB) : AH ? wgb : cur.w[1];
        }
        if constexpr (NH == 2) {
            // row q (a: 0, b: 1) of array k with its neighbours
            auto gather = [&](int k, int q) {
                const float *t = stages + ((size_t)s * NA + k) * kGroup2;
                const float *hk = hbase + k * L::kHalo;
                const int o = q * ZB, ho = q * HB;
                RowVals v;
                v.u = *reinterpret_cast<const float4 *>(t + va + o);
                v.xm = hxm ? (ixm >= 0 ? t[ixm + o] : hk[sxm + ho]) : t[va + o - 1];
                v.xp = hxp ? (ixp >= 0 ? t[ixp + o] : hk[sxp + ho]) : t[va + o + 4];
                v.ym = *reinterpret_cast<const float4 *>(hym ? hk + sym + ho : t + va + o - B);
                v.yp = *reinterpret_cast<const float4 *>(hyp ? hk + syp + ho : t + va + o + B);
                v.zm = *reinterpret_cast<const float4 *>((q == 0 && hzm) ? hk + szm : t + va + o - B * B);
                v.zp = *reinterpret_cast<const float4 *>((q == 1 && hzp) ? hk + szp : t + va + o + B * B);
                return v;
            };
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const RowVals v0 = gather(0, q), v1 = gather(1, q);
                const uint32_t hq = hbits >> (4 * q);
                float *d0 = io.dst[0] + b * B3 + la + q * ZB;
                if (MODE == kInh) {
                    *reinterpret_cast<float4 *>(d0) = row_update_inh(v0, v1, hq, a.cf);
                } else if (MODE == kAdj) {
                    float qd = 0.f, qk = 0.f;
                    *reinterpret_cast<float4 *>(d0) = row_adjoint1<REACT>(v0, v1, q ? w1 : w0, hq, a.cf, io.inv2[0],
                                                                          io.inv2[1], io.inv2[2], qd, qk);
                    df_add(gh[0], gl[0], qd, 0.f);
                    if (REACT) df_add(gh[1], gl[1], qk, 0.f);
                } else {
                    float4 o0, o1;
                    if (MODE == kX2) row_update_x2<REACT>(v0, v1, q ? w1 : w0, hq, a.cf, o0, o1);
                    else row_update_fwd2<REACT>(v0, v1, q ? w1 : w0, hq, a.cf, o0, o1);
                    *reinterpret_cast<float4 *>(d0) = o0;
                    *reinterpret_cast<float4 *>(io.dst[1] + b * B3 + la + q * ZB) = o1;
                }
            }
            return true;
        }

        const float *t = stages + (size_t)s * NA * kGroup2;
        const float4 ua = *reinterpret_cast<const float4 *>(t + va);
        const float4 ub = *reinterpret_cast<const float4 *>(t + va + ZB);
        const float xma = hxm ? (ixm >= 0 ? t[ixm] : hbase[sxm]) : t[va - 1];
        const float xmb = hxm ? (ixm >= 0 ? t[ixm + ZB] : hbase[sxm + HB]) : t[va + ZB - 1];
        const float xpa = hxp ? (ixp >= 0 ? t[ixp] : hbase[sxp]) : t[va + 4];
        const float xpb = hxp ? (ixp >= 0 ? t[ixp + ZB] : hbase[sxp + HB]) : t[va + ZB + 4];
        const float4 yma = *reinterpret_cast<const float4 *>(hym ? hbase + sym : t + va - B);
        const float4 ymb = *reinterpret_cast<const float4 *>(hym ? hbase + sym + HB : t + va + ZB - B);
        const float4 ypa = *reinterpret_cast<const float4 *>(hyp ? hbase + syp : t + va + B);
        const float4 ypb = *reinterpret_cast<const float4 *>(hyp ? hbase + syp + HB : t + va + ZB + B);
        const float4 zma = *reinterpret_cast<const float4 *>(hzm ? hbase + szm : t + va - B * B);
        const float4 zpa = *reinterpret_cast<const float4 *>(t + va + B * B);
        const float4 zmb = *reinterpret_cast<const float4 *>(t + va + ZB - B * B);
        const float4 zpb = *reinterpret_cast<const float4 *>(hzp ? hbase + szp : t + va + ZB + B * B);
        const float4 na = row_update<MODE, REACT>(ua, xma, xpa, yma, ypa, zma, zpa, ra, w0, hbits, a.cf);
        const float4 nbv = row_update<MODE, REACT>(ub, xmb, xpb, ymb, ypb, zmb, zpb, rb, w1, hbits >> 4, a.cf);
        *reinterpret_cast<float4 *>(io.dst[0] + b * B3 + la) = na;
        *reinterpret_cast<float4 *>(io.dst[0] + b * B3 + la + ZB) = nbv;
        return true;
    };

    Ids idA = load_ids(g0), idB;
    Halo hc;
    if (AH) {
        issue_async(g0, idA, 0);
        idA = load_ids(g0 + 1);
    }
    int it = 0;
    bool ok = true;
    for (int gi = g0; gi < g1; gi += 2, it += 2) {
        if (!body(gi, it, hc, idA, idB)) {
            ok = false;
            break;
        }
        if (gi + 1 >= g1) break;
        if (!body(gi + 1, it + 1, hc, idB, idA)) {
            ok = false;
            break;
        }
    }
    if (AH) cp_async_wait_all();  // no copy may land after the CTA's shared memory is gone
    if constexpr (MODE == kAdj) {
        if (!ok) return;  // uniform over the CTA (the time-out test is a CTA-wide vote)
        // CTA sums: double-float across the warp, FP64 across the warps, added to
        // the CTA's own slots (dL/dD_0 and dL/dk), so the order of additions is fixed
        __shared__ double red[kPipeThreads / 32][2];
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float h2 = __shfl_down_sync(0xffffffffu, gh[qq], o);
                const float l2 = __shfl_down_sync(0xffffffffu, gl[qq], o);
                df_add(gh[qq], gl[qq], h2, l2);
            }
            if ((tid & 31) == 0) red[tid >> 5][qq] = (double)gh[qq] + (double)gl[qq];
        }
        __syncthreads();
        if (tid < 2) {
            double v = 0.0;
            for (int w = 0; w < kPipeThreads / 32; ++w) v += red[w][tid];
            io.gsum[(int64_t)blockIdx.x * 3 + (tid == 0 ? 0 : 2)] += v;
        }
    }
}

template <int MODE, int NA>
struct PipeStages {
    static constexpr int S = NA == 1 ? 6 : NA == 2 ? (MODE == kAdj ? 3 : 4) : 3;  // adjoint: 3 leaves room for 6 CTAs
};

template <int MODE, int B, int NS, bool REACT, int HV>
static cudaError_t launch_pipe_hv(const StepArgs &a, const PipeIO &io, int ctas_per_sm, int max_ctas, int *err,
                                  cudaStream_t s, int *grid_out) {
    constexpr int NA = PipeShape<MODE, NS>::NA;
    constexpr int S = PipeStages<MODE, NA>::S;
    constexpr size_t smem = PipeSmem<MODE, B, NS, REACT, HV>::bytes(S);
    constexpr int G = kGroupVox / (B * B * B);
    // Without prefetch: 64 registers per thread (8 CTAs of 128 threads per SM)
    // with one array, 80 (6 CTAs) with two (the adjoint too, its gradient sums
    // included: 6 CTAs and 3 stages measured 2% faster than 5 and 4), 128
    // (4 CTAs) with four.  With register prefetch
    // (HV 1) the two register sets need up to 128 registers (4 CTAs per SM).
    // No more CTAs than fit in the SM's 228 KB of shared memory (1 KB of it
    // reserved per CTA) are asked for, so the registers go to those that fit.
    constexpr int kBase = HV == 1 ? 4 : (NA == 1 ? 8 : NA == 2 ? 6 : 4);
    constexpr int kFit = (int)((228 * 1024) / (smem + 1024));
    constexpr int MINB = kBase < kFit ? kBase : (kFit > 0 ? kFit : 1);
    auto kern = k_step_pipe<MODE, B, NS, REACT, S, MINB, HV>;
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
    const int64_t ngroups = a.items ? a.nitems : (a.nb + G - 1) / G;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > ngroups) grid = ngroups;
    if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
    if (grid_out) *grid_out = (int)(grid > 0 ? grid : 0);
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, kPipeThreads, smem, s>>>(a, io, err);
    return cudaGetLastError();
}

template <int MODE, int NH, int B, bool REACT, bool AH, bool WL>
static cudaError_t launch_rows2(const StepArgs &a, const PipeIO &io, int ctas_per_sm, int *err, cudaStream_t s,
                                int max_ctas = 0, int *grid_out = nullptr) {
    constexpr int NA = NH;
    constexpr bool WSM = AH && REACT && NH == 1;
    // Two ring stages (one group copied ahead while one computes) leave room for 9-10
    // CTAs per SM; the row loads are conflict-free, so resident warps are what hides the
    // latency: 9 CTAs (56 registers) for the SBG_F32R correction, 10 (51) for the rest,
    // fewer where the shared memory does not fit them (measured on grf256: 33.5 -> 28.4 us
    // and 29.6 -> 23.8 us against four stages and 5-6 CTAs).  Without cp.async halos the
    // halo values wait in registers across the group, so that variant keeps 7.  The
    // SBG_F32R work-list instance (batch solver) keeps 8, as 9 would spill.  Two arrays:
    // the shared memory holds 5 CTAs with 4^3 blocks (40 KB each), 7 with 8^3 blocks.
    constexpr int S = 2;
    constexpr size_t smem = ((size_t)S * NA * kGroup2 + (AH ? 2 : 1) * NH * Rows2Layout<B>::kHalo +
                             (WSM ? 2 * kGroup2 : 0)) * sizeof(float) + S * sizeof(uint64_t);
    constexpr int kFit = (int)((228 * 1024) / (smem + 1024));
    constexpr int kWant = NH == 2 ? 5 : !AH ? 7 : MODE == kSrc ? (WL ? 8 : 9) : 10;  // the work-list walk needs 4 more
    constexpr int MINB = kWant < kFit ? kWant : kFit;
    auto kern = k_step_rows2<MODE, NH, B, REACT, S, MINB, AH, WL>;
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
    constexpr int G = kGroup2 / (B * B * B);
    const int64_t ngroups = WL ? a.nitems : (a.nb + G - 1) / G;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > ngroups) grid = ngroups;
    if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
    if (grid_out) *grid_out = (int)(grid > 0 ? grid : 0);
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, kPipeThreads, smem, s>>>(a, io, err);
    return cudaGetLastError();
}

template <int MODE, bool AH>
static cudaError_t launch_rows2_a(const StepArgs &a, const PipeIO &io, int B, bool react, int ctas_per_sm, int *err,
                                  cudaStream_t s) {
    if (a.items) {
        if (B == 8)
            return react ? launch_rows2<MODE, 1, 8, true, AH, true>(a, io, ctas_per_sm, err, s)
                         : launch_rows2<MODE, 1, 8, false, AH, true>(a, io, ctas_per_sm, err, s);
        return react ? launch_rows2<MODE, 1, 4, true, AH, true>(a, io, ctas_per_sm, err, s)
                     : launch_rows2<MODE, 1, 4, false, AH, true>(a, io, ctas_per_sm, err, s);
    }
    if (B == 8)
        return react ? launch_rows2<MODE, 1, 8, true, AH, false>(a, io, ctas_per_sm, err, s)
                     : launch_rows2<MODE, 1, 8, false, AH, false>(a, io, ctas_per_sm, err, s);
    return react ? launch_rows2<MODE, 1, 4, true, AH, false>(a, io, ctas_per_sm, err, s)
                 : launch_rows2<MODE, 1, 4, false, AH, false>(a, io, ctas_per_sm, err, s);
}
// two arrays (species A and B, or u and the diffusivity factor): cp.async
// halos and the walk over the block list only
template <int MODE>
static cudaError_t launch_rows2_two(const StepArgs &a, const PipeIO &io, int B, bool react, int ctas_per_sm,
                                    int *err, cudaStream_t s) {
    if constexpr (MODE == kInh) {
        return B == 8 ? launch_rows2<kInh, 2, 8, false, true, false>(a, io, ctas_per_sm, err, s)
                      : launch_rows2<kInh, 2, 4, false, true, false>(a, io, ctas_per_sm, err, s);
    } else {
        if (B == 8)
            return react ? launch_rows2<MODE, 2, 8, true, true, false>(a, io, ctas_per_sm, err, s)
                         : launch_rows2<MODE, 2, 8, false, true, false>(a, io, ctas_per_sm, err, s);
        return react ? launch_rows2<MODE, 2, 4, true, true, false>(a, io, ctas_per_sm, err, s)
                     : launch_rows2<MODE, 2, 4, false, true, false>(a, io, ctas_per_sm, err, s);
    }
}
// halo variant 0: loads when the group comes up; 2: cp.async one group ahead
template <int MODE>
static cudaError_t launch_rows2_b(const StepArgs &a, const PipeIO &io, int B, bool react, int hv, int ctas_per_sm,
                                  int *err, cudaStream_t s) {
    return hv == 2 ? launch_rows2_a<MODE, true>(a, io, B, react, ctas_per_sm, err, s)
                   : launch_rows2_a<MODE, false>(a, io, B, react, ctas_per_sm, err, s);
}

template <int MODE, int B, int NS, bool REACT>
static cudaError_t launch_pipe_t(const StepArgs &a, const PipeIO &io, int hv, int ctas_per_sm, int *err,
                                 cudaStream_t s) {
    if (hv == 1) return launch_pipe_hv<MODE, B, NS, REACT, 1>(a, io, ctas_per_sm, 0, err, s, nullptr);
    if (hv == 2) return launch_pipe_hv<MODE, B, NS, REACT, 2>(a, io, ctas_per_sm, 0, err, s, nullptr);
    return launch_pipe_hv<MODE, B, NS, REACT, 0>(a, io, ctas_per_sm, 0, err, s, nullptr);
}

template <int MODE, int NS>
static cudaError_t launch_pipe_b(const StepArgs &a, const PipeIO &io, int B, bool react, int hv,
                                 int ctas_per_sm, int *err, cudaStream_t s) {
    if (B == 8)
        return react ? launch_pipe_t<MODE, 8, NS, true>(a, io, hv, ctas_per_sm, err, s)
                     : launch_pipe_t<MODE, 8, NS, false>(a, io, hv, ctas_per_sm, err, s);
    return react ? launch_pipe_t<MODE, 4, NS, true>(a, io, hv, ctas_per_sm, err, s)
                 : launch_pipe_t<MODE, 4, NS, false>(a, io, hv, ctas_per_sm, err, s);
}

// The single-array modes (FP32 one species, SBG_F32R) run the two-row kernel
// unless register-prefetched halos are asked for; its groups (and work-list
// spans) hold up to 1024 voxels, the one-row kernel's 512.  The two-array
// modes (two FP32 species; one species with a diffusivity factor; SBG_F32X2)
// run it with cp.async halos when they walk the block list; work lists and
// the other halo variants keep the one-row kernel.
static bool rows2_path(sbg_dtype dtype, int ns, bool eps, int hv, bool worklist) {
    if (hv != 1 && ns == 1 && !eps && (dtype == SBG_F32 || dtype == SBG_F32R)) return true;
    if (hv != 2 || worklist) return false;
    return (dtype == SBG_F32 && ((ns == 2 && !eps) || (ns == 1 && eps))) || (dtype == SBG_F32X2 && ns == 1 && !eps);
}
int step_work_group_voxels(sbg_dtype dtype, int ns, bool eps, int halo_variant) {
    return rows2_path(dtype, ns, eps, halo_variant, true) ? kGroup2 : kGroupVox;
}

bool launch_step_pipe(const StepArgs &a, sbg_dtype dtype, int ns, int B, bool react, int halo_variant,
                      int ctas_per_sm, int *err_flag, cudaStream_t s, cudaError_t *launch_err) {
    const int hv = halo_variant;
    if (a.nb * (int64_t)(B * B * B) >= (int64_t(1) << 31)) return false;  // 32-bit slot indices in the kernel
    PipeIO io;
    std::memset(&io, 0, sizeof(io));
    cudaError_t e = cudaSuccess;
    if (dtype == SBG_F32X2 && ns == 1) {
        io.src[0] = (const float *)a.in[0];
        io.src[1] = a.in_lo[0];
        io.dst[0] = (float *)a.out[0];
        io.dst[1] = a.out_lo[0];
        e = rows2_path(dtype, ns, a.eps != nullptr, hv, a.items != nullptr)
                ? launch_rows2_two<kX2>(a, io, B, react, ctas_per_sm, err_flag, s)
                : launch_pipe_b<kX2, 1>(a, io, B, react, hv, ctas_per_sm, err_flag, s);
    } else if (dtype == SBG_F32R && ns == 1) {
        io.src[0] = (const float *)a.in[0];
        io.src[1] = a.src_term;
        io.dst[0] = (float *)a.out[0];
        e = rows2_path(dtype, ns, a.eps != nullptr, hv, a.items != nullptr)
                ? launch_rows2_b<kSrc>(a, io, B, react, hv, ctas_per_sm, err_flag, s)
                : launch_pipe_b<kSrc, 1>(a, io, B, react, hv, ctas_per_sm, err_flag, s);
    } else if (dtype == SBG_F32 && ns == 1 && a.eps) {
        io.src[0] = (const float *)a.in[0];
        io.src[1] = a.eps;
        io.dst[0] = (float *)a.out[0];
        e = rows2_path(dtype, ns, true, hv, a.items != nullptr)
                ? launch_rows2_two<kInh>(a, io, B, false, ctas_per_sm, err_flag, s)
                : launch_pipe_b<kInh, 1>(a, io, B, false, hv, ctas_per_sm, err_flag, s);
    } else if (dtype == SBG_F32 && (ns == 1 || ns == 2)) {
        for (int k = 0; k < ns; ++k) {
            io.src[k] = (const float *)a.in[k];
            io.dst[k] = (float *)a.out[k];
        }
        if (ns == 1)
            e = rows2_path(dtype, ns, false, hv, a.items != nullptr)
                    ? launch_rows2_b<kFwd>(a, io, B, react, hv, ctas_per_sm, err_flag, s)
                    : launch_pipe_b<kFwd, 1>(a, io, B, react, hv, ctas_per_sm, err_flag, s);
        else
            e = rows2_path(dtype, ns, false, hv, a.items != nullptr)
                    ? launch_rows2_two<kFwd>(a, io, B, react, ctas_per_sm, err_flag, s)
                    : launch_pipe_b<kFwd, 2>(a, io, B, react, hv, ctas_per_sm, err_flag, s);
    } else {
        return false;
    }
    *launch_err = e;
    return true;
}

cudaError_t launch_adjoint_pipe(const StepArgs &a, const PipeIO &io, int ns, int B, bool react, int max_ctas,
                                int *err_flag, cudaStream_t s, int *grid_out) {
    if (a.nb * (int64_t)(B * B * B) >= (int64_t(1) << 31)) return cudaErrorInvalidValue;  // 32-bit slot indices
    // halo values copied one group ahead with cp.async (2% faster than loading them when the
    // group comes up, gradients bitwise the same); one species (lambda and u^n) on the
    // two-row kernel
    if (ns == 1 && !a.items) {
        if (B == 8)
            return react ? launch_rows2<kAdj, 2, 8, true, true, false>(a, io, 0, err_flag, s, max_ctas, grid_out)
                         : launch_rows2<kAdj, 2, 8, false, true, false>(a, io, 0, err_flag, s, max_ctas, grid_out);
        return react ? launch_rows2<kAdj, 2, 4, true, true, false>(a, io, 0, err_flag, s, max_ctas, grid_out)
                     : launch_rows2<kAdj, 2, 4, false, true, false>(a, io, 0, err_flag, s, max_ctas, grid_out);
    }
    if (ns == 1) {
        if (B == 8)
            return react ? launch_pipe_hv<kAdj, 8, 1, true, 2>(a, io, 0, max_ctas, err_flag, s, grid_out)
                         : launch_pipe_hv<kAdj, 8, 1, false, 2>(a, io, 0, max_ctas, err_flag, s, grid_out);
        return react ? launch_pipe_hv<kAdj, 4, 1, true, 2>(a, io, 0, max_ctas, err_flag, s, grid_out)
                     : launch_pipe_hv<kAdj, 4, 1, false, 2>(a, io, 0, max_ctas, err_flag, s, grid_out);
    }
    if (B == 8)
        return react ? launch_pipe_hv<kAdj, 8, 2, true, 2>(a, io, 0, max_ctas, err_flag, s, grid_out)
                     : launch_pipe_hv<kAdj, 8, 2, false, 2>(a, io, 0, max_ctas, err_flag, s, grid_out);
    return react ? launch_pipe_hv<kAdj, 4, 2, true, 2>(a, io, 0, max_ctas, err_flag, s, grid_out)
                 : launch_pipe_hv<kAdj, 4, 2, false, 2>(a, io, 0, max_ctas, err_flag, s, grid_out);
}

}  // namespace sbg
