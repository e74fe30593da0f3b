// The time step: forward-Euler FTCS of Eq. 1 on the sparse block grid
// (Sec. 2.3), with the no-flux rule applied inside the stencil (a neighbour
// outside Omega takes the centre value; Appendix B Listing 6), active voxels
// of Dirichlet faces held, and the linear bulk/surface reactions of Sec. 3.5.
//
// Kernel design (one CTA updates BPC blocks, one thread per voxel):
//  - each thread loads its own voxel (coalesced: a warp reads 128 contiguous
//    bytes of one block) and stores it in a shared-memory tile;
//  - threads on a block face load the one-voxel halo from the face
//    neighbour (id from the precomputed face table; -1 or an inactive voxel
//    reads as the sentinel, which the mirror rule replaces by the centre);
//  - after one barrier every interior neighbour comes from shared memory.
// The update is one expression per voxel, identical for B = 4 and B = 8, so
// results do not depend on the block size.
#include <math.h>

#include <algorithm>
#include <cstring>

#include "sbg_internal.cuh"
#include "sbg_step.cuh"
#include "sbg_trace.cuh"

#ifndef SBG_DEBUG
#define SBG_DEBUG 0
#endif

namespace sbg {

// Plain FP32 / FP64 state, NS species, optional reaction (REACT: k_surf != 0).
// SRC: the correction d of an SBG_F32R state (one FP32 species), whose update
// takes the stored source r = L_h b in place of the transfer term and the
// surface loss k w in its rate.
// EXT: an external space-time source a_n S_s(x) joins the transfer term
// (rounded as fma(a_n, S_s, t)).
template <typename T, int B, int BPC, int NS, bool REACT, bool SRC = false, bool EXT = false>
__global__ void __launch_bounds__(BPC * B * B * B, (sizeof(T) == 8 ? 1024 : 2048) / (BPC * B * B * B))
k_step(const StepArgs a) {
    constexpr int B3 = B * B * B;
    __shared__ T tile[NS][BPC * B3];
    const int tid = threadIdx.x;
    const int j = tid / B3;
    const int l = tid - j * B3;
    const int64_t b = (int64_t)blockIdx.x * BPC + j;
    const bool valid = b < a.nb;
    const int x = l % B, y = (l / B) % B, z = l / (B * B);

    T uc[NS], hxm[NS], hxp[NS], hym[NS], hyp[NS], hzm[NS], hzp[NS];
    int4 bc = make_int4(0, 0, 0, 0);
    if (valid) {
        bc = a.blocks[b];
        const int32_t *fn = a.face + b * 6;
        int nxm = (x == 0) ? fn[0] : -1, nxp = (x == B - 1) ? fn[1] : -1;
        int nym = (y == 0) ? fn[2] : -1, nyp = (y == B - 1) ? fn[3] : -1;
        int nzm = (z == 0) ? fn[4] : -1, nzp = (z == B - 1) ? fn[5] : -1;
#if SBG_DEBUG
        // the debug build checks every face id against the block list before using it
        int *ids[6] = {&nxm, &nxp, &nym, &nyp, &nzm, &nzp};
#pragma unroll
        for (int f = 0; f < 6; ++f)
            if (*ids[f] < -1 || *ids[f] >= a.nb) {
                atomicExch(a.err, (int)SBG_ERR_BOUNDS);
                *ids[f] = -1;
            }
#endif
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const T *in = (const T *)a.in[s];
            uc[s] = in[b * B3 + l];
            tile[s][tid] = uc[s];
            const T sent = sentinel<T>();
            hxm[s] = (nxm >= 0) ? in[(int64_t)nxm * B3 + l + (B - 1)] : sent;
            hxp[s] = (nxp >= 0) ? in[(int64_t)nxp * B3 + l - (B - 1)] : sent;
            hym[s] = (nym >= 0) ? in[(int64_t)nym * B3 + l + (B - 1) * B] : sent;
            hyp[s] = (nyp >= 0) ? in[(int64_t)nyp * B3 + l - (B - 1) * B] : sent;
            hzm[s] = (nzm >= 0) ? in[(int64_t)nzm * B3 + l + (B - 1) * B * B] : sent;
            hzp[s] = (nzp >= 0) ? in[(int64_t)nzp * B3 + l - (B - 1) * B * B] : sent;
        }
    }
    __syncthreads();
    if (!valid) return;

    const int nx = a.gdims[bc.w * 4 + 0], ny = a.gdims[bc.w * 4 + 1], nz = a.gdims[bc.w * 4 + 2];
    const bool held = is_held(a.held_mask, bc.x * B + x, bc.y * B + y, bc.z * B + z, nx, ny, nz);
    const StepCoef<T> &k = coef<T>(a);
    T w = T(0);
    if (REACT) {
        const int ws = a.wslab[b];
        if (ws >= 0) w = sizeof(T) == 8 ? (T)a.w64[(int64_t)ws * B3 + l] : (T)a.w[(int64_t)ws * B3 + l];
    }
    const T transfer = (REACT && !SRC) ? k.k * w * uc[0] : T(0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const T u = uc[s];
        T res = u;
        if (SRC && !is_sent(u) && !held) {
            const T *t = tile[s] + j * B3;
            const T xm = mirror(x > 0 ? t[l - 1] : hxm[s], u);
            const T xp = mirror(x < B - 1 ? t[l + 1] : hxp[s], u);
            const T ym = mirror(y > 0 ? t[l - B] : hym[s], u);
            const T yp = mirror(y < B - 1 ? t[l + B] : hyp[s], u);
            const T zm = mirror(z > 0 ? t[l - B * B] : hzm[s], u);
            const T zp = mirror(z < B - 1 ? t[l + B * B] : hzp[s], u);
            const float rate = REACT ? __fmaf_rn(a.cf.k, (float)w, a.cf.decay[0]) : a.cf.decay[0];
            res = (T)fused_update((float)u, (float)xm, (float)xp, (float)ym, (float)yp, (float)zm, (float)zp,
                                  a.cf.c[0], a.cf.dt, rate, a.src_term[b * B3 + l]);
        } else if (!is_sent(u) && !held) {
            const T *t = tile[s] + j * B3;
            const T xm = mirror(x > 0 ? t[l - 1] : hxm[s], u);
            const T xp = mirror(x < B - 1 ? t[l + 1] : hxp[s], u);
            const T ym = mirror(y > 0 ? t[l - B] : hym[s], u);
            const T yp = mirror(y < B - 1 ? t[l + B] : hyp[s], u);
            const T zm = mirror(z > 0 ? t[l - B * B] : hzm[s], u);
            const T zp = mirror(z < B - 1 ? t[l + B * B] : hzp[s], u);
            T tt = s == 0 ? -transfer : transfer;
            if (EXT && a.ext[s]) tt = fma_pinned((T)a.ext_scale, ((const T *)a.ext[s])[b * B3 + l], tt);
            res = fused_update(u, xm, xp, ym, yp, zm, zp, k.c[s], k.dt, k.decay[s], tt);
        }
        ((T *)a.out[s])[b * B3 + l] = res;
    }
}

// Compensated FP32 (value = hi + lo), one species.  The Laplacian is
// evaluated as (differences of hi) + (differences of lo); the increment is
// added with an error-free two-sum and renormalised, so increments far below
// one FP32 ulp of the state accumulate in lo instead of being rounded away.
template <int B, int BPC, bool REACT>
__global__ void __launch_bounds__(BPC * B * B * B, 2048 / (BPC * B * B * B))
k_step_x2(const StepArgs a) {
    constexpr int B3 = B * B * B;
    __shared__ float th[BPC * B3];
    __shared__ float tl[BPC * B3];
    const int tid = threadIdx.x;
    const int j = tid / B3;
    const int l = tid - j * B3;
    const int64_t b = (int64_t)blockIdx.x * BPC + j;
    const bool valid = b < a.nb;
    const int x = l % B, y = (l / B) % B, z = l / (B * B);
    const float *ih = (const float *)a.in[0];
    const float *il = a.in_lo[0];
    float hc = 0.f, lc = 0.f;
    float h[6], lo6[6];
    int4 bc = make_int4(0, 0, 0, 0);
    if (valid) {
        bc = a.blocks[b];
        const int32_t *fn = a.face + b * 6;
        hc = ih[b * B3 + l];
        lc = il[b * B3 + l];
        th[tid] = hc;
        tl[tid] = lc;
        const int nid[6] = {(x == 0) ? fn[0] : -1,     (x == B - 1) ? fn[1] : -1,
                            (y == 0) ? fn[2] : -1,     (y == B - 1) ? fn[3] : -1,
                            (z == 0) ? fn[4] : -1,     (z == B - 1) ? fn[5] : -1};
        const int off[6] = {B - 1, -(B - 1), (B - 1) * B, -(B - 1) * B, (B - 1) * B * B, -(B - 1) * B * B};
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            if (nid[f] >= 0) {
                h[f] = ih[(int64_t)nid[f] * B3 + l + off[f]];
                lo6[f] = il[(int64_t)nid[f] * B3 + l + off[f]];
            } else {
                h[f] = sentinel_f32();
                lo6[f] = 0.f;
            }
        }
    }
    __syncthreads();
    if (!valid) return;
    const int nx = a.gdims[bc.w * 4 + 0], ny = a.gdims[bc.w * 4 + 1], nz = a.gdims[bc.w * 4 + 2];
    const bool held = is_held(a.held_mask, bc.x * B + x, bc.y * B + y, bc.z * B + z, nx, ny, nz);
    float rh = hc, rl = lc;
    if (!is_sent(hc) && !held) {
        const float *t = th + j * B3;
        const float *u = tl + j * B3;
        // neighbour (hi, lo) per direction: -x, +x, -y, +y, -z, +z
        float nh[6], nl[6];
        nh[0] = x > 0 ? t[l - 1] : h[0];             nl[0] = x > 0 ? u[l - 1] : lo6[0];
        nh[1] = x < B - 1 ? t[l + 1] : h[1];         nl[1] = x < B - 1 ? u[l + 1] : lo6[1];
        nh[2] = y > 0 ? t[l - B] : h[2];             nl[2] = y > 0 ? u[l - B] : lo6[2];
        nh[3] = y < B - 1 ? t[l + B] : h[3];         nl[3] = y < B - 1 ? u[l + B] : lo6[3];
        nh[4] = z > 0 ? t[l - B * B] : h[4];         nl[4] = z > 0 ? u[l - B * B] : lo6[4];
        nh[5] = z < B - 1 ? t[l + B * B] : h[5];     nl[5] = z < B - 1 ? u[l + B * B] : lo6[5];
#pragma unroll
        for (int f = 0; f < 6; ++f)
            if (is_sent(nh[f])) {
                nh[f] = hc;
                nl[f] = lc;
            }
        const StepCoef<float> &k = a.cf;
        float rate = k.decay[0];
        if (REACT) {
            const int ws = a.wslab[b];
            rate = __fmaf_rn(k.k, ws >= 0 ? a.w[(int64_t)ws * B3 + l] : 0.f, rate);
        }
        fused_update_x2(hc, lc, nh, nl, k.c[0], k.dt, rate, rh, rl);
    }
    ((float *)a.out[0])[b * B3 + l] = rh;
    a.out_lo[0][b * B3 + l] = rl;
}

// ---------------------------------------------------------------------------
// held-voxel bits of each block for the Dirichlet face set `mask`: one
// thread per 64-voxel word
template <int B>
__global__ void k_held_bits(const int4 *blocks, const int32_t *gdims, int mask, int64_t nb, uint64_t *out) {
    constexpr int B3 = B * B * B;
    constexpr int W = (B3 + 63) / 64;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * W) return;
    const int64_t b = i / W;
    const int w = (int)(i - b * W);
    const int4 bc = blocks[b];
    const int nx = gdims[bc.w * 4], ny = gdims[bc.w * 4 + 1], nz = gdims[bc.w * 4 + 2];
    uint64_t bits = 0;
    for (int q = 0; q < 64 && w * 64 + q < B3; ++q) {
        const int l = w * 64 + q;
        if (is_held(mask, bc.x * B + l % B, bc.y * B + (l / B) % B, bc.z * B + l / (B * B), nx, ny, nz))
            bits |= 1ull << q;
    }
    out[i] = bits;
}

static int held_mask_of(const sbg_params *p) {
    int m = 0;
    for (int f = 0; f < 6; ++f)
        if (p->face_type[f] == SBG_FACE_DIRICHLET) m |= 1 << f;
    return m;
}

sbg_status prepare_held_bits(sbg_grid g, const sbg_params *p, cudaStream_t s) {
    const int mask = held_mask_of(p);
    if (mask == 0 || g->nb == 0 || g->heldbits_mask == mask) return SBG_OK;
    const int64_t n = g->nb * g->words();
    if (!g->heldbits) {
        cudaError_t e = dmalloc((void **)&g->heldbits, sizeof(uint64_t) * n);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (held bits)");
        g->bytes += (int64_t)(sizeof(uint64_t) * n);
    }
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (g->B == 8) k_held_bits<8><<<grid, 256, 0, s>>>(g->blocks, g->gdims, mask, g->nb, g->heldbits);
    else k_held_bits<4><<<grid, 256, 0, s>>>(g->blocks, g->gdims, mask, g->nb, g->heldbits);
    SBG_LAUNCH_CHECK("held-bits kernel launch");
    g->heldbits_mask = mask;
    return SBG_OK;
}

// Grid tables and coefficients of a step (no state arrays).
void fill_step_args(sbg_grid g, const sbg_params *p, StepArgs &a) {
    std::memset(&a, 0, sizeof(a));
    a.blocks = g->blocks;
    a.face = g->face_nbr;
    a.wslab = g->wslab;
    a.w = g->w;
    a.w64 = g->w64;
    a.pad = g->pad;
    a.gdims = g->gdims;
    a.nb = g->nb;
    a.held_mask = held_mask_of(p);
    a.eps = g->has_eps ? g->eps : nullptr;
    a.eps64 = g->has_eps ? g->eps64 : nullptr;
    a.heldbits = (a.held_mask && g->heldbits_mask == a.held_mask) ? g->heldbits : nullptr;
    a.err = g->err;
    a.stall_group = g->inject_stall_group;
    a.wait_cycles = g->inject_stall_group >= 0 ? g->inject_wait_cycles : (1ll << 31);
    for (int s = 0; s < 2; ++s) {
        for (int ax = 0; ax < 3; ++ax) {
            double c = p->D[s] / (p->dx[ax] * p->dx[ax]);
            a.cd.c[s][ax] = c;
            a.cf.c[s][ax] = (float)c;
        }
        a.cd.decay[s] = p->decay[s];
        a.cf.decay[s] = (float)p->decay[s];
    }
    a.cd.dt = p->dt;
    a.cf.dt = (float)p->dt;
    a.cd.k = p->k_surf;
    a.cf.k = (float)p->k_surf;
}

static void fill_args(sbg_grid g, sbg_state st, const sbg_params *p, int src, StepArgs &a) {
    fill_step_args(g, p, a);
    for (int s = 0; s < st->ns; ++s) {
        a.in[s] = st->val[src][s];
        a.out[s] = st->val[1 - src][s];
        a.in_lo[s] = st->lo[src][s];
        a.out_lo[s] = st->lo[1 - src][s];
    }
    a.src_term = st->rsrc;
}

template <typename T, int B, int NS, bool SRC = false, bool EXT = false>
static void launch_plain(const StepArgs &a, bool react, cudaStream_t s) {
    constexpr int BPC = (B == 8) ? 1 : 8;
    const unsigned grid = (unsigned)((a.nb + BPC - 1) / BPC);
    if (react) k_step<T, B, BPC, NS, true, SRC, EXT><<<grid, BPC * B * B * B, 0, s>>>(a);
    else k_step<T, B, BPC, NS, false, SRC, EXT><<<grid, BPC * B * B * B, 0, s>>>(a);
}

// Plain kernel for inhomogeneous diffusion (one species, FP32 or FP64): the
// state and the diffusivity factor are staged as block tiles; a halo factor
// of an absent neighbour block reads 0 (its face carries no flux anyway).
template <typename T, int B, int BPC>
__global__ void __launch_bounds__(BPC * B * B * B, (sizeof(T) == 8 ? 1024 : 2048) / (BPC * B * B * B))
k_step_inh(const StepArgs a) {
    constexpr int B3 = B * B * B;
    __shared__ T tile[BPC * B3];
    __shared__ T etile[BPC * B3];
    const int tid = threadIdx.x;
    const int j = tid / B3;
    const int l = tid - j * B3;
    const int64_t b = (int64_t)blockIdx.x * BPC + j;
    const bool valid = b < a.nb;
    const int x = l % B, y = (l / B) % B, z = l / (B * B);
    const T *in = (const T *)a.in[0];
    const T *ep = sizeof(T) == 8 ? (const T *)a.eps64 : (const T *)a.eps;
    T uc = T(0), ec = T(0), hu[6], he[6];
    int4 bc = make_int4(0, 0, 0, 0);
    const int off[6] = {B - 1, -(B - 1), (B - 1) * B, -(B - 1) * B, (B - 1) * B * B, -(B - 1) * B * B};
    const bool edge[6] = {x == 0, x == B - 1, y == 0, y == B - 1, z == 0, z == B - 1};
    if (valid) {
        bc = a.blocks[b];
        uc = in[b * B3 + l];
        ec = ep[b * B3 + l];
        tile[tid] = uc;
        etile[tid] = ec;
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const int nid = edge[f] ? a.face[b * 6 + f] : -1;
            hu[f] = nid >= 0 ? in[(int64_t)nid * B3 + l + off[f]] : sentinel<T>();
            he[f] = nid >= 0 ? ep[(int64_t)nid * B3 + l + off[f]] : T(0);
        }
    }
    __syncthreads();
    if (!valid) return;
    const int nx = a.gdims[bc.w * 4 + 0], ny = a.gdims[bc.w * 4 + 1], nz = a.gdims[bc.w * 4 + 2];
    const bool held = is_held(a.held_mask, bc.x * B + x, bc.y * B + y, bc.z * B + z, nx, ny, nz);
    T res = uc;
    if (!is_sent(uc) && !held) {
        const T *t = tile + j * B3;
        const T *e = etile + j * B3;
        const int step[6] = {-1, 1, -B, B, -B * B, B * B};
        T nv[6], en[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            nv[f] = mirror(edge[f] ? hu[f] : t[l + step[f]], uc);
            en[f] = edge[f] ? he[f] : e[l + step[f]];
        }
        T dp[3], dm[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            dp[ax] = nv[2 * ax + 1] - uc;
            dm[ax] = uc - nv[2 * ax];
        }
        const StepCoef<T> &k = coef<T>(a);
        res = inh_update(uc, dp, dm, ec, en, k.c[0], k.dt, k.decay[0]);
    }
    ((T *)a.out[0])[b * B3 + l] = res;
}

template <typename T, int B>
static void launch_inh(const StepArgs &a, cudaStream_t s) {
    constexpr int BPC = (B == 8) ? 1 : 8;
    const unsigned grid = (unsigned)((a.nb + BPC - 1) / BPC);
    k_step_inh<T, B, BPC><<<grid, BPC * B * B * B, 0, s>>>(a);
}

template <int B>
static void launch_x2(const StepArgs &a, bool react, cudaStream_t s) {
    constexpr int BPC = (B == 8) ? 1 : 8;
    const unsigned grid = (unsigned)((a.nb + BPC - 1) / BPC);
    if (react) k_step_x2<B, BPC, true><<<grid, BPC * B * B * B, 0, s>>>(a);
    else k_step_x2<B, BPC, false><<<grid, BPC * B * B * B, 0, s>>>(a);
}

// One step from buffer `src` into 1 - src (no state bookkeeping).
sbg_status launch_step(sbg_grid g, sbg_state st, const sbg_params *p, int src, cudaStream_t s) {
    if (g->nb == 0) return SBG_OK;
    StepArgs a;
    fill_args(g, st, p, src, a);
    const bool react = p->k_surf != 0.0;
    if (a.held_mask && !a.heldbits) return fail(SBG_ERR_INVALID_ARG, "internal: held bits not prepared");
    const bool inh = a.eps != nullptr;
    if (inh && ((st->dtype != SBG_F32 && st->dtype != SBG_F64) || st->ns != 1))
        return fail(SBG_ERR_INVALID_ARG, "a diffusivity factor is set: SBG_F32 or SBG_F64 states of one species only");
    // a diffusivity factor: the streaming form where it applies (asked for or automatic; 231.7 us
    // against 368.7 us for the two-row ring kernel per 512^3 step)
    if (inh && (st->variant == SBG_KERNEL_STREAM || st->variant == SBG_KERNEL_AUTO) && stream_inh_applies(g, st)) {
        cudaError_t e = launch_step_stream_inh(a, g, st->ctas_per_sm, s);
        if (e != cudaSuccess) return cuda_fail(e, "streaming step kernel launch (diffusivity factor)");
        return SBG_OK;
    }
    // compensated states: the streaming form where it applies (asked for or automatic; 41.6 us against
    // 55.3 us for the two-row ring kernel per grf256 step)
    if (st->dtype == SBG_F32X2 && (st->variant == SBG_KERNEL_STREAM || st->variant == SBG_KERNEL_AUTO) &&
        stream_x2_applies(g, st)) {
        cudaError_t e = launch_step_stream_x2(a, g, react, st->ctas_per_sm, s);
        if (e != cudaSuccess) return cuda_fail(e, "streaming step kernel launch (compensated state)");
        return SBG_OK;
    }
    // the streaming kernel: asked for, or the automatic choice wherever it applies (measured per
    // step against the two-row ring kernel: 259 us against 390 us for the 512^3 two-species run,
    // 19.0 against 23.8 us for one FP32 species and 26.4 against 27.4 us for SBG_F32R on grf256)
    const bool stream = st->variant == SBG_KERNEL_STREAM || st->variant == SBG_KERNEL_WAVE ||
                        st->variant == SBG_KERNEL_WAVE4 || st->variant == SBG_KERNEL_AUTO;
    if (stream && stream_kernel_applies(g, st) && !(st->dtype == SBG_F32R && react)) {
        cudaError_t e = launch_step_stream(a, g, st->ns, react, st->ctas_per_sm, s);
        if (e != cudaSuccess) return cuda_fail(e, "streaming step kernel launch");
        return SBG_OK;
    }
    if (st->variant != SBG_KERNEL_PLAIN) {
        cudaError_t e = cudaSuccess;
        if (launch_step_pipe(a, st->dtype, st->ns, g->B, react, halo_variant_of(st->variant),
                             st->ctas_per_sm, g->err, s, &e)) {
            if (e != cudaSuccess) return cuda_fail(e, "pipelined step kernel launch");
            return SBG_OK;
        }
        if (st->variant >= SBG_KERNEL_PIPELINED && st->variant < SBG_KERNEL_STREAM)
            return fail(SBG_ERR_INVALID_ARG,
                        st->dtype == SBG_F64 ? "the pipelined kernel handles FP32-based states only"
                                             : "the pipelined kernel needs fewer than 2^31 voxel slots (blocks x B^3)");
    }
    if (st->dtype == SBG_F32X2) {
        if (g->B == 8) launch_x2<8>(a, react, s);
        else launch_x2<4>(a, react, s);
    } else if (st->dtype == SBG_F32R) {
        if (g->B == 8) launch_plain<float, 8, 1, true>(a, react, s);
        else launch_plain<float, 4, 1, true>(a, react, s);
    } else if (inh) {
        if (st->dtype == SBG_F32) {
            if (g->B == 8) launch_inh<float, 8>(a, s);
            else launch_inh<float, 4>(a, s);
        } else {
            if (g->B == 8) launch_inh<double, 8>(a, s);
            else launch_inh<double, 4>(a, s);
        }
    } else if (st->dtype == SBG_F32) {
        if (g->B == 8) {
            if (st->ns == 1) launch_plain<float, 8, 1>(a, react, s);
            else launch_plain<float, 8, 2>(a, react, s);
        } else {
            if (st->ns == 1) launch_plain<float, 4, 1>(a, react, s);
            else launch_plain<float, 4, 2>(a, react, s);
        }
    } else {
        if (g->B == 8) {
            if (st->ns == 1) launch_plain<double, 8, 1>(a, react, s);
            else launch_plain<double, 8, 2>(a, react, s);
        } else {
            if (st->ns == 1) launch_plain<double, 4, 1>(a, react, s);
            else launch_plain<double, 4, 2>(a, react, s);
        }
    }
    SBG_LAUNCH_CHECK("step kernel launch");
    return SBG_OK;
}

// One step with the external source of the state scaled by `scale` (plain
// kernel, SBG_F32 / SBG_F64 states, constant D).
sbg_status launch_step_ext(sbg_grid g, sbg_state st, const sbg_params *p, int src, double scale, cudaStream_t s) {
    if (g->nb == 0) return SBG_OK;
    StepArgs a;
    fill_args(g, st, p, src, a);
    if (a.held_mask && !a.heldbits) return fail(SBG_ERR_INVALID_ARG, "internal: held bits not prepared");
    if (a.eps) return fail(SBG_ERR_INVALID_ARG, "an external source with a diffusivity factor is not supported");
    a.ext[0] = st->ext[0];
    a.ext[1] = st->ext[1];
    a.ext_scale = scale;
    const bool react = p->k_surf != 0.0;
    if (st->dtype == SBG_F32) {
        if (g->B == 8) {
            if (st->ns == 1) launch_plain<float, 8, 1, false, true>(a, react, s);
            else launch_plain<float, 8, 2, false, true>(a, react, s);
        } else {
            if (st->ns == 1) launch_plain<float, 4, 1, false, true>(a, react, s);
            else launch_plain<float, 4, 2, false, true>(a, react, s);
        }
    } else if (st->dtype == SBG_F64) {
        if (g->B == 8) {
            if (st->ns == 1) launch_plain<double, 8, 1, false, true>(a, react, s);
            else launch_plain<double, 8, 2, false, true>(a, react, s);
        } else {
            if (st->ns == 1) launch_plain<double, 4, 1, false, true>(a, react, s);
            else launch_plain<double, 4, 2, false, true>(a, react, s);
        }
    } else {
        return fail(SBG_ERR_INVALID_ARG, "an external source needs an SBG_F32 or SBG_F64 state");
    }
    SBG_LAUNCH_CHECK("step kernel launch (external source)");
    return SBG_OK;
}

double stability_limit(const sbg_params *p, const int64_t dims[3], double band_eps) {
    double inv2 = 0.0;
    for (int a = 0; a < 3; ++a)
        if (dims[a] > 1) inv2 += 1.0 / (p->dx[a] * p->dx[a]);
    double lim = INFINITY;
    for (int s = 0; s < p->nspecies; ++s) {
        double rate = 2.0 * p->D[s] * inv2 + p->decay[s];
        if (s == 0 && p->k_surf > 0.0) rate += p->k_surf / band_eps;
        double l = rate > 0.0 ? 1.0 / rate : INFINITY;
        if (l < lim) lim = l;
    }
    return lim;
}

sbg_status validate_params(sbg_grid g, const sbg_params *p, int ns) {
    if (!p) return fail(SBG_ERR_INVALID_ARG, "null params");
    if (p->nspecies != ns) return fail(SBG_ERR_INVALID_ARG, "params.nspecies differs from the state's");
    for (int a = 0; a < 3; ++a)
        if (!(p->dx[a] > 0.0) || !isfinite(p->dx[a])) return fail(SBG_ERR_INVALID_ARG, "dx must be finite and > 0");
    if (!(p->dt > 0.0) || !isfinite(p->dt)) return fail(SBG_ERR_INVALID_ARG, "dt must be finite and > 0");
    for (int s = 0; s < ns; ++s)
        if (!(p->D[s] >= 0.0) || !isfinite(p->D[s]) || !(p->decay[s] >= 0.0) || !isfinite(p->decay[s]))
            return fail(SBG_ERR_INVALID_ARG, "D and decay must be finite and >= 0");
    if (!(p->k_surf >= 0.0) || !isfinite(p->k_surf)) return fail(SBG_ERR_INVALID_ARG, "k_surf must be finite and >= 0");
    for (int f = 0; f < 6; ++f)
        if (p->face_type[f] != SBG_FACE_NOFLUX && p->face_type[f] != SBG_FACE_DIRICHLET)
            return fail(SBG_ERR_INVALID_ARG, "face_type must be NOFLUX or DIRICHLET");
    if (g->has_eps && (ns != 1 || p->k_surf != 0.0))
        return fail(SBG_ERR_INVALID_ARG, "a diffusivity factor is set: one species and k_surf = 0 only");
    sbg_params pe = *p;
    if (g->has_eps) pe.D[0] = p->D[0] * (double)g->eps_max;  // the largest diffusivity bounds dt
    if (!p->allow_unstable) {
        for (int i = 0; i < g->n_geoms; ++i) {
            double lim = stability_limit(&pe, &g->dims[3 * i], g->band_eps);
            if (p->dt > lim)
                return fail(SBG_ERR_UNSTABLE_DT, "dt " + std::to_string(p->dt) + " above the explicit limit " +
                                                     std::to_string(lim));
        }
    }
    return SBG_OK;
}

constexpr int64_t kGraphSteps = 64;  // steps per captured graph (even: parity preserved)

// Steps one launch of the state's step kernel advances: K for the wavefront
// kernel (SBG_KERNEL_WAVE: 2, SBG_KERNEL_WAVE4: 4) where it applies, else 1.
// Each launch leaves the state in the other buffer, and kGraphSteps / K is
// even, so a graph keeps the buffer parity.
static int steps_per_launch(sbg_grid g, sbg_state st) {
    if (st->variant != SBG_KERNEL_WAVE && st->variant != SBG_KERNEL_WAVE4) return 1;
    if (!wave_kernel_applies(g, st)) return 1;
    return st->variant == SBG_KERNEL_WAVE4 ? 4 : 2;
}

// k steps from buffer src into 1 - src: one wavefront launch (k > 1) or one step.
static sbg_status launch_steps(sbg_grid g, sbg_state st, const sbg_params *p, int src, int k, cudaStream_t s) {
    if (k == 1) return launch_step(g, st, p, src, s);
    StepArgs a;
    fill_args(g, st, p, src, a);
    if (a.held_mask && !a.heldbits) return fail(SBG_ERR_INVALID_ARG, "internal: held bits not prepared");
    cudaError_t e = launch_step_wave(a, g, st, p->k_surf != 0.0, s);
    if (e != cudaSuccess) return cuda_fail(e, "wavefront step kernel launch");
    return SBG_OK;
}

static sbg_status ensure_graph(sbg_grid g, sbg_state st, const sbg_params *p) {
    if (st->graph && st->graph_cur == st->cur && st->graph_variant == st->variant &&
        st->graph_ctas == st->ctas_per_sm && st->graph_eps_version == g->eps_version &&
        st->graph_inject_version == g->inject_version &&
        std::memcmp(&st->graph_params, p, sizeof(*p)) == 0)
        return SBG_OK;
    if (st->graph) {
        cudaGraphExecDestroy(st->graph);
        st->graph = nullptr;
    }
    cudaStream_t cs;
    SBG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    sbg_status rc = SBG_OK;
    if (e == cudaSuccess) {
        int src = st->cur;
        const int k = steps_per_launch(g, st);
        for (int64_t i = 0; i < kGraphSteps && rc == SBG_OK; i += k) {
            rc = launch_steps(g, st, p, src, k, cs);
            src = 1 - src;
        }
        e = cudaStreamEndCapture(cs, &graph);
    }
    if (e == cudaSuccess && rc == SBG_OK) e = cudaGraphInstantiate(&st->graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (rc != SBG_OK) return rc;
    if (e != cudaSuccess) {
        st->graph = nullptr;
        return cuda_fail(e, "step graph capture");
    }
    st->graph_cur = st->cur;
    st->graph_variant = st->variant;
    st->graph_ctas = st->ctas_per_sm;
    st->graph_eps_version = g->eps_version;
    st->graph_inject_version = g->inject_version;
    st->graph_params = *p;
    st->graph_steps = kGraphSteps;
    return SBG_OK;
}

static sbg_status step_n_plain(sbg_grid g, sbg_state st, const sbg_params *p, int64_t nsteps, cudaStream_t s);

// SBG_F32R states: before every kRefreshSteps steps (and before the first
// step after sbg_state_set) the source r is recomputed from b + d and d is
// folded into b, so that d stays the change of the last <= kRefreshSteps steps.
sbg_status step_n(sbg_grid g, sbg_state st, const sbg_params *p, int64_t nsteps, cudaStream_t s) {
    sbg_status prc = prepare_held_bits(g, p, s);
    if (prc != SBG_OK) return prc;
    const int k = steps_per_launch(g, st);
    if (k > 1 && nsteps >= k) {
        prc = prepare_wave(g, st, k, s);
        if (prc != SBG_OK) return prc;
    }
    if (st->dtype != SBG_F32R) return step_n_plain(g, st, p, nsteps, s);
    int64_t done = 0;
    while (done < nsteps) {
        if (!st->r_valid || st->since_refresh >= kRefreshSteps) {
            sbg_status rc = refresh_source(g, st, p, s);
            if (rc != SBG_OK) return rc;
        }
        const int64_t m = std::min<int64_t>(nsteps - done, kRefreshSteps - st->since_refresh);
        sbg_status rc = step_n_plain(g, st, p, m, s);
        if (rc != SBG_OK) return rc;
        done += m;
        st->since_refresh += m;
    }
    return SBG_OK;
}

static sbg_status step_n_plain(sbg_grid g, sbg_state st, const sbg_params *p, int64_t nsteps, cudaStream_t s) {
    int64_t done = 0;
    if (nsteps >= kGraphSteps && g->nb > 0) {
        sbg_status rc = ensure_graph(g, st, p);
        if (rc != SBG_OK) return rc;
        while (nsteps - done >= kGraphSteps) {
            SBG_CUDA(cudaGraphLaunch(st->graph, s));
            done += kGraphSteps;
        }
    }
    const int k = steps_per_launch(g, st);
    while (done < nsteps) {
        const int m = nsteps - done >= k ? k : 1;
        sbg_status rc = launch_steps(g, st, p, st->cur, m, s);
        if (rc != SBG_OK) return rc;
        st->cur = 1 - st->cur;
        done += m;
    }
    return SBG_OK;
}

}  // namespace sbg

using namespace sbg;

extern "C" double sbg_stability_limit(const sbg_params *p, const int64_t dims[3], double band_eps) {
    if (!p || !dims) return -1.0;
    return stability_limit(p, dims, band_eps > 0 ? band_eps : 1.0);
}

extern "C" sbg_status sbg_step(sbg_grid g, sbg_state st, const sbg_params *p, int64_t nsteps, void *stream) {
    TraceRange trace_range("sbg_step");
    if (!g || !st || !p) return fail(SBG_ERR_INVALID_ARG, "sbg_step: null pointer");
    if (st->grid != g) return fail(SBG_ERR_INVALID_ARG, "sbg_step: state of another grid");
    if (nsteps < 0) return fail(SBG_ERR_INVALID_ARG, "sbg_step: nsteps < 0");
    if (st->dtype == SBG_F32X2 && st->ns != 1)
        return fail(SBG_ERR_INVALID_ARG, "sbg_step: SBG_F32X2 states hold one species");
    sbg_status rc = validate_params(g, p, st->ns);
    if (rc != SBG_OK) return rc;
    return step_n(g, st, p, nsteps, (cudaStream_t)stream);
}

extern "C" sbg_status sbg_state_set_kernel(sbg_state st, int32_t variant, int32_t ctas_per_sm) {
    if (!st) return fail(SBG_ERR_INVALID_ARG, "sbg_state_set_kernel: null state");
    if (variant < SBG_KERNEL_AUTO || variant > SBG_KERNEL_WAVE4 || ctas_per_sm < 0 || ctas_per_sm > 64)
        return fail(SBG_ERR_INVALID_ARG, "sbg_state_set_kernel: bad variant or ctas_per_sm");
    if (variant >= SBG_KERNEL_PIPELINED && variant < SBG_KERNEL_STREAM && st->dtype == SBG_F64)
        return fail(SBG_ERR_INVALID_ARG, "sbg_state_set_kernel: no pipelined kernel for FP64 states");
    st->variant = variant;
    st->ctas_per_sm = ctas_per_sm;
    return SBG_OK;
}

namespace sbg {
// One pipelined step from buffer `src` over an explicit device work list of
// (first block, block count) spans; used by the batch solver.
sbg_status launch_step_work(sbg_grid g, sbg_state st, const sbg_params *p, int src, const int64_t *items,
                            int64_t nitems, cudaStream_t s) {
    StepArgs a;
    fill_args(g, st, p, src, a);
    if (a.held_mask && !a.heldbits) return fail(SBG_ERR_INVALID_ARG, "internal: held bits not prepared");
    a.items = items;
    a.nitems = nitems;
    cudaError_t e = cudaSuccess;
    // the streaming kernel takes work-list spans of at most 16 blocks (the spans the batch solver
    // makes for these states: step_work_group_voxels / B^3 <= 1024 / 64)
    const bool react = p->k_surf != 0.0;
    if ((st->variant == SBG_KERNEL_AUTO || st->variant == SBG_KERNEL_STREAM) && stream_kernel_applies(g, st) &&
        !(st->dtype == SBG_F32R && react) &&
        step_work_group_voxels(st->dtype, st->ns, g->has_eps, halo_variant_of(st->variant)) <= 16 * g->b3()) {
        e = launch_step_stream(a, g, st->ns, react, st->ctas_per_sm, s);
        if (e != cudaSuccess) return cuda_fail(e, "streaming step kernel launch (work list)");
        return SBG_OK;
    }
    if (!launch_step_pipe(a, st->dtype, st->ns, g->B, p->k_surf != 0.0,
                          halo_variant_of(st->variant), st->ctas_per_sm, g->err, s, &e))
        return fail(SBG_ERR_INVALID_ARG, "batched stepping needs an FP32-based state (SBG_F32, SBG_F32X2 or "
                                         "SBG_F32R) and fewer than 2^31 voxel slots (blocks x B^3)");
    if (e != cudaSuccess) return cuda_fail(e, "pipelined step kernel launch (work list)");
    return SBG_OK;
}
}  // namespace sbg

extern "C" sbg_status sbg_debug_stall_stage(sbg_grid g, int64_t group, int64_t wait_cycles) {
    if (!g) return fail(SBG_ERR_INVALID_ARG, "sbg_debug_stall_stage: null grid");
    if (group >= 0 && (wait_cycles < 1 || wait_cycles > (int64_t(1) << 31) || group > INT32_MAX))
        return fail(SBG_ERR_INVALID_ARG, "sbg_debug_stall_stage: 0 <= group <= 2^31 - 1, 1 <= wait_cycles <= 2^31");
    g->inject_stall_group = group >= 0 ? (int)group : -1;
    g->inject_wait_cycles = group >= 0 ? (long long)wait_cycles : 0;
    g->inject_version++;
    return SBG_OK;
}

extern "C" sbg_status sbg_debug_set_face(sbg_grid g, int64_t block, int32_t face, int32_t id, int32_t *old_id) {
    if (!g) return fail(SBG_ERR_INVALID_ARG, "sbg_debug_set_face: null grid");
    if (block < 0 || block >= g->nb || face < 0 || face > 5)
        return fail(SBG_ERR_INVALID_ARG, "sbg_debug_set_face: block or face out of range");
    int32_t *slot = g->face_nbr + block * 6 + face;
    if (old_id) SBG_CUDA(cudaMemcpy(old_id, slot, sizeof(int32_t), cudaMemcpyDeviceToHost));
    SBG_CUDA(cudaMemcpy(slot, &id, sizeof(int32_t), cudaMemcpyHostToDevice));
    g->inject_version++;  // captured step graphs hold no table contents, but re-capture anyway
    return SBG_OK;
}
