// Adjoint of the time step, with checkpointing (no counterpart in the paper:
// the differentiation pattern of this library).
//
// The forward step is linear, u^{n+1} = M u^n, with for a free active voxel i
// of species s
//   M_ii = 1 - dt sum_{active nbr j} c_a - dt (decay_s + [s = A] k w_i),
//   M_ij = dt c_a for every active neighbour j (held ones included),
//   d u_B,i^{n+1} / d u_A,i^n = dt k w_i   (two species),
// and identity rows for Dirichlet-held voxels.  Held values are not free
// parameters, so lambda is 0 on held (and inactive) voxels, and
//   lambda^n = M^T lambda^{n+1}:
//   lambda_i^n = lambda_i (1 - dt sum c - dt rate_i) + dt sum_{free active nbr j} c_a lambda_j
//                (+ dt k w_i lambda_B,i for species A).
// The same kernel accumulates this step's contribution to
//   dL/dD_s += sum_i lambda_{s,i}^{n+1} dt g_{s,i}(u^n),  g = sum_a [(u~+ - u) - (u - u~-)] / dx_a^2,
//   dL/dk   += sum_i dt w_i u_{A,i}^n (lambda_{B,i}^{n+1} - lambda_{A,i}^{n+1}),
// with u~ the no-flux mirror.  Per-CTA partial sums go to a buffer of the tape
// and one CTA adds them, in a fixed order, to the tape's accumulator.
//
// Checkpointing: sbg_forward_record keeps the state every K steps; sbg_adjoint
// walks the segments backwards, recomputes the K states of a segment from its
// checkpoint (each step writes straight into the next recompute buffer, so no
// state is copied) and runs K adjoint steps over them.  Each CTA adds its
// partial sums to its own FP64 slot in every adjoint step (a fixed order: the
// steps'), and one CTA sums the slots once at the end.
#include <math.h>

#include <cstring>
#include <vector>

#include "sbg_internal.cuh"
#include "sbg_step.cuh"
#include "sbg_trace.cuh"

struct sbg_tape_s {
    sbg_grid grid = nullptr;
    sbg_params p{};
    int ns = 1;
    sbg_dtype dtype = SBG_F32;
    int64_t nsteps = 0, K = 1;
    size_t state_bytes = 0;          // one species-set of one state, bytes
    size_t ghost_bytes = 0;          // the ghost block before each species array of a buffer
    size_t buf_bytes = 0;            // one buffer: per species a ghost block and the array
    std::vector<void *> ckpt;        // states at n = 0, K, 2K, ...
    std::vector<void *> seg;         // recompute buffer: up to K states
    double *partials = nullptr;      // per-CTA sums, accumulated over the adjoint steps
    double *acc = nullptr;           // dL/dD_0, dL/dD_1, dL/dk
    int64_t nctas = 0;
    int64_t bytes = 0;
};

namespace sbg {

sbg_status step_n(sbg_grid g, sbg_state st, const sbg_params *p, int64_t nsteps, cudaStream_t s);
sbg_status launch_step(sbg_grid g, sbg_state st, const sbg_params *p, int src, cudaStream_t s);

// Tape buffers hold, per species, a ghost block of sentinels and then the
// species array (the layout of a state's buffers, so that the streaming
// kernels can step the recompute buffers).  Species sp of buffer `buf`:
static void *tape_sp(const sbg_tape_s *tp, const void *buf, int sp) {
    const size_t per = tp->state_bytes / tp->ns;
    return (char *)buf + tp->ghost_bytes + (size_t)sp * (per + tp->ghost_bytes);
}

template <typename T>
__global__ void k_tape_ghosts(T *base, int64_t stride_elems, int ns, int ghost_elems) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ns * ghost_elems) return;
    base[(int64_t)(i / ghost_elems) * stride_elems + i % ghost_elems] = sentinel<T>();
}

template <typename T>
struct AdjArgs {
    const T *lam_in[2];
    T *lam_out[2];
    const T *u[2];
    const int4 *blocks;
    const int32_t *face;
    const int32_t *wslab;
    const T *w;
    const int32_t *gdims;
    int64_t nb;
    int held_mask;
    T c[2][3];      // D_s / dx_a^2
    T inv2[3];      // 1 / dx_a^2
    T dt, decay[2], k;
    double *partials;
};

// Per-voxel gradient terms and their warp sums are formed in the state's
// precision (one product per voxel, 32 terms per warp); warp partials are
// converted to FP64 and everything above the warp is summed in FP64.
template <typename T, int B, int BPC, int NS>
__global__ void __launch_bounds__(BPC * B * B * B, (sizeof(T) == 8 ? 1 : 2)) k_adjoint(const AdjArgs<T> a) {
    constexpr int B3 = B * B * B;
    constexpr int NT = BPC * B3;
    __shared__ T tl[NS][NT];   // lambda^{n+1}
    __shared__ T tu[NS][NT];   // u^n
    __shared__ double red[NT / 32][3];
    const int tid = threadIdx.x;
    const int j = tid / B3;
    const int l = tid - j * B3;
    const int64_t b = (int64_t)blockIdx.x * BPC + j;
    const bool valid = b < a.nb;
    const int x = l % B, y = (l / B) % B, z = l / (B * B);
    const int off[6] = {B - 1, -(B - 1), (B - 1) * B, -(B - 1) * B, (B - 1) * B * B, -(B - 1) * B * B};
    const bool edge[6] = {x == 0, x == B - 1, y == 0, y == B - 1, z == 0, z == B - 1};

    T hl[NS][6], hu[NS][6];
    int4 bc = make_int4(0, 0, 0, 0);
    if (valid) {
        bc = a.blocks[b];
        int nid[6];
#pragma unroll
        for (int f = 0; f < 6; ++f) nid[f] = edge[f] ? a.face[b * 6 + f] : -1;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            tl[s][tid] = a.lam_in[s][b * B3 + l];
            tu[s][tid] = a.u[s][b * B3 + l];
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                hl[s][f] = nid[f] >= 0 ? a.lam_in[s][(int64_t)nid[f] * B3 + l + off[f]] : sentinel<T>();
                hu[s][f] = nid[f] >= 0 ? a.u[s][(int64_t)nid[f] * B3 + l + off[f]] : sentinel<T>();
            }
        }
    }
    __syncthreads();

    T gD[2] = {T(0), T(0)}, gk = T(0);
    if (valid) {
        const int nx = a.gdims[bc.w * 4 + 0], ny = a.gdims[bc.w * 4 + 1], nz = a.gdims[bc.w * 4 + 2];
        const int gx = bc.x * B + x, gy = bc.y * B + y, gz = bc.z * B + z;
        const bool held_c = is_held(a.held_mask, gx, gy, gz, nx, ny, nz);
        const int step[6] = {-1, 1, -B, B, -B * B, B * B};
        const int ddx[6] = {-1, 1, 0, 0, 0, 0}, ddy[6] = {0, 0, -1, 1, 0, 0}, ddz[6] = {0, 0, 0, 0, -1, 1};
        T w = T(0);
        if (a.k != T(0)) {
            const int ws = a.wslab[b];
            if (ws >= 0) w = a.w[(int64_t)ws * B3 + l];
        }
        T lc[NS];
#pragma unroll
        for (int s = 0; s < NS; ++s) lc[s] = tl[s][tid];
#pragma unroll
        for (int s = 0; s < NS; ++s) {
            const T lam = lc[s];
            T out = lam;
            if (!is_sent(lam)) {
                if (held_c) {
                    out = T(0);
                } else {
                    const T uc = tu[s][tid];
                    T sum_c = T(0), offd = T(0), g = T(0);
#pragma unroll
                    for (int f = 0; f < 6; ++f) {
                        const int ax = f >> 1;
                        const T ln = edge[f] ? hl[s][f] : tl[s][tid + step[f]];
                        const T un = edge[f] ? hu[s][f] : tu[s][tid + step[f]];
                        const bool act = !is_sent(ln);
                        // differences for g with the no-flux mirror: 0 towards an inactive neighbour
                        const T du = act ? (un - uc) : T(0);
                        g += a.inv2[ax] * du;
                        if (act) {
                            sum_c += a.c[s][ax];
                            const bool held_n = is_held(a.held_mask, gx + ddx[f], gy + ddy[f], gz + ddz[f], nx,
                                                        ny, nz);
                            if (!held_n) offd += a.c[s][ax] * ln;
                        }
                    }
                    const T rate = a.decay[s] + (s == 0 ? a.k * w : T(0));
                    out = lam * (T(1) - a.dt * sum_c - a.dt * rate) + a.dt * offd;
                    if (s == 0 && NS == 2) out += a.dt * a.k * w * lc[NS - 1];
                    gD[s] += lam * a.dt * g;
                    if (s == 0 && a.k != T(0)) {
                        const T lb = NS == 2 ? lc[NS - 1] : T(0);
                        gk += a.dt * w * uc * (lb - lam);
                    }
                }
            }
            a.lam_out[s][b * B3 + l] = out;
        }
    }
    // CTA partial sums (warp shuffle, then FP64 in shared memory, fixed order)
    T v[3] = {gD[0], gD[1], gk};
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
        if (lane == 0) red[warp][q] = (double)v[q];
    }
    __syncthreads();
    if (tid < 3) {
        double acc = 0.0;
        for (int wi = 0; wi < NT / 32; ++wi) acc += red[wi][tid];
        a.partials[(int64_t)blockIdx.x * 3 + tid] += acc;
    }
}

__global__ void k_adj_accum(const double *partials, int64_t nctas, double *acc) {
    __shared__ double sm[256][3];
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t c = threadIdx.x; c < nctas; c += blockDim.x)
        for (int q = 0; q < 3; ++q) v[q] += partials[c * 3 + q];
    for (int q = 0; q < 3; ++q) sm[threadIdx.x][q] = v[q];
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st)
            for (int q = 0; q < 3; ++q) sm[threadIdx.x][q] += sm[threadIdx.x + st][q];
        __syncthreads();
    }
    if (threadIdx.x < 3) acc[threadIdx.x] = sm[0][threadIdx.x];
}

template <typename T>
static void fill_adj(sbg_grid g, const sbg_params *p, AdjArgs<T> &a) {
    std::memset(&a, 0, sizeof(a));
    a.blocks = g->blocks;
    a.face = g->face_nbr;
    a.wslab = g->wslab;
    a.w = sizeof(T) == 8 ? (const T *)g->w64 : (const T *)g->w;
    a.gdims = g->gdims;
    a.nb = g->nb;
    for (int f = 0; f < 6; ++f)
        if (p->face_type[f] == SBG_FACE_DIRICHLET) a.held_mask |= 1 << f;
    for (int s = 0; s < 2; ++s) {
        for (int ax = 0; ax < 3; ++ax) a.c[s][ax] = (T)(p->D[s] / (p->dx[ax] * p->dx[ax]));
        a.decay[s] = (T)p->decay[s];
    }
    for (int ax = 0; ax < 3; ++ax) a.inv2[ax] = (T)(1.0 / (p->dx[ax] * p->dx[ax]));
    a.dt = (T)p->dt;
    a.k = (T)p->k_surf;
}

template <typename T, int B, int NS>
static sbg_status launch_adj_t(sbg_tape tp, const void *u, const void *const *lin, void *const *lout,
                               cudaStream_t s) {
    constexpr int BPC = (B == 8) ? 1 : 8;
    sbg_grid g = tp->grid;
    AdjArgs<T> a;
    fill_adj<T>(g, &tp->p, a);
    for (int sp = 0; sp < NS; ++sp) {
        a.lam_in[sp] = (const T *)lin[sp];
        a.lam_out[sp] = (T *)lout[sp];
        a.u[sp] = (const T *)tape_sp(tp, u, sp);
    }
    a.partials = tp->partials;
    const int64_t nctas = (g->nb + BPC - 1) / BPC;
    k_adjoint<T, B, BPC, NS><<<(unsigned)nctas, BPC * B * B * B, 0, s>>>(a);
    SBG_LAUNCH_CHECK("adjoint kernel launch");
    return SBG_OK;
}

// One FP64 adjoint step with the one-thread-per-voxel kernel.
static sbg_status launch_adj(sbg_tape tp, const void *u, sbg_state lam, cudaStream_t s) {
    sbg_grid g = tp->grid;
    const void *lin[2] = {lam->val[lam->cur][0], lam->val[lam->cur][1]};
    void *lout[2] = {lam->val[1 - lam->cur][0], lam->val[1 - lam->cur][1]};
    sbg_status rc;
    if (g->B == 8) rc = tp->ns == 1 ? launch_adj_t<double, 8, 1>(tp, u, lin, lout, s) : launch_adj_t<double, 8, 2>(tp, u, lin, lout, s);
    else rc = tp->ns == 1 ? launch_adj_t<double, 4, 1>(tp, u, lin, lout, s) : launch_adj_t<double, 4, 2>(tp, u, lin, lout, s);
    if (rc == SBG_OK) lam->cur = 1 - lam->cur;
    return rc;
}

// lambda := 0 on Dirichlet-held voxels (held values are not free parameters)
template <int B>
__global__ void k_zero_held(float *l0, float *l1, const int4 *blocks, const int32_t *gdims, int held_mask,
                            int64_t nb) {
    constexpr int B3 = B * B * B;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * B3) return;
    const int64_t b = i / B3;
    const int l = (int)(i - b * B3);
    const int4 bc = blocks[b];
    const int gx = bc.x * B + l % B, gy = bc.y * B + (l / B) % B, gz = bc.z * B + l / (B * B);
    if (!is_held(held_mask, gx, gy, gz, gdims[bc.w * 4], gdims[bc.w * 4 + 1], gdims[bc.w * 4 + 2])) return;
    if (!is_sent(l0[i])) l0[i] = 0.f;
    if (l1 && !is_sent(l1[i])) l1[i] = 0.f;
}

static sbg_status zero_held(sbg_tape tp, sbg_state lam, cudaStream_t s) {
    sbg_grid g = tp->grid;
    StepArgs a;
    fill_step_args(g, &tp->p, a);
    if (!a.held_mask || g->nb == 0) return SBG_OK;
    float *l0 = (float *)lam->val[lam->cur][0];
    float *l1 = tp->ns == 2 ? (float *)lam->val[lam->cur][1] : nullptr;
    const int64_t n = g->nb * g->b3();
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (g->B == 8) k_zero_held<8><<<grid, 256, 0, s>>>(l0, l1, g->blocks, g->gdims, a.held_mask, g->nb);
    else k_zero_held<4><<<grid, 256, 0, s>>>(l0, l1, g->blocks, g->gdims, a.held_mask, g->nb);
    SBG_LAUNCH_CHECK("adjoint held-voxel kernel launch");
    return SBG_OK;
}

// One FP32 adjoint step with the pipelined kernel.
static sbg_status launch_adj_pipe(sbg_tape tp, const void *u, sbg_state lam, cudaStream_t s) {
    sbg_grid g = tp->grid;
    if (g->nb * (int64_t)g->b3() >= (int64_t(1) << 31))  // 32-bit slot indices in the kernel
        return fail(SBG_ERR_INVALID_ARG, "the FP32 adjoint needs fewer than 2^31 voxel slots (blocks x B^3)");
    StepArgs a;
    fill_step_args(g, &tp->p, a);
    PipeIO io;
    std::memset(&io, 0, sizeof(io));
    for (int sp = 0; sp < tp->ns; ++sp) {
        io.src[sp] = (const float *)lam->val[lam->cur][sp];
        io.src[tp->ns + sp] = (const float *)tape_sp(tp, u, sp);
        io.dst[sp] = (float *)lam->val[1 - lam->cur][sp];
    }
    io.gsum = tp->partials;
    for (int ax = 0; ax < 3; ++ax) io.inv2[ax] = (float)(1.0 / (tp->p.dx[ax] * tp->p.dx[ax]));
    if (tp->ns == 1 && adjoint_stream_applies(g, lam)) {
        // the streaming form (lambda bitwise the ring kernel's; 4^3 blocks, one species)
        cudaError_t e = launch_adjoint_stream(a, io.src[0], io.src[1], io.dst[0], tp->partials, io.inv2, g, true,
                                              (int)tp->nctas, s);
        if (e != cudaSuccess) return cuda_fail(e, "streaming adjoint kernel launch");
        lam->cur = 1 - lam->cur;
        return SBG_OK;
    }
    int grid = 0;
    // the surface terms always: dL/dk is not 0 at k = 0 (and with k = 0 they leave lambda unchanged)
    cudaError_t e = launch_adjoint_pipe(a, io, tp->ns, g->B, true, (int)tp->nctas, g->err, s, &grid);
    if (e != cudaSuccess) return cuda_fail(e, "pipelined adjoint kernel launch");
    lam->cur = 1 - lam->cur;
    return SBG_OK;
}

// state's current species arrays -> one packed buffer (species-major)
static sbg_status save_state(sbg_tape tp, sbg_state st, void *dst, cudaStream_t s) {
    const size_t per = tp->state_bytes / tp->ns;
    for (int sp = 0; sp < tp->ns; ++sp)
        SBG_CUDA(cudaMemcpyAsync(tape_sp(tp, dst, sp), st->val[st->cur][sp], per, cudaMemcpyDeviceToDevice, s));
    return SBG_OK;
}

// One forward step from packed buffer `src` into packed buffer `dst`, through
// a state object that owns no memory and points at the two buffers.
static sbg_status step_packed(sbg_tape tp, const void *src, void *dst, cudaStream_t s) {
    sbg_state_s view;
    view.grid = tp->grid;
    view.ns = tp->ns;
    view.dtype = tp->dtype;
    view.nslots = (int64_t)(tp->state_bytes / tp->ns / (tp->dtype == SBG_F64 ? 8 : 4));
    for (int sp = 0; sp < tp->ns; ++sp) {
        view.val[0][sp] = tape_sp(tp, src, sp);
        view.val[1][sp] = tape_sp(tp, dst, sp);
    }
    view.has_ghost = true;  // the tape's buffers have a state's layout
    view.variant = SBG_KERNEL_AUTO;
    return launch_step(tp->grid, &view, &tp->p, 0, s);
}

// the ghost blocks of a new tape buffer hold the sentinel
static sbg_status fill_tape_ghosts(sbg_tape tp, void *buf, cudaStream_t s) {
    const int elem = tp->dtype == SBG_F64 ? 8 : 4;
    const int ghost_elems = (int)(tp->ghost_bytes / elem);
    const int64_t stride = (int64_t)((tp->state_bytes / tp->ns + tp->ghost_bytes) / elem);
    const int n = tp->ns * ghost_elems;
    if (elem == 8) k_tape_ghosts<double><<<(n + 255) / 256, 256, 0, s>>>((double *)buf, stride, tp->ns, ghost_elems);
    else k_tape_ghosts<float><<<(n + 255) / 256, 256, 0, s>>>((float *)buf, stride, tp->ns, ghost_elems);
    SBG_LAUNCH_CHECK("tape ghost blocks");
    return SBG_OK;
}

static void tape_free(sbg_tape tp) {
    if (!tp) return;
    for (void *p : tp->ckpt) dfree(p);
    for (void *p : tp->seg) dfree(p);
    dfree(tp->partials);
    dfree(tp->acc);
    delete tp;
}

}  // namespace sbg

using namespace sbg;

extern "C" sbg_status sbg_forward_record(sbg_grid g, sbg_state st, const sbg_params *p, int64_t nsteps,
                                         int64_t checkpoint_every, void *stream, sbg_tape *out) {
    TraceRange trace_range("sbg_forward_record");
    if (!g || !st || !p || !out) return fail(SBG_ERR_INVALID_ARG, "sbg_forward_record: null pointer");
    if (st->grid != g) return fail(SBG_ERR_INVALID_ARG, "sbg_forward_record: state of another grid");
    if (nsteps < 0 || checkpoint_every < 1) return fail(SBG_ERR_INVALID_ARG, "sbg_forward_record: nsteps >= 0, checkpoint_every >= 1");
    if (st->dtype == SBG_F32X2) return fail(SBG_ERR_INVALID_ARG, "sbg_forward_record: SBG_F32 or SBG_F64 states only");
    sbg_status rc = validate_params(g, p, st->ns);
    if (rc != SBG_OK) return rc;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    sbg_tape tp = new sbg_tape_s();
    tp->grid = g;
    tp->p = *p;
    tp->ns = st->ns;
    tp->dtype = st->dtype;
    tp->nsteps = nsteps;
    tp->K = checkpoint_every;
    tp->state_bytes = (size_t)st->nslots * st->elem() * st->ns;
    tp->ghost_bytes = ((size_t)g->b3() * st->elem() + 255) / 256 * 256;
    tp->buf_bytes = tp->state_bytes + (size_t)st->ns * tp->ghost_bytes;
    const int64_t nck = nsteps == 0 ? 1 : (nsteps + checkpoint_every - 1) / checkpoint_every;
    auto alloc = [&](void **pp, size_t bytes) -> sbg_status {
        cudaError_t e = dmalloc((void **)pp, bytes > 0 ? bytes : 16);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (tape)");
        tp->bytes += (int64_t)bytes;
        return SBG_OK;
    };
    for (int64_t c = 0; c < nck && rc == SBG_OK; ++c) {
        void *q = nullptr;
        rc = alloc(&q, tp->buf_bytes);
        if (rc == SBG_OK) rc = fill_tape_ghosts(tp, q, s);
        tp->ckpt.push_back(q);
        if (rc == SBG_OK) rc = save_state(tp, st, q, s);
        if (rc == SBG_OK) {
            const int64_t n = std::min<int64_t>(checkpoint_every, nsteps - c * checkpoint_every);
            if (n > 0) rc = step_n(g, st, p, n, s);
        }
    }
    const int BPC = g->B == 8 ? 1 : 8;
    // one partial-sum slot per CTA of either adjoint kernel
    tp->nctas = std::max<int64_t>(2048, (g->nb + BPC - 1) / BPC);
    if (rc == SBG_OK) rc = alloc((void **)&tp->partials, sizeof(double) * 3 * tp->nctas);
    if (rc == SBG_OK) rc = alloc((void **)&tp->acc, sizeof(double) * 3);
    if (rc != SBG_OK) {
        tape_free(tp);
        return rc;
    }
    *out = tp;
    return SBG_OK;
}

extern "C" sbg_status sbg_adjoint(sbg_grid g, sbg_tape tp, sbg_state lam, double *grad, void *stream) {
    TraceRange trace_range("sbg_adjoint");
    if (!g || !tp || !lam || !grad) return fail(SBG_ERR_INVALID_ARG, "sbg_adjoint: null pointer");
    if (tp->grid != g || lam->grid != g) return fail(SBG_ERR_INVALID_ARG, "sbg_adjoint: tape or state of another grid");
    if (lam->dtype != tp->dtype || lam->ns != tp->ns)
        return fail(SBG_ERR_INVALID_ARG, "sbg_adjoint: lambda state must match the recorded state's dtype and species");
    cudaStream_t s = (cudaStream_t)stream;
    SBG_CUDA(cudaMemsetAsync(tp->partials, 0, sizeof(double) * 3 * tp->nctas, s));
    sbg_status rc = prepare_held_bits(g, &tp->p, s);
    if (rc == SBG_OK && tp->dtype == SBG_F32) rc = zero_held(tp, lam, s);
    if (rc != SBG_OK) return rc;
    const int64_t K = tp->K;
    // recompute buffers for u^{n0+1} .. u^{n0+K-1} (u^{n0} is the checkpoint itself)
    while ((int64_t)tp->seg.size() < std::min<int64_t>(K, std::max<int64_t>(tp->nsteps, 1)) - 1) {
        void *q = nullptr;
        cudaError_t e = dmalloc((void **)&q, tp->buf_bytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (tape recompute buffer)");
        tp->bytes += (int64_t)tp->buf_bytes;
        tp->seg.push_back(q);
        rc = fill_tape_ghosts(tp, q, s);
        if (rc != SBG_OK) return rc;
    }
    const int64_t nck = (int64_t)tp->ckpt.size();
    for (int64_t c = nck - 1; c >= 0 && rc == SBG_OK; --c) {
        const int64_t n0 = c * K;
        const int64_t len = std::min<int64_t>(K, tp->nsteps - n0);
        if (len <= 0) continue;
        auto u_at = [&](int64_t m) -> void * { return m == 0 ? tp->ckpt[c] : tp->seg[m - 1]; };
        for (int64_t m = 1; m < len && rc == SBG_OK; ++m) rc = step_packed(tp, u_at(m - 1), u_at(m), s);
        for (int64_t m = len - 1; m >= 0 && rc == SBG_OK; --m)
            rc = tp->dtype == SBG_F32 ? launch_adj_pipe(tp, u_at(m), lam, s) : launch_adj(tp, u_at(m), lam, s);
    }
    if (rc == SBG_OK) {
        k_adj_accum<<<1, 256, 0, s>>>(tp->partials, tp->nctas, tp->acc);
        SBG_LAUNCH_CHECK("adjoint sum kernel launch");
    }
    if (rc != SBG_OK) return rc;
    SBG_CUDA(cudaMemcpyAsync(g->red_host, tp->acc, sizeof(double) * 3, cudaMemcpyDeviceToHost, s));
    SBG_CUDA(cudaStreamSynchronize(s));
    rc = check_device_error(g, s);
    if (rc != SBG_OK) return rc;
    grad[0] = g->red_host[0];
    grad[1] = g->red_host[1];
    grad[2] = g->red_host[2];
    return SBG_OK;
}

extern "C" sbg_status sbg_tape_info(sbg_tape tp, int64_t *device_bytes, int64_t *n_checkpoints) {
    if (!tp) return fail(SBG_ERR_INVALID_ARG, "sbg_tape_info: null tape");
    if (device_bytes) *device_bytes = tp->bytes;
    if (n_checkpoints) *n_checkpoints = (int64_t)tp->ckpt.size();
    return SBG_OK;
}

extern "C" void sbg_tape_destroy(sbg_tape tp) { tape_free(tp); }
