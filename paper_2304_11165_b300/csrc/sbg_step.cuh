// Arguments and per-voxel helpers shared by the step kernels.
#pragma once
#include "sbg_internal.cuh"

namespace sbg {

template <typename R>
struct StepCoef {
    R c[2][3];       // D_s / dx_a^2
    R dt;
    R decay[2];
    R k;
};

struct StepArgs {
    const void *in[2];
    void *out[2];
    const float *in_lo[2];
    float *out_lo[2];
    const int4 *blocks;
    const int32_t *face;     // [nb * 6]
    const int32_t *wslab;
    const float *w;
    const double *w64;
    const float *pad;        // 4 sentinels, then 4 zeros
    const int32_t *gdims;
    const uint64_t *heldbits;  // per block, B^3 bits: voxel held by a Dirichlet face (null without)
    int64_t nb;
    const float *src_term;   // SBG_F32R: per-slot source r = L_h b of the correction step
    const float *eps;        // inhomogeneous diffusion: per-slot diffusivity factor (null: constant D)
    const double *eps64;     //   the same in FP64
    const int64_t *items;    // optional work list for the pipelined kernel: (first block, count)
    int64_t nitems;          //   pairs, each within one geometry and at most 512 voxels
    const void *ext[2];      // external source S_s per slot (state precision; null: none)
    double ext_scale;        //   its time factor a_n for this step: the term a_n S_s(x)
    int held_mask;           // bit f: face f is Dirichlet
    int stall_group;         // test hook: the ring kernels never copy this group (-1: none)
    long long wait_cycles;   // bound of every wait on a ring stage (SM cycles)
    int *err;                // the grid's device error word
    StepCoef<float> cf;
    StepCoef<double> cd;
};

template <typename R> __device__ __forceinline__ const StepCoef<R> &coef(const StepArgs &a);
template <> __device__ __forceinline__ const StepCoef<float> &coef<float>(const StepArgs &a) { return a.cf; }
template <> __device__ __forceinline__ const StepCoef<double> &coef<double>(const StepArgs &a) { return a.cd; }

__device__ __forceinline__ bool is_held(int mask, int gx, int gy, int gz, int nx, int ny, int nz) {
    return ((mask & 1) && gx == 0) || ((mask & 2) && gx == nx - 1) || ((mask & 4) && gy == 0) ||
           ((mask & 8) && gy == ny - 1) || ((mask & 16) && gz == 0) || ((mask & 32) && gz == nz - 1);
}

template <typename T>
__device__ __forceinline__ T mirror(T v, T c) { return is_sent(v) ? c : v; }

// The per-voxel FTCS update with the rounding of every operation pinned
// (explicit _rn intrinsics), so that all step kernels produce bitwise the
// same value for the same neighbourhood whatever their data movement:
//   u' = u + dt ( sum_a c_a [(u_{+a} - u) - (u - u_{-a})] - decay u + t )
// with t = -k w u_A for species A and +k w u_A for species B.
// The same update given the x second difference dx = (xp - u) - (u - xm)
// (the pipelined kernel forms the x differences once per row and shares them
// between neighbouring voxels).
__device__ __forceinline__ float fused_update_dx(float u, float dx, float ym, float yp, float zm, float zp,
                                                 const float c[3], float dt, float decay, float t) {
    const float dy = __fsub_rn(__fsub_rn(yp, u), __fsub_rn(u, ym));
    const float dz = __fsub_rn(__fsub_rn(zp, u), __fsub_rn(u, zm));
    const float lap = __fmaf_rn(c[2], dz, __fmaf_rn(c[1], dy, __fmul_rn(c[0], dx)));
    const float react = __fmaf_rn(-decay, u, t);
    return __fmaf_rn(dt, __fadd_rn(lap, react), u);
}
__device__ __forceinline__ float fused_update(float u, float xm, float xp, float ym, float yp, float zm,
                                              float zp, const float c[3], float dt, float decay,
                                              float t) {
    const float dx = __fsub_rn(__fsub_rn(xp, u), __fsub_rn(u, xm));
    return fused_update_dx(u, dx, ym, yp, zm, zp, c, dt, decay, t);
}
__device__ __forceinline__ double fused_update(double u, double xm, double xp, double ym, double yp,
                                               double zm, double zp, const double c[3], double dt,
                                               double decay, double t) {
    const double dx = __dsub_rn(__dsub_rn(xp, u), __dsub_rn(u, xm));
    const double dy = __dsub_rn(__dsub_rn(yp, u), __dsub_rn(u, ym));
    const double dz = __dsub_rn(__dsub_rn(zp, u), __dsub_rn(u, zm));
    const double lap = __fma_rn(c[2], dz, __fma_rn(c[1], dy, __dmul_rn(c[0], dx)));
    const double react = __fma_rn(-decay, u, t);
    return __fma_rn(dt, __dadd_rn(lap, react), u);
}

__device__ __forceinline__ float fma_pinned(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_pinned(double a, double b, double c) { return __fma_rn(a, b, c); }

// Inhomogeneous diffusion (the functor of Appendix B Listing 6): given the
// one-sided differences dp_a = u~_{+a} - u and dm_a = u - u~_{-a} (0 towards a
// neighbour outside Omega) and the factors of the centre (ec) and of the six
// neighbours (en: -x, +x, -y, +y, -z, +z; any finite value where the
// difference is 0), with c_a = D / dx_a^2:
//   u' = u + dt ( sum_a c_a [ (ec + en_{+a})/2 dp_a - (ec + en_{-a})/2 dm_a ] - decay u ).
// (FP32 and FP64, with every rounding pinned so that all kernels agree bitwise)
__device__ __forceinline__ float inh_update(float u, const float dp[3], const float dm[3], float ec,
                                            const float en[6], const float c[3], float dt, float decay) {
    float tx[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float fp = __fmul_rn(__fadd_rn(ec, en[2 * ax + 1]), 0.5f);
        const float fm = __fmul_rn(__fadd_rn(ec, en[2 * ax]), 0.5f);
        tx[ax] = __fsub_rn(__fmul_rn(fp, dp[ax]), __fmul_rn(fm, dm[ax]));
    }
    const float lap = __fmaf_rn(c[2], tx[2], __fmaf_rn(c[1], tx[1], __fmul_rn(c[0], tx[0])));
    const float react = __fmul_rn(-decay, u);
    return __fmaf_rn(dt, __fadd_rn(lap, react), u);
}
__device__ __forceinline__ double inh_update(double u, const double dp[3], const double dm[3], double ec,
                                             const double en[6], const double c[3], double dt, double decay) {
    double tx[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const double fp = __dmul_rn(__dadd_rn(ec, en[2 * ax + 1]), 0.5);
        const double fm = __dmul_rn(__dadd_rn(ec, en[2 * ax]), 0.5);
        tx[ax] = __dsub_rn(__dmul_rn(fp, dp[ax]), __dmul_rn(fm, dm[ax]));
    }
    const double lap = __fma_rn(c[2], tx[2], __fma_rn(c[1], tx[1], __dmul_rn(c[0], tx[0])));
    const double react = __dmul_rn(-decay, u);
    return __fma_rn(dt, __dadd_rn(lap, react), u);
}

// Error-free sum a + b = s + e (Knuth's two-sum, exact in FP32).
__device__ __forceinline__ float two_sum(float a, float b, float &e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// Compensated update of one voxel: value = hi + lo.  Per axis, the second
// difference of hi, X_a = (hi_- - hi) + (hi_+ - hi), and of lo are formed
// separately.  At a steady state the X_a are not small, only their sum over
// the three axes vanishes, so c_a X_a are combined with exact products
// (fma) and error-free two-sums, and every rounding error joins the lo part;
// the FP32 rounding of that cross-axis sum would otherwise leave the
// iteration's fixed point ~1e-9 (relative residual) away from the true steady
// state.  The increment d is added to hi with an error-free two-sum and the
// pair is renormalised, so increments far below one FP32 ulp of the state
// accumulate in lo instead of being rounded away.
__device__ __forceinline__ void fused_update_x2(float hc, float lc, const float nh[6], const float nl[6],
                                                const float c[3], float dt, float rate, float &rh,
                                                float &rl) {
    float p[3], lo = 0.f;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const float x = __fadd_rn(__fsub_rn(nh[2 * ax], hc), __fsub_rn(nh[2 * ax + 1], hc));
        const float xl = __fadd_rn(__fsub_rn(nl[2 * ax], lc), __fsub_rn(nl[2 * ax + 1], lc));
        p[ax] = __fmul_rn(c[ax], x);
        lo = __fadd_rn(lo, __fmaf_rn(c[ax], x, -p[ax]));  // exact rounding error of the product
        lo = __fmaf_rn(c[ax], xl, lo);
    }
    float e1, e2;
    float sum = two_sum(p[0], p[1], e1);
    sum = two_sum(sum, p[2], e2);
    const float lap = __fadd_rn(sum, __fadd_rn(__fadd_rn(e1, e2), lo));
    const float react = __fmul_rn(-rate, __fadd_rn(hc, lc));
    const float d = __fmul_rn(dt, __fadd_rn(lap, react));
    const float s = __fadd_rn(hc, d);
    const float bb = __fsub_rn(s, hc);
    const float e = __fadd_rn(__fsub_rn(hc, __fsub_rn(s, bb)), __fsub_rn(d, bb));
    const float l2 = __fadd_rn(lc, e);
    rh = __fadd_rn(s, l2);
    rl = __fsub_rn(l2, __fsub_rn(rh, s));
}

// Grid tables and coefficients of a step (no state arrays); sbg_step.cu.
void fill_step_args(sbg_grid g, const sbg_params *p, StepArgs &a);

// Double-float accumulation (value = hi + lo): adds (h2, l2) to (h, l).
__device__ __forceinline__ void df_add(float &h, float &l, float h2, float l2) {
    float e;
    const float s = two_sum(h, h2, e);
    e = __fadd_rn(e, __fadd_rn(l, l2));
    h = __fadd_rn(s, e);
    l = __fsub_rn(e, __fsub_rn(h, s));
}

// Arrays of one pipelined launch beyond StepArgs (set by the launchers).
struct PipeIO {
    const float *src[4];  // streamed arrays, in the kernel mode's order
    float *dst[2];        // written arrays
    double *gsum;         // adjoint: per-CTA sums of dL/dD_0, dL/dD_1, dL/dk, added to across launches
    float inv2[3];        // adjoint: 1 / dx_a^2
};

// halo_variant: 0 halo loaded when its group comes up, 1 prefetched one group
// ahead in registers, 2 copied one group ahead with cp.async (sbg_step_pipe.cu).
// voxels per work-list span the pipelined step kernel takes for this state
// (1024 for the two-row kernel's modes, else 512)
int step_work_group_voxels(sbg_dtype dtype, int ns, bool eps, int halo_variant);
bool launch_step_pipe(const StepArgs &a, sbg_dtype dtype, int ns, int B, bool react, int halo_variant,
                      int ctas_per_sm, int *err_flag, cudaStream_t s, cudaError_t *launch_err);
// the halo variant of a state's kernel choice (SBG_KERNEL_AUTO: cp.async one
// group ahead, measured as fast as or faster than the others on every workload)
inline int halo_variant_of(int variant) {
    return variant == SBG_KERNEL_PIPELINED_PREFETCH ? 1 : variant == SBG_KERNEL_PIPELINED ? 0 : 2;
}

// Streaming step kernel (sbg_step_stream.cu): SBG_F32 states of one or two
// species on 4^3 blocks with ghost blocks, no diffusivity factor, no work list.
bool stream_kernel_applies(sbg_grid g, sbg_state st);
cudaError_t launch_step_stream(const StepArgs &a, sbg_grid g, int ns, bool react, int ctas_per_sm, cudaStream_t s);
// The streaming kernel's inhomogeneous-diffusion form: SBG_F32 states of one
// species on 4^3 blocks with a diffusivity factor.
bool stream_inh_applies(sbg_grid g, sbg_state st);
// ... and its compensated form: SBG_F32X2 states (one species) on 4^3 blocks.
bool stream_x2_applies(sbg_grid g, sbg_state st);
cudaError_t launch_step_stream_x2(const StepArgs &a, sbg_grid g, bool react, int ctas_per_sm, cudaStream_t s);
cudaError_t launch_step_stream_inh(const StepArgs &a, sbg_grid g, int ctas_per_sm, cudaStream_t s);

// Wavefront kernel (sbg_step_stream.cu): K steps per launch of the streaming
// kernel's states on a plane-ordered grid of one geometry, the intermediate
// steps in L2-sized plane rings.  prepare_wave builds the state's plan (host
// synchronisation; call it before any stream capture); launch_step_wave runs
// K steps from a.in into a.out; wave_destroy frees the plan.
bool wave_kernel_applies(sbg_grid g, sbg_state st);
sbg_status prepare_wave(sbg_grid g, sbg_state st, int K, cudaStream_t s);
cudaError_t launch_step_wave(const StepArgs &a, sbg_grid g, sbg_state st, bool react, cudaStream_t s);
// The ticket order of a wavefront launch over planes of the given block
// counts, in tickets of up to ticket_blocks blocks: false when some ticket would wait on a later
// one (or bad K, L, R, ticket_blocks).
bool wave_plan_tickets(const std::vector<int> &blocks_per_plane, int K, int L, int R, int ticket_blocks,
                       std::vector<int4> &tick, std::vector<int4> &plane, int &maxplane);

// One adjoint step of one FP32 species on 4^3 blocks with the streaming
// structure (sbg_adjoint_stream.cu): lambda^{n+1} from a state (ghost block
// before it), u^n from a tape buffer laid out the same way; each CTA adds its
// sums of dL/dD and dL/dk to gsum[cta * 3 + 0 / 2]; at most max_ctas CTAs.
bool adjoint_stream_applies(sbg_grid g, sbg_state lam);
cudaError_t launch_adjoint_stream(const StepArgs &a, const float *lam_in, const float *u_in, float *lam_out,
                                  double *gsum, const float inv2[3], sbg_grid g, bool react, int max_ctas,
                                  cudaStream_t s);

// One adjoint step on FP32 arrays with the pipelined kernel: io.src = lambda^{n+1}
// (NS arrays) then u^n (NS arrays), io.dst = lambda^n.  *grid_out receives the
// number of CTAs (each adds to io.gsum[cta * 3 + q]); at most max_ctas are used.
cudaError_t launch_adjoint_pipe(const StepArgs &a, const PipeIO &io, int ns, int B, bool react, int max_ctas,
                                int *err_flag, cudaStream_t s, int *grid_out);

}  // namespace sbg
