// FP64 reductions over the block-layout state: mass (the monitored total of
// Sec. 3.4), x-face fluxes, the residual ||L_h u||_2 and min/max/non-finite
// counts; effective diffusivity and tortuosity (Eq. 2); the steady-state
// driver.
//
// FP32 and compensated states: each thread evaluates the residual and
// accumulates its sums in double-float arithmetic (hi + lo FP32 pairs with
// error-free two-sums and fma products, ~48-bit significand), warps combine
// the pairs with __shfl_down_sync, and FP64 starts at the warp partials; B300
// runs FP64 at a small fraction of its FP32 rate, so per-voxel FP64 would cost
// several times the step itself.  FP64 states accumulate in FP64 throughout.
// Each CTA writes one partial record to the grid's scratch buffer, and a
// single CTA adds the records in a fixed order, so the result is
// deterministic for a given grid.  The residual is evaluated from the stored
// values (hi + lo for compensated states) to ~1e-14 relative, so that a
// steady-state test at a 1e-10 relative residual measures the state, not FP32
// rounding of the stencil.
#include <math.h>

#include <cstring>
#include <vector>
#include <string>

#include "sbg_internal.cuh"
#include "sbg_trace.cuh"

namespace sbg {

sbg_status step_n(sbg_grid g, sbg_state st, const sbg_params *p, int64_t nsteps, cudaStream_t s);

struct RedArgs {
    const void *val[2];
    const float *lo[2];
    const int4 *blocks;
    const int32_t *face;
    const int32_t *wslab;
    const double *w;
    const int32_t *gdims;
    int64_t b_begin, b_count;
    int species, ns, held_mask;
    double c[3];
    double D, decay, k, inv_dx, area, dv;
    double *partials;
    // the same coefficients as double-float pairs, and the FP32 surface weights
    float ch[3], cl[3], dech, decl, kh, kl;
    const float *wf;
    // SBG_F32R: base pair (val[s] is the correction d) and, when set, the
    // source array the reduction writes (r = fl32(L_h u) on free voxels, 0 on held)
    const float *bh, *bl;
    float *rout;
    // inhomogeneous diffusion: diffusivity factor per slot (null: constant D)
    const float *epsf;
    const double *eps64;
    // 1: the residual is not evaluated (its slot reads NaN); the other scalars are unchanged
    int no_residual;
};

template <typename T, bool X2>
__device__ __forceinline__ double load_val(const RedArgs &a, int s, int64_t slot, bool &act) {
    const T v = ((const T *)a.val[s])[slot];
    act = !is_sent(v);
    double d = (double)v;
    if (X2) d += (double)a.lo[s][slot];
    return d;
}

// value of the neighbour of (block b, local l) across face f, with the no-flux rule
template <typename T, bool X2, int B>
__device__ __forceinline__ double nbr_val(const RedArgs &a, int s, int64_t b, int l, int x, int y,
                                          int z, int f, double vc, bool *act_out = nullptr) {
    constexpr int B3 = B * B * B;
    int64_t nb = b;
    int ln = l;
    switch (f) {
        case 0: if (x > 0) ln = l - 1; else { nb = a.face[b * 6 + 0]; ln = l + (B - 1); } break;
        case 1: if (x < B - 1) ln = l + 1; else { nb = a.face[b * 6 + 1]; ln = l - (B - 1); } break;
        case 2: if (y > 0) ln = l - B; else { nb = a.face[b * 6 + 2]; ln = l + (B - 1) * B; } break;
        case 3: if (y < B - 1) ln = l + B; else { nb = a.face[b * 6 + 3]; ln = l - (B - 1) * B; } break;
        case 4: if (z > 0) ln = l - B * B; else { nb = a.face[b * 6 + 4]; ln = l + (B - 1) * B * B; } break;
        default: if (z < B - 1) ln = l + B * B; else { nb = a.face[b * 6 + 5]; ln = l - (B - 1) * B * B; } break;
    }
    if (nb < 0) {
        if (act_out) *act_out = false;
        return vc;
    }
    bool act;
    double v = load_val<T, X2>(a, s, nb * B3 + ln, act);
    if (act_out) *act_out = act;
    return act ? v : vc;
}

// diffusivity factor of the neighbour across face f (0 for an absent block:
// that face carries no flux, the value only has to be finite)
__device__ __forceinline__ int64_t nbr_slot_of(const RedArgs &a, int64_t b, int l, int x, int y, int z, int f,
                                               int B) {
    const int B3 = B * B * B;
    int64_t nb = b;
    int ln = l;
    switch (f) {
        case 0: if (x > 0) ln = l - 1; else { nb = a.face[b * 6 + 0]; ln = l + (B - 1); } break;
        case 1: if (x < B - 1) ln = l + 1; else { nb = a.face[b * 6 + 1]; ln = l - (B - 1); } break;
        case 2: if (y > 0) ln = l - B; else { nb = a.face[b * 6 + 2]; ln = l + (B - 1) * B; } break;
        case 3: if (y < B - 1) ln = l + B; else { nb = a.face[b * 6 + 3]; ln = l - (B - 1) * B; } break;
        case 4: if (z > 0) ln = l - B * B; else { nb = a.face[b * 6 + 4]; ln = l + (B - 1) * B * B; } break;
        default: if (z < B - 1) ln = l + B * B; else { nb = a.face[b * 6 + 5]; ln = l - (B - 1) * B * B; } break;
    }
    return nb < 0 ? -1 : nb * B3 + ln;
}
template <int B>
__device__ __forceinline__ double nbr_eps64(const RedArgs &a, int64_t b, int l, int x, int y, int z, int f) {
    const int64_t q = nbr_slot_of(a, b, l, x, y, z, f, B);
    return q < 0 ? 0.0 : a.eps64[q];
}
template <int B>
__device__ __forceinline__ float nbr_epsf(const RedArgs &a, int64_t b, int l, int x, int y, int z, int f) {
    const int64_t q = nbr_slot_of(a, b, l, x, y, z, f, B);
    return q < 0 ? 0.f : a.epsf[q];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

constexpr int kRedThreads = 256;

template <typename T, bool X2, int B>
__global__ void __launch_bounds__(kRedThreads) k_reduce(const RedArgs a) {
    constexpr int B3 = B * B * B;
    double acc[kNumRed];
    acc[SBG_RED_MASS] = acc[SBG_RED_JIN] = acc[SBG_RED_JOUT] = acc[SBG_RED_RESIDUAL] = 0.0;
    acc[SBG_RED_MIN] = INFINITY;
    acc[SBG_RED_MAX] = -INFINITY;
    acc[SBG_RED_NONFINITE] = acc[SBG_RED_NACTIVE] = 0.0;
    const int s = a.species;
    const int64_t total = a.b_count * B3;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = a.b_begin + t / B3;
        const int l = (int)(t % B3);
        bool act;
        const double v = load_val<T, X2>(a, s, b * B3 + l, act);
        if (!act) continue;
        const int x = l % B, y = (l / B) % B, z = l / (B * B);
        const int4 bc = a.blocks[b];
        const int nx = a.gdims[bc.w * 4 + 0], ny = a.gdims[bc.w * 4 + 1], nz = a.gdims[bc.w * 4 + 2];
        const int gx = bc.x * B + x, gy = bc.y * B + y, gz = bc.z * B + z;
        acc[SBG_RED_NACTIVE] += 1.0;
        if (!isfinite(v)) {
            acc[SBG_RED_NONFINITE] += 1.0;
            continue;
        }
        acc[SBG_RED_MASS] += v * a.dv;
        acc[SBG_RED_MIN] = fmin(acc[SBG_RED_MIN], v);
        acc[SBG_RED_MAX] = fmax(acc[SBG_RED_MAX], v);
        const bool held = ((a.held_mask & 1) && gx == 0) || ((a.held_mask & 2) && gx == nx - 1) ||
                          ((a.held_mask & 4) && gy == 0) || ((a.held_mask & 8) && gy == ny - 1) ||
                          ((a.held_mask & 16) && gz == 0) || ((a.held_mask & 32) && gz == nz - 1);
        const double ec = a.eps64 ? a.eps64[b * B3 + l] : 1.0;
        if (!held && !a.no_residual) {
            double lap = 0.0;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const double vm = nbr_val<T, X2, B>(a, s, b, l, x, y, z, 2 * ax, v);
                const double vp = nbr_val<T, X2, B>(a, s, b, l, x, y, z, 2 * ax + 1, v);
                if (a.eps64) {  // face diffusivities (eps_c + eps_nb) / 2
                    const double fm = 0.5 * (ec + nbr_eps64<B>(a, b, l, x, y, z, 2 * ax));
                    const double fp = 0.5 * (ec + nbr_eps64<B>(a, b, l, x, y, z, 2 * ax + 1));
                    lap += a.c[ax] * (fp * (vp - v) - fm * (v - vm));
                } else {
                    lap += a.c[ax] * ((vp - v) - (v - vm));
                }
            }
            double react = -a.decay * v;
            if (a.k != 0.0) {
                const int ws = a.wslab[b];
                const double w = ws >= 0 ? a.w[(int64_t)ws * B3 + l] : 0.0;
                bool act0;
                const double ua = (s == 0) ? v : load_val<T, X2>(a, 0, b * B3 + l, act0);
                const double tr = a.k * w * ua;
                react += (s == 0) ? -tr : tr;
            }
            const double r = lap + react;
            acc[SBG_RED_RESIDUAL] += r * r;
        }
        if (nx >= 2 && (gx == 0 || gx == nx - 2)) {
            bool act1;
            const double v1 = nbr_val<T, X2, B>(a, s, b, l, x, y, z, 1, v, &act1);
            if (act1) {
                const double f = a.eps64 ? 0.5 * (ec + nbr_eps64<B>(a, b, l, x, y, z, 1)) : 1.0;
                const double j = a.D * f * (v - v1) * a.inv_dx * a.area;
                if (gx == 0) acc[SBG_RED_JIN] += j;
                if (gx == nx - 2) acc[SBG_RED_JOUT] += j;
            }
        }
    }
    __shared__ double sm[kRedThreads / 32][kNumRed];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kNumRed; ++q) {
        double v = acc[q];
        v = (q == SBG_RED_MIN) ? warp_min(v) : (q == SBG_RED_MAX) ? warp_max(v) : warp_sum(v);
        if (lane == 0) sm[warp][q] = v;
    }
    __syncthreads();
    if (threadIdx.x < kNumRed) {
        const int q = threadIdx.x;
        double v = sm[0][q];
        for (int wi = 1; wi < kRedThreads / 32; ++wi)
            v = (q == SBG_RED_MIN) ? fmin(v, sm[wi][q]) : (q == SBG_RED_MAX) ? fmax(v, sm[wi][q]) : v + sm[wi][q];
        if (q == SBG_RED_RESIDUAL && a.no_residual) v = NAN;
        a.partials[(int64_t)blockIdx.x * kNumRed + q] = v;
    }
}

// The final pass of a reduction: the per-CTA records summed in a fixed order
// (min and max for those two), the residual's square root taken last.
__device__ __forceinline__ void reduce_final_body(const double *partials, int nctas, double *out,
                                                  double (*sm)[kNumRed]) {
    double acc[kNumRed];
    for (int q = 0; q < kNumRed; ++q)
        acc[q] = (q == SBG_RED_MIN) ? INFINITY : (q == SBG_RED_MAX) ? -INFINITY : 0.0;
    for (int c = threadIdx.x; c < nctas; c += blockDim.x)
        for (int q = 0; q < kNumRed; ++q) {
            const double v = partials[(int64_t)c * kNumRed + q];
            acc[q] = (q == SBG_RED_MIN) ? fmin(acc[q], v) : (q == SBG_RED_MAX) ? fmax(acc[q], v) : acc[q] + v;
        }
    for (int q = 0; q < kNumRed; ++q) sm[threadIdx.x][q] = acc[q];
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride)
            for (int q = 0; q < kNumRed; ++q) {
                const double o = sm[threadIdx.x + stride][q];
                double &m = sm[threadIdx.x][q];
                m = (q == SBG_RED_MIN) ? fmin(m, o) : (q == SBG_RED_MAX) ? fmax(m, o) : m + o;
            }
        __syncthreads();
    }
    if (threadIdx.x < kNumRed) {
        double v = sm[0][threadIdx.x];
        if (threadIdx.x == SBG_RED_RESIDUAL) v = sqrt(v);
        out[threadIdx.x] = v;
    }
}

__global__ void __launch_bounds__(256) k_reduce_final(const double *partials, int nctas, double *out) {
    __shared__ double sm[256][kNumRed];
    reduce_final_body(partials, nctas, out, sm);
}

// The same final pass for several reductions at once: CTA i sums the records
// [seg[2i], seg[2i] + seg[2i+1]) into out[i * kNumRed ..], each exactly as
// k_reduce_final would.
__global__ void __launch_bounds__(256) k_reduce_final_seg(const double *records, const int *seg, double *out) {
    __shared__ double sm[256][kNumRed];
    const int i = blockIdx.x;
    reduce_final_body(records + (int64_t)seg[2 * i] * kNumRed, seg[2 * i + 1], out + (int64_t)i * kNumRed, sm);
}

// ---------------------------------------------------------------------------
// FP32 / compensated states: double-float per voxel and per warp.
struct DF {
    float h, l;
};
__device__ __forceinline__ float tsum(float a, float b, float &e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    float e;
    const float s = tsum(a.h, b.h, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ DF df_mul(DF a, DF c) {
    const float p = __fmul_rn(a.h, c.h);
    float e = __fmaf_rn(a.h, c.h, -p);
    e = __fmaf_rn(a.h, c.l, e);
    e = __fmaf_rn(a.l, c.h, e);
    const float h = __fadd_rn(p, e);
    return {h, __fsub_rn(e, __fsub_rn(h, p))};
}
__device__ __forceinline__ double df_to_d(DF a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ DF df_shfl_add(DF a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DF b = {__shfl_down_sync(0xffffffffu, a.h, o), __shfl_down_sync(0xffffffffu, a.l, o)};
        a = df_add(a, b);
    }
    return a;
}

// Value modes of the FP32-based reduction: the stored value, hi + lo, or
// (SBG_F32R) base hi + lo plus the correction d.
enum ValMode : int { kVF32 = 0, kVX2 = 1, kVR = 2 };

// value at `slot` as an (unnormalised) double-float pair; false outside Omega
template <int VM>
__device__ __forceinline__ bool load_df(const RedArgs &a, int s, int64_t slot, float &h, float &l) {
    const float v = ((const float *)a.val[s])[slot];
    if (is_sent(v)) return false;
    if (VM == kVF32) {
        h = v;
        l = 0.f;
    } else if (VM == kVX2) {
        h = v;
        l = a.lo[s][slot];
    } else {
        float e;
        h = tsum(a.bh[slot], v, e);
        l = __fadd_rn(e, a.bl[slot]);
    }
    return true;
}

// neighbour (hi, lo) across face f; false when it is outside Omega (mirrored)
template <int VM, int B>
__device__ __forceinline__ bool nbr_f(const RedArgs &a, int s, int64_t b, int l, int x, int y, int z, int f,
                                      float &nh, float &nl) {
    constexpr int B3 = B * B * B;
    int64_t nb = b;
    int ln = l;
    switch (f) {
        case 0: if (x > 0) ln = l - 1; else { nb = a.face[b * 6 + 0]; ln = l + (B - 1); } break;
        case 1: if (x < B - 1) ln = l + 1; else { nb = a.face[b * 6 + 1]; ln = l - (B - 1); } break;
        case 2: if (y > 0) ln = l - B; else { nb = a.face[b * 6 + 2]; ln = l + (B - 1) * B; } break;
        case 3: if (y < B - 1) ln = l + B; else { nb = a.face[b * 6 + 3]; ln = l - (B - 1) * B; } break;
        case 4: if (z > 0) ln = l - B * B; else { nb = a.face[b * 6 + 4]; ln = l + (B - 1) * B * B; } break;
        default: if (z < B - 1) ln = l + B * B; else { nb = a.face[b * 6 + 5]; ln = l - (B - 1) * B * B; } break;
    }
    if (nb < 0) return false;
    return load_df<VM>(a, s, nb * B3 + ln, nh, nl);
}

template <int VM, int B>
__global__ void __launch_bounds__(kRedThreads) k_reduce_f(const RedArgs a) {
    constexpr int B3 = B * B * B;
    DF mass = {0.f, 0.f}, res = {0.f, 0.f}, jin = {0.f, 0.f}, jout = {0.f, 0.f};
    float mn = INFINITY, mx = -INFINITY;
    int nact = 0, nonfin = 0;
    const int s = a.species;
    const DF c[3] = {{a.ch[0], a.cl[0]}, {a.ch[1], a.cl[1]}, {a.ch[2], a.cl[2]}};
    const DF dec = {a.dech, a.decl}, kk = {a.kh, a.kl};
    const int64_t total = a.b_count * B3;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = a.b_begin + t / B3;
        const int l = (int)(t % B3);
        const int64_t slot = b * B3 + l;
        float h, lo;
        if (!load_df<VM>(a, s, slot, h, lo)) continue;
        ++nact;
        if (!isfinite(h)) {
            ++nonfin;
            continue;
        }
        const DF u = {h, lo};
        mass = df_add(mass, u);
        mn = fminf(mn, h);
        mx = fmaxf(mx, h);
        const int x = l % B, y = (l / B) % B, z = l / (B * B);
        const int4 bc = a.blocks[b];
        const int nx = a.gdims[bc.w * 4 + 0], ny = a.gdims[bc.w * 4 + 1], nz = a.gdims[bc.w * 4 + 2];
        const int gx = bc.x * B + x, gy = bc.y * B + y, gz = bc.z * B + z;
        const bool held = ((a.held_mask & 1) && gx == 0) || ((a.held_mask & 2) && gx == nx - 1) ||
                          ((a.held_mask & 4) && gy == 0) || ((a.held_mask & 8) && gy == ny - 1) ||
                          ((a.held_mask & 16) && gz == 0) || ((a.held_mask & 32) && gz == nz - 1);
        if (!held && !a.no_residual) {
            // L_h u = sum_a c_a [(u~- - u) + (u~+ - u)] - rate u (+ transfer), double-float
            DF lap = {0.f, 0.f};
            const float ec = a.epsf ? a.epsf[slot] : 1.f;
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                DF d = {0.f, 0.f};
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    float nh, nl;
                    if (nbr_f<VM, B>(a, s, b, l, x, y, z, 2 * ax + side, nh, nl)) {
                        float e;
                        const float dh = tsum(nh, -h, e);
                        DF diff = {dh, VM != kVF32 ? __fadd_rn(e, __fsub_rn(nl, lo)) : e};
                        if (a.epsf) {  // face diffusivity (eps_c + eps_nb) / 2, exact as a pair
                            float fe;
                            const float fs = tsum(ec, nbr_epsf<B>(a, b, l, x, y, z, 2 * ax + side), fe);
                            diff = df_mul(diff, {__fmul_rn(fs, 0.5f), __fmul_rn(fe, 0.5f)});
                        }
                        d = df_add(d, diff);
                    }
                }
                lap = df_add(lap, df_mul(d, c[ax]));
            }
            DF rate = dec;
            float w = 0.f;
            if (a.k != 0.0) {
                const int ws = a.wslab[b];
                w = ws >= 0 ? a.wf[(int64_t)ws * B3 + l] : 0.f;
                if (s == 0) rate = df_add(rate, df_mul(kk, {w, 0.f}));
            }
            DF r = df_mul(rate, u);
            r = df_add(lap, {-r.h, -r.l});
            if (a.k != 0.0 && s == 1) {
                // + k w u_A
                DF ua = {0.f, 0.f};
                load_df<VM>(a, 0, slot, ua.h, ua.l);
                r = df_add(r, df_mul(df_mul(kk, {w, 0.f}), ua));
            }
            const float p = __fmul_rn(r.h, r.h);
            res = df_add(res, {p, __fmaf_rn(r.h, r.h, -p) + 2.f * r.h * r.l});
            if (VM == kVR && a.rout) a.rout[slot] = __fadd_rn(r.h, r.l);
        } else if (VM == kVR && a.rout) {
            a.rout[slot] = 0.f;
        }
        if (nx >= 2 && (gx == 0 || gx == nx - 2)) {
            float nh, nl;
            if (nbr_f<VM, B>(a, s, b, l, x, y, z, 1, nh, nl)) {
                // u - u_{x+1}, double-float; scaled by D / dx * area below
                float e;
                const float dh = tsum(h, -nh, e);
                DF d = {dh, VM != kVF32 ? __fadd_rn(e, __fsub_rn(lo, nl)) : e};
                if (a.epsf) {
                    float fe;
                    const float fs = tsum(a.epsf[slot], nbr_epsf<B>(a, b, l, x, y, z, 1), fe);
                    d = df_mul(d, {__fmul_rn(fs, 0.5f), __fmul_rn(fe, 0.5f)});
                }
                if (gx == 0) jin = df_add(jin, d);
                if (gx == nx - 2) jout = df_add(jout, d);
            }
        }
    }
    mass = df_shfl_add(mass);
    res = df_shfl_add(res);
    jin = df_shfl_add(jin);
    jout = df_shfl_add(jout);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        nact += __shfl_down_sync(0xffffffffu, nact, o);
        nonfin += __shfl_down_sync(0xffffffffu, nonfin, o);
    }
    __shared__ double sm[kRedThreads / 32][kNumRed];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        const double flux = a.D * a.inv_dx * a.area;
        sm[warp][SBG_RED_MASS] = df_to_d(mass) * a.dv;
        sm[warp][SBG_RED_JIN] = df_to_d(jin) * flux;
        sm[warp][SBG_RED_JOUT] = df_to_d(jout) * flux;
        sm[warp][SBG_RED_RESIDUAL] = df_to_d(res);
        sm[warp][SBG_RED_MIN] = (double)mn;
        sm[warp][SBG_RED_MAX] = (double)mx;
        sm[warp][SBG_RED_NONFINITE] = (double)nonfin;
        sm[warp][SBG_RED_NACTIVE] = (double)nact;
    }
    __syncthreads();
    if (threadIdx.x < kNumRed) {
        const int q = threadIdx.x;
        double v = sm[0][q];
        for (int wi = 1; wi < kRedThreads / 32; ++wi)
            v = (q == SBG_RED_MIN) ? fmin(v, sm[wi][q]) : (q == SBG_RED_MAX) ? fmax(v, sm[wi][q]) : v + sm[wi][q];
        if (q == SBG_RED_RESIDUAL && a.no_residual) v = NAN;
        a.partials[(int64_t)blockIdx.x * kNumRed + q] = v;
    }
}

// The same reduction for constant D (with or without the surface reaction,
// REACT), one thread per x-row of four voxels: the row and its four y/z
// neighbour rows are loaded and combined into double-float values once (not
// once per voxel and face), x neighbours come from the row itself, the
// surface weights and (species B) the row of u_A are read as rows too, and
// the per-voxel arithmetic is that of k_reduce_f in the same order, so r and
// every per-voxel term are bitwise the same.
template <int VM>
__device__ __forceinline__ void load_row_df(const RedArgs &a, int s, int64_t slot, float h[4], float l[4],
                                            bool act[4]) {
    const float4 v = *reinterpret_cast<const float4 *>((const float *)a.val[s] + slot);
    const float vv[4] = {v.x, v.y, v.z, v.w};
    float4 lo4 = make_float4(0.f, 0.f, 0.f, 0.f), bh4 = lo4, bl4 = lo4;
    if (VM == kVX2) lo4 = *reinterpret_cast<const float4 *>(a.lo[s] + slot);
    if (VM == kVR) {
        bh4 = *reinterpret_cast<const float4 *>(a.bh + slot);
        bl4 = *reinterpret_cast<const float4 *>(a.bl + slot);
    }
    const float lv[4] = {lo4.x, lo4.y, lo4.z, lo4.w};
    const float bhv[4] = {bh4.x, bh4.y, bh4.z, bh4.w}, blv[4] = {bl4.x, bl4.y, bl4.z, bl4.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        act[i] = !is_sent(vv[i]);
        if (VM == kVF32) {
            h[i] = vv[i];
            l[i] = 0.f;
        } else if (VM == kVX2) {
            h[i] = vv[i];
            l[i] = lv[i];
        } else {
            float e;
            h[i] = tsum(bhv[i], vv[i], e);
            l[i] = __fadd_rn(e, blv[i]);
        }
    }
}

template <int VM, int B, bool REACT, bool RESID>
__global__ void __launch_bounds__(kRedThreads, 4) k_reduce_rows(const RedArgs a) {
    constexpr int B3 = B * B * B;
    constexpr int RX = B / 4;              // rows of four along x per block row
    constexpr int RPB = B * B * RX;        // threads per block
    constexpr int BPC = kRedThreads / RPB; // blocks per CTA pass
    DF mass = {0.f, 0.f}, res = {0.f, 0.f}, jin = {0.f, 0.f}, jout = {0.f, 0.f};
    float mn = INFINITY, mx = -INFINITY;
    int nact = 0, nonfin = 0;
    const int s = a.species;
    const DF dec = {a.dech, a.decl};
    const int j = threadIdx.x / RPB, rr = threadIdx.x % RPB;
    const int x0 = (rr % RX) * 4, y = (rr / RX) % B, z = rr / (RX * B);
    const int lrow = (z * B + y) * B + x0;
    const int rowbase = lrow - x0;  // x = 0 of this row
    for (int64_t bb = (int64_t)blockIdx.x * BPC; bb < a.b_count; bb += (int64_t)gridDim.x * BPC) {
        if (bb + j >= a.b_count) continue;
        const int64_t b = a.b_begin + bb + j;
        float ch[4], cl[4];
        bool ca[4];
        load_row_df<VM>(a, s, b * B3 + lrow, ch, cl, ca);
        if (!(ca[0] || ca[1] || ca[2] || ca[3])) continue;
        const int32_t *fn = a.face + b * 6;
        const int4 bc = a.blocks[b];
        const int nx = a.gdims[bc.w * 4 + 0], ny = a.gdims[bc.w * 4 + 1], nz = a.gdims[bc.w * 4 + 2];
        const int gy = bc.y * B + y, gz = bc.z * B + z;
        const bool held_yz = ((a.held_mask & 4) && gy == 0) || ((a.held_mask & 8) && gy == ny - 1) ||
                             ((a.held_mask & 16) && gz == 0) || ((a.held_mask & 32) && gz == nz - 1);
        // without the residual only the +x values of rows on the inlet or outlet flux plane are read
        const int gx0 = bc.x * B + x0;
        const bool flux_row = nx >= 2 && (gx0 == 0 || (gx0 <= nx - 2 && nx - 2 <= gx0 + 3));
        // the Laplacian, built one axis and one side at a time: d_a = (0 + diff_-) + diff_+,
        // lap = sum_a d_a c_a; the x-face differences u - u_{x+1} of the inlet and outlet
        // planes go to the fluxes on the way
        DF lap[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) lap[i] = {0.f, 0.f};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            DF d[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) d[i] = {0.f, 0.f};
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const bool minus = side == 0;
                if (!RESID && (ax > 0 || minus || !flux_row)) continue;
                float vh[4], vl[4];
                bool va[4];
                if (ax == 0) {
                    // x: the row itself, shifted, and one value beyond it
                    float eh = 0.f, el = 0.f;
                    bool ea = false;
                    if (minus) {
                        if (x0 > 0) ea = load_df<VM>(a, s, b * B3 + lrow - 1, eh, el);
                        else if (fn[0] >= 0) ea = load_df<VM>(a, s, (int64_t)fn[0] * B3 + rowbase + (B - 1), eh, el);
                    } else {
                        if (x0 + 4 < B) ea = load_df<VM>(a, s, b * B3 + lrow + 4, eh, el);
                        else if (fn[1] >= 0) ea = load_df<VM>(a, s, (int64_t)fn[1] * B3 + rowbase, eh, el);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int k = minus ? i - 1 : i + 1;
                        const bool edge = minus ? i == 0 : i == 3;
                        vh[i] = edge ? eh : ch[k < 0 ? 0 : (k > 3 ? 3 : k)];
                        vl[i] = edge ? el : cl[k < 0 ? 0 : (k > 3 ? 3 : k)];
                        va[i] = edge ? ea : ca[k < 0 ? 0 : (k > 3 ? 3 : k)];
                    }
                } else {
                    const bool ydir = ax == 1;
                    const int coord = ydir ? y : z;
                    const int stride = ydir ? B : B * B;
                    int64_t nbk = b;
                    int lr = lrow + (minus ? -stride : stride);
                    if (minus ? coord == 0 : coord == B - 1) {
                        nbk = fn[ydir ? (minus ? 2 : 3) : (minus ? 4 : 5)];
                        lr = lrow + (minus ? (B - 1) * stride : -(B - 1) * stride);
                    }
                    if (nbk >= 0) {
                        load_row_df<VM>(a, s, nbk * B3 + lr, vh, vl, va);
                    } else {
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            vh[i] = 0.f;
                            vl[i] = 0.f;
                            va[i] = false;
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    if (ca[i] && va[i]) {
                        float e;
                        const float dh = tsum(vh[i], -ch[i], e);
                        const DF diff = {dh, VM != kVF32 ? __fadd_rn(e, __fsub_rn(vl[i], cl[i])) : e};
                        d[i] = df_add(d[i], diff);
                        const int gx = bc.x * B + x0 + i;
                        if (ax == 0 && !minus && nx >= 2 && (gx == 0 || gx == nx - 2) && isfinite(ch[i])) {
                            float e2;  // u - u_{x+1}
                            const float fh = tsum(ch[i], -vh[i], e2);
                            const DF f = {fh, VM != kVF32 ? __fadd_rn(e2, __fsub_rn(cl[i], vl[i])) : e2};
                            if (gx == 0) jin = df_add(jin, f);
                            if (gx == nx - 2) jout = df_add(jout, f);
                        }
                    }
                }
            }
            const DF cax = {a.ch[ax], a.cl[ax]};
#pragma unroll
            for (int i = 0; i < 4; ++i) lap[i] = df_add(lap[i], df_mul(d[i], cax));
        }
        // surface transfer: the row's weights and, for species B, the row of u_A
        float wv[4] = {0.f, 0.f, 0.f, 0.f}, uah[4] = {0.f, 0.f, 0.f, 0.f}, ual[4] = {0.f, 0.f, 0.f, 0.f};
        if (REACT && RESID) {
            const int ws = a.wslab[b];
            if (ws >= 0) {
                const float4 w4 = *reinterpret_cast<const float4 *>(a.wf + (int64_t)ws * B3 + lrow);
                wv[0] = w4.x;
                wv[1] = w4.y;
                wv[2] = w4.z;
                wv[3] = w4.w;
            }
            if (s == 1) {
                bool aa[4];
                load_row_df<VM>(a, 0, b * B3 + lrow, uah, ual, aa);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (!aa[i]) uah[i] = ual[i] = 0.f;
            }
        }
        const DF kk = {a.kh, a.kl};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (!ca[i]) continue;
            ++nact;
            const float h = ch[i], lo = cl[i];
            if (!isfinite(h)) {
                ++nonfin;
                continue;
            }
            const DF u = {h, lo};
            mass = df_add(mass, u);
            mn = fminf(mn, h);
            mx = fmaxf(mx, h);
            const int gx = bc.x * B + x0 + i;
            const bool held = held_yz || ((a.held_mask & 1) && gx == 0) || ((a.held_mask & 2) && gx == nx - 1);
            const int64_t slot = b * B3 + lrow + i;
            if (RESID && !held) {
                DF rate = dec;
                if (REACT && s == 0) rate = df_add(rate, df_mul(kk, {wv[i], 0.f}));
                DF r = df_mul(rate, u);
                r = df_add(lap[i], {-r.h, -r.l});
                if (REACT && s == 1) r = df_add(r, df_mul(df_mul(kk, {wv[i], 0.f}), {uah[i], ual[i]}));
                const float p = __fmul_rn(r.h, r.h);
                res = df_add(res, {p, __fmaf_rn(r.h, r.h, -p) + 2.f * r.h * r.l});
                if (VM == kVR && a.rout) a.rout[slot] = __fadd_rn(r.h, r.l);
            } else if (VM == kVR && a.rout) {
                a.rout[slot] = 0.f;
            }
        }
    }
    mass = df_shfl_add(mass);
    res = df_shfl_add(res);
    jin = df_shfl_add(jin);
    jout = df_shfl_add(jout);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        nact += __shfl_down_sync(0xffffffffu, nact, o);
        nonfin += __shfl_down_sync(0xffffffffu, nonfin, o);
    }
    __shared__ double sm[kRedThreads / 32][kNumRed];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        const double flux = a.D * a.inv_dx * a.area;
        sm[warp][SBG_RED_MASS] = df_to_d(mass) * a.dv;
        sm[warp][SBG_RED_JIN] = df_to_d(jin) * flux;
        sm[warp][SBG_RED_JOUT] = df_to_d(jout) * flux;
        sm[warp][SBG_RED_RESIDUAL] = RESID ? df_to_d(res) : (double)NAN;
        sm[warp][SBG_RED_MIN] = (double)mn;
        sm[warp][SBG_RED_MAX] = (double)mx;
        sm[warp][SBG_RED_NONFINITE] = (double)nonfin;
        sm[warp][SBG_RED_NACTIVE] = (double)nact;
    }
    __syncthreads();
    if (threadIdx.x < kNumRed) {
        const int q = threadIdx.x;
        double v = sm[0][q];
        for (int wi = 1; wi < kRedThreads / 32; ++wi)
            v = (q == SBG_RED_MIN) ? fmin(v, sm[wi][q]) : (q == SBG_RED_MAX) ? fmax(v, sm[wi][q]) : v + sm[wi][q];
        if (q == SBG_RED_RESIDUAL && a.no_residual) v = NAN;
        a.partials[(int64_t)blockIdx.x * kNumRed + q] = v;
    }
}

// coefficients as double-float pairs (host side)
static void split_df(double x, float &h, float &l) {
    h = (float)x;
    l = (float)(x - (double)h);
}
static void fill_df(RedArgs &a, const float *wf) {
    for (int ax = 0; ax < 3; ++ax) split_df(a.c[ax], a.ch[ax], a.cl[ax]);
    split_df(a.decay, a.dech, a.decl);
    split_df(a.k, a.kh, a.kl);
    a.wf = wf;
}

// SBG_F32R: b := b + d (double-float, renormalised), d := 0, in place over a slot range
__global__ void k_fold(float *__restrict__ d, float *__restrict__ bh, float *__restrict__ bl, int64_t begin,
                       int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t slot = begin + i;
    const float dv = d[slot];
    if (is_sent(dv) || dv == 0.f) return;
    float e;
    const float h = tsum(bh[slot], dv, e);
    const float l = __fadd_rn(e, bl[slot]);
    const float h2 = __fadd_rn(h, l);
    bh[slot] = h2;
    bl[slot] = __fsub_rn(l, __fsub_rn(h2, h));
    d[slot] = 0.f;
}

template <typename T, int VM, int B>
static void launch_reduce(const RedArgs &a, int nctas, cudaStream_t s) {
    if (sizeof(T) == 8) k_reduce<double, false, B><<<nctas, kRedThreads, 0, s>>>(a);
    else if (!a.epsf && a.no_residual) k_reduce_rows<VM, B, false, false><<<nctas, kRedThreads, 0, s>>>(a);
    else if (a.k == 0.0 && !a.epsf) k_reduce_rows<VM, B, false, true><<<nctas, kRedThreads, 0, s>>>(a);
    else if (!a.epsf) k_reduce_rows<VM, B, true, true><<<nctas, kRedThreads, 0, s>>>(a);
    else k_reduce_f<VM, B><<<nctas, kRedThreads, 0, s>>>(a);
}

// Arguments of a reduction of species `species` of buffer `buf` over one
// geometry (geom >= 0) or all blocks.
static void fill_red_args(sbg_grid g, sbg_state st, const sbg_params *p, int geom, int species, int buf,
                          double *partials, RedArgs &a) {
    std::memset(&a, 0, sizeof(a));
    for (int sp = 0; sp < st->ns; ++sp) {
        a.val[sp] = st->val[buf][sp];
        a.lo[sp] = st->lo[buf][sp];
    }
    a.bh = st->bh;
    a.bl = st->bl;
    a.blocks = g->blocks;
    a.face = g->face_nbr;
    a.wslab = g->wslab;
    a.w = g->w64;
    a.gdims = g->gdims;
    a.b_begin = geom < 0 ? 0 : g->geom_begin[geom];
    a.b_count = geom < 0 ? g->nb : g->geom_count[geom];
    a.species = species;
    a.ns = st->ns;
    for (int f = 0; f < 6; ++f)
        if (p->face_type[f] == SBG_FACE_DIRICHLET) a.held_mask |= 1 << f;
    for (int ax = 0; ax < 3; ++ax) a.c[ax] = p->D[species] / (p->dx[ax] * p->dx[ax]);
    a.D = p->D[species];
    a.decay = p->decay[species];
    a.k = p->k_surf;
    a.inv_dx = 1.0 / p->dx[0];
    a.area = p->dx[1] * p->dx[2];
    a.dv = p->dx[0] * p->dx[1] * p->dx[2];
    fill_df(a, g->w);
    a.partials = partials;
    if (g->has_eps && st->ns == 1) {
        if (st->dtype == SBG_F64) a.eps64 = g->eps64;
        else if (st->dtype == SBG_F32) a.epsf = g->eps;
    }
}

static void dispatch_reduce(sbg_grid g, sbg_state st, const RedArgs &a, int nctas, cudaStream_t s) {
    if (st->dtype == SBG_F64) {
        if (g->B == 8) launch_reduce<double, kVF32, 8>(a, nctas, s);
        else launch_reduce<double, kVF32, 4>(a, nctas, s);
    } else if (st->dtype == SBG_F32) {
        if (g->B == 8) launch_reduce<float, kVF32, 8>(a, nctas, s);
        else launch_reduce<float, kVF32, 4>(a, nctas, s);
    } else if (st->dtype == SBG_F32X2) {
        if (g->B == 8) launch_reduce<float, kVX2, 8>(a, nctas, s);
        else launch_reduce<float, kVX2, 4>(a, nctas, s);
    } else {
        if (g->B == 8) launch_reduce<float, kVR, 8>(a, nctas, s);
        else launch_reduce<float, kVR, 4>(a, nctas, s);
    }
}

static int reduce_ctas(const RedArgs &a, sbg_grid g) {
    const int64_t work = a.b_count * g->b3();
    const int nctas = (int)std::min<int64_t>(kRedMaxCtas, (work + kRedThreads - 1) / kRedThreads);
    return nctas < 1 ? 1 : nctas;
}

// SBG_F32R: the reduction pass of `a` (with a.rout set) has written r over
// its block range; fold d into b there.
static sbg_status fold_range(sbg_grid g, sbg_state st, const RedArgs &a, cudaStream_t s) {
    const int64_t n = a.b_count * g->b3();
    if (n > 0)
        k_fold<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((float *)st->val[st->cur][0], st->bh, st->bl,
                                                           a.b_begin * g->b3(), n);
    SBG_LAUNCH_CHECK("fold kernel launch");
    return SBG_OK;
}

sbg_status refresh_source(sbg_grid g, sbg_state st, const sbg_params *p, cudaStream_t s) {
    if (st->dtype != SBG_F32R) return SBG_OK;
    if (g->nb > 0) {
        RedArgs a;
        fill_red_args(g, st, p, -1, 0, st->cur, g->partials, a);
        a.rout = st->rsrc;
        dispatch_reduce(g, st, a, reduce_ctas(a, g), s);
        SBG_LAUNCH_CHECK("source refresh launch");
        sbg_status rc = fold_range(g, st, a, s);
        if (rc != SBG_OK) return rc;
    }
    st->r_valid = true;
    st->since_refresh = 0;
    return SBG_OK;
}

// Records of a per-geometry reduction (reduce_geometries): the number of CTA
// records the reduction of geometry `geom` writes.
int64_t reduce_records(sbg_grid g, sbg_state st, const sbg_params *p, int geom) {
    RedArgs a;
    fill_red_args(g, st, p, geom, 0, st->cur, nullptr, a);
    return reduce_ctas(a, g);
}

// One segmented reduction of species `species` (current buffer) over the
// geometries geoms[0..ngeoms): every geometry's CTAs write their records into
// their own segment of `records` (reduce_records(geom) each, in the order of
// geoms), one final kernel sums every segment (CTA i -> out_dev[i * kNumRed]),
// one copy brings all results to out_host and the stream is synchronised
// once.  The results equal reduce_species' per geometry bit for bit (the same
// kernels, records and summation order).  SBG_F32R states: also refreshes r
// and folds d over every reduced geometry, as reduce_species does.
sbg_status reduce_geometries(sbg_grid g, sbg_state st, const sbg_params *p, const int *geoms, int ngeoms,
                             int species, double *records, int *seg_dev, double *out_dev, double *out_host,
                             cudaStream_t s) {
    if (ngeoms <= 0) return SBG_OK;
    std::vector<int> seg(2 * (size_t)ngeoms);
    int64_t off = 0;
    const bool refresh = st->dtype == SBG_F32R;
    for (int i = 0; i < ngeoms; ++i) {
        RedArgs a;
        fill_red_args(g, st, p, geoms[i], species, st->cur, records + off * kNumRed, a);
        if (refresh) a.rout = st->rsrc;
        const int nctas = reduce_ctas(a, g);
        dispatch_reduce(g, st, a, nctas, s);
        SBG_LAUNCH_CHECK("segmented reduction launch");
        if (refresh) {
            sbg_status rc = fold_range(g, st, a, s);
            if (rc != SBG_OK) return rc;
        }
        seg[2 * i] = (int)off;
        seg[2 * i + 1] = nctas;
        off += nctas;
    }
    SBG_CUDA(cudaMemcpyAsync(seg_dev, seg.data(), sizeof(int) * seg.size(), cudaMemcpyHostToDevice, s));
    k_reduce_final_seg<<<ngeoms, 256, 0, s>>>(records, seg_dev, out_dev);
    SBG_LAUNCH_CHECK("segmented reduction final pass");
    SBG_CUDA(cudaMemcpyAsync(out_host, out_dev, sizeof(double) * kNumRed * ngeoms, cudaMemcpyDeviceToHost, s));
    SBG_CUDA(cudaStreamSynchronize(s));
    return check_device_error(g, s);
}

// Enqueues the reduction of species `species` of buffer `which` (st->cur when
// < 0) into g->red_dev[kNumRed] (kernel launches only).  SBG_F32R states: also
// refreshes r and folds d over the reduced range.
static sbg_status enqueue_reduce(sbg_grid g, sbg_state st, const sbg_params *p, int geom, int species, int which,
                                 cudaStream_t s, bool residual = true) {
    const int buf = which < 0 ? st->cur : which;
    RedArgs a;
    fill_red_args(g, st, p, geom, species, buf, g->partials, a);
    a.no_residual = residual ? 0 : 1;
    // (without the residual there is no source r to refresh)
    const bool refresh = st->dtype == SBG_F32R && buf == st->cur && residual;
    if (refresh) a.rout = st->rsrc;
    const int nctas = reduce_ctas(a, g);
    dispatch_reduce(g, st, a, nctas, s);
    k_reduce_final<<<1, 256, 0, s>>>(g->partials, nctas, g->red_dev);
    SBG_LAUNCH_CHECK("reduction launch");
    if (refresh) {
        sbg_status rc = fold_range(g, st, a, s);
        if (rc != SBG_OK) return rc;
        if (geom < 0 || g->n_geoms == 1) {
            st->r_valid = true;
            st->since_refresh = 0;
        }
    }
    return SBG_OK;
}

// Reduces species `species` of buffer `which` (st->cur when < 0) into
// out_host[kNumRed] and synchronises.
sbg_status reduce_species(sbg_grid g, sbg_state st, const sbg_params *p, int geom, int species,
                          int which, double *out_host, cudaStream_t s) {
    sbg_status rc = enqueue_reduce(g, st, p, geom, species, which, s);
    if (rc != SBG_OK) return rc;
    SBG_CUDA(cudaMemcpyAsync(g->red_host, g->red_dev, sizeof(double) * kNumRed, cudaMemcpyDeviceToHost, s));
    SBG_CUDA(cudaStreamSynchronize(s));
    std::memcpy(out_host, g->red_host, sizeof(double) * kNumRed);
    return check_device_error(g, s);
}

sbg_status check_device_error(sbg_grid g, cudaStream_t s) {
    SBG_CUDA(cudaMemcpyAsync(g->err_host, g->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    SBG_CUDA(cudaStreamSynchronize(s));
    if (*g->err_host != 0) {
        const int code = *g->err_host;
        SBG_CUDA(cudaMemsetAsync(g->err, 0, sizeof(int), s));
        SBG_CUDA(cudaStreamSynchronize(s));
        return fail((sbg_status)code, "a step kernel gave up a bounded wait (device error word set)");
    }
    return SBG_OK;
}

static sbg_status check_common(sbg_grid g, sbg_state st, const sbg_params *p, int geom) {
    if (!g || !st || !p) return fail(SBG_ERR_INVALID_ARG, "null pointer");
    if (st->grid != g) return fail(SBG_ERR_INVALID_ARG, "state of another grid");
    if (geom < -1 || geom >= g->n_geoms) return fail(SBG_ERR_INVALID_ARG, "bad geometry index");
    if (p->nspecies != st->ns) return fail(SBG_ERR_INVALID_ARG, "params.nspecies differs from the state's");
    for (int a = 0; a < 3; ++a)
        if (!(p->dx[a] > 0.0)) return fail(SBG_ERR_INVALID_ARG, "dx must be > 0");
    return SBG_OK;
}

// ---------------------------------------------------------------------------
// Sum of u over the active voxels of a box of one geometry (the bleached
// region of a simulated FRAP experiment, Sec. 3.3): double-float per thread
// and warp for FP32-based states, FP64 for FP64 states; per-CTA records in the
// grid's scratch, one fixed-order final pass.
template <typename T, int VM, int B>
__global__ void __launch_bounds__(kRedThreads) k_box_sum(const RedArgs a, int4 lo, int4 hi) {
    constexpr int B3 = B * B * B;
    DF m = {0.f, 0.f};
    double md = 0.0;
    int cnt = 0;
    const int64_t total = a.b_count * B3;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = a.b_begin + t / B3;
        const int l = (int)(t % B3);
        const int4 bc = a.blocks[b];
        const int x = bc.x * B + l % B, y = bc.y * B + (l / B) % B, z = bc.z * B + l / (B * B);
        if (x < lo.x || y < lo.y || z < lo.z || x >= hi.x || y >= hi.y || z >= hi.z) continue;
        const int64_t slot = b * B3 + l;
        if (sizeof(T) == 8) {
            const double v = ((const double *)a.val[a.species])[slot];
            if (is_sent(v)) continue;
            md += v;
        } else {
            float h, lw;
            if (!load_df<VM>(a, a.species, slot, h, lw)) continue;
            m = df_add(m, {h, lw});
        }
        ++cnt;
    }
    __shared__ double sm[kRedThreads / 32][2];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double v = sizeof(T) == 8 ? warp_sum(md) : df_to_d(df_shfl_add(m));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if (lane == 0) {
        sm[warp][0] = v;
        sm[warp][1] = (double)cnt;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double acc = 0.0;
        for (int w = 0; w < kRedThreads / 32; ++w) acc += sm[w][threadIdx.x];
        a.partials[(int64_t)blockIdx.x * 2 + threadIdx.x] = acc;
    }
}

// 256 threads: strided partial sums, then a fixed tree (deterministic for a
// given CTA count)
__global__ void __launch_bounds__(256) k_box_final(const double *partials, int nctas, double *out) {
    __shared__ double sm[2][256];
    double a0 = 0.0, a1 = 0.0;
    for (int c = threadIdx.x; c < nctas; c += 256) {
        a0 += partials[(int64_t)c * 2];
        a1 += partials[(int64_t)c * 2 + 1];
    }
    sm[0][threadIdx.x] = a0;
    sm[1][threadIdx.x] = a1;
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride) {
            sm[0][threadIdx.x] += sm[0][threadIdx.x + stride];
            sm[1][threadIdx.x] += sm[1][threadIdx.x + stride];
        }
        __syncthreads();
    }
    if (threadIdx.x < 2) out[threadIdx.x] = sm[threadIdx.x][0];
}

sbg_status launch_box_sum(sbg_grid g, sbg_state st, int geom, int species, const int64_t lo[3], const int64_t hi[3],
                          double *dst, cudaStream_t s) {
    RedArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int sp = 0; sp < st->ns; ++sp) {
        a.val[sp] = st->val[st->cur][sp];
        a.lo[sp] = st->lo[st->cur][sp];
    }
    a.bh = st->bh;
    a.bl = st->bl;
    a.blocks = g->blocks;
    a.b_begin = g->geom_begin[geom];
    a.b_count = g->geom_count[geom];
    a.species = species;
    a.partials = g->partials;
    auto clampi = [](int64_t v) { return (int)(v < -1 ? -1 : v > ((int64_t)1 << 30) ? ((int64_t)1 << 30) : v); };
    const int4 l4 = make_int4(clampi(lo[0]), clampi(lo[1]), clampi(lo[2]), 0);
    const int4 h4 = make_int4(clampi(hi[0]), clampi(hi[1]), clampi(hi[2]), 0);
    const int64_t work = a.b_count * g->b3();
    int nctas = (int)std::min<int64_t>(kRedMaxCtas, (work + kRedThreads - 1) / kRedThreads);
    if (nctas < 1) nctas = 1;
#define BOX_LAUNCH(T, VM)                                                                   \
    do {                                                                                    \
        if (g->B == 8) k_box_sum<T, VM, 8><<<nctas, kRedThreads, 0, s>>>(a, l4, h4);          \
        else k_box_sum<T, VM, 4><<<nctas, kRedThreads, 0, s>>>(a, l4, h4);                   \
    } while (0)
    if (st->dtype == SBG_F64) BOX_LAUNCH(double, kVF32);
    else if (st->dtype == SBG_F32) BOX_LAUNCH(float, kVF32);
    else if (st->dtype == SBG_F32X2) BOX_LAUNCH(float, kVX2);
    else BOX_LAUNCH(float, kVR);
#undef BOX_LAUNCH
    k_box_final<<<1, 256, 0, s>>>(g->partials, nctas, dst);
    SBG_LAUNCH_CHECK("box sum launch");
    return SBG_OK;
}

sbg_status check_box_args(sbg_grid g, sbg_state st, int geom, int species, const char *who) {
    if (!g || !st) return fail(SBG_ERR_INVALID_ARG, std::string(who) + ": null pointer");
    if (st->grid != g) return fail(SBG_ERR_INVALID_ARG, std::string(who) + ": state of another grid");
    if (geom < 0 || geom >= g->n_geoms) return fail(SBG_ERR_INVALID_ARG, std::string(who) + ": bad geometry");
    if (species < 0 || species >= st->ns) return fail(SBG_ERR_INVALID_ARG, std::string(who) + ": bad species");
    return SBG_OK;
}

}  // namespace sbg

using namespace sbg;

extern "C" sbg_status sbg_reduce_box(sbg_grid g, sbg_state st, int32_t geom, int32_t species, const int64_t lo[3],
                                     const int64_t hi[3], double *out, void *stream) {
    TraceRange trace_range("sbg_reduce_box");
    sbg_status rc = check_box_args(g, st, geom, species, "sbg_reduce_box");
    if (rc != SBG_OK) return rc;
    if (!lo || !hi || !out) return fail(SBG_ERR_INVALID_ARG, "sbg_reduce_box: null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    rc = launch_box_sum(g, st, geom, species, lo, hi, g->red_dev, s);
    if (rc != SBG_OK) return rc;
    SBG_CUDA(cudaMemcpyAsync(g->red_host, g->red_dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    SBG_CUDA(cudaStreamSynchronize(s));
    out[0] = g->red_host[0];
    out[1] = g->red_host[1];
    return SBG_OK;
}

extern "C" sbg_status sbg_reduce(sbg_grid g, sbg_state st, const sbg_params *p, int32_t geom,
                                 double *out, void *stream) {
    TraceRange trace_range("sbg_reduce");
    sbg_status rc = check_common(g, st, p, geom);
    if (rc != SBG_OK) return rc;
    if (!out) return fail(SBG_ERR_INVALID_ARG, "sbg_reduce: null output");
    for (int s = 0; s < st->ns; ++s) {
        rc = reduce_species(g, st, p, geom, s, -1, out + s * kNumRed, (cudaStream_t)stream);
        if (rc != SBG_OK) return rc;
    }
    return SBG_OK;
}

extern "C" sbg_status sbg_reduce_async(sbg_grid g, sbg_state st, const sbg_params *p, int32_t geom,
                                       double *out, void *stream) {
    TraceRange trace_range("sbg_reduce_async");
    sbg_status rc = check_common(g, st, p, geom);
    if (rc != SBG_OK) return rc;
    if (!out) return fail(SBG_ERR_INVALID_ARG, "sbg_reduce_async: null output");
    cudaStream_t s = (cudaStream_t)stream;
    for (int sp = 0; sp < st->ns; ++sp) {
        rc = enqueue_reduce(g, st, p, geom, sp, -1, s);
        if (rc != SBG_OK) return rc;
        // stream order keeps the next species' final pass off g->red_dev until this copy is done
        SBG_CUDA(cudaMemcpyAsync(out + sp * kNumRed, g->red_dev, sizeof(double) * kNumRed, cudaMemcpyDefault, s));
    }
    return SBG_OK;
}

extern "C" sbg_status sbg_check_async(sbg_grid g, sbg_state st, const sbg_params *p, int32_t geom, double *out,
                                      void *stream) {
    TraceRange trace_range("sbg_check_async");
    sbg_status rc = check_common(g, st, p, geom);
    if (rc != SBG_OK) return rc;
    if (!out) return fail(SBG_ERR_INVALID_ARG, "sbg_check_async: null output");
    cudaStream_t s = (cudaStream_t)stream;
    for (int sp = 0; sp < st->ns; ++sp) {
        rc = enqueue_reduce(g, st, p, geom, sp, -1, s, false);
        if (rc != SBG_OK) return rc;
        SBG_CUDA(cudaMemcpyAsync(out + sp * kNumRed, g->red_dev, sizeof(double) * kNumRed, cudaMemcpyDefault, s));
    }
    return SBG_OK;
}

extern "C" sbg_status sbg_effective_D(sbg_grid g, sbg_state st, const sbg_params *p, int32_t geom,
                                      double *D_eff, double *tau, double *psi, void *stream) {
    TraceRange trace_range("sbg_effective_D");
    sbg_status rc = check_common(g, st, p, geom);
    if (rc != SBG_OK) return rc;
    if (geom < 0) return fail(SBG_ERR_INVALID_ARG, "sbg_effective_D: needs one geometry");
    if (!D_eff || !tau || !psi) return fail(SBG_ERR_INVALID_ARG, "sbg_effective_D: null output");
    double r[kNumRed];
    rc = reduce_species(g, st, p, geom, 0, -1, r, (cudaStream_t)stream);
    if (rc != SBG_OK) return rc;
    const int64_t *d = &g->dims[3 * geom];
    const double L = (double)(d[0] - 1) * p->dx[0];
    const double A = (double)d[1] * p->dx[1] * (double)d[2] * p->dx[2];
    const double dC = fabs(p->face_value[0] - p->face_value[1]);
    const double J = 0.5 * (r[SBG_RED_JIN] + r[SBG_RED_JOUT]);
    *psi = r[SBG_RED_NACTIVE] / ((double)d[0] * (double)d[1] * (double)d[2]);
    *D_eff = (dC > 0.0) ? J * L / (dC * A) : NAN;
    *tau = (*D_eff > 0.0) ? (*psi) * p->D[0] / (*D_eff) : INFINITY;
    return SBG_OK;
}

extern "C" sbg_status sbg_run_to_steady(sbg_grid g, sbg_state st, const sbg_params *p, double tol,
                                        int64_t check_every, int64_t max_steps, int64_t *steps_done,
                                        double *rel_residual, void *stream) {
    TraceRange trace_range("sbg_run_to_steady");
    sbg_status rc = check_common(g, st, p, -1);
    if (rc != SBG_OK) return rc;
    if (check_every < 1 || max_steps < 0 || !(tol > 0.0))
        return fail(SBG_ERR_INVALID_ARG, "sbg_run_to_steady: check_every >= 1, max_steps >= 0, tol > 0");
    rc = validate_params(g, p, st->ns);
    if (rc != SBG_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    double r[kNumRed];
    rc = reduce_species(g, st, p, -1, 0, -1, r, s);
    if (rc != SBG_OK) return rc;
    const double r0 = r[SBG_RED_RESIDUAL];
    int64_t done = 0;
    double rel = r0 > 0.0 ? 1.0 : 0.0;
    if (steps_done) *steps_done = 0;
    if (rel_residual) *rel_residual = rel;
    if (r[SBG_RED_NONFINITE] > 0) return fail(SBG_ERR_NONFINITE, "sbg_run_to_steady: non-finite initial state");
    while (rel >= tol && done < max_steps) {
        const int64_t n = std::min<int64_t>(check_every, max_steps - done);
        rc = step_n(g, st, p, n, s);
        if (rc != SBG_OK) return rc;
        done += n;
        rc = reduce_species(g, st, p, -1, 0, -1, r, s);
        if (rc != SBG_OK) return rc;
        rel = r[SBG_RED_RESIDUAL] / r0;
        if (steps_done) *steps_done = done;
        if (rel_residual) *rel_residual = rel;
        if (r[SBG_RED_NONFINITE] > 0) return fail(SBG_ERR_NONFINITE, "sbg_run_to_steady: non-finite value");
    }
    if (rel >= tol) return fail(SBG_ERR_NOT_CONVERGED, "sbg_run_to_steady: max_steps reached");
    return SBG_OK;
}

// ---------------------------------------------------------------------------
// Reduction without any allocation.
//
// Some callers cannot call cudaMalloc: a serving process whose device memory
// is owned and budgeted by another allocator (a framework's caching
// allocator or a fixed arena), or a hot loop where an allocation's latency
// or its implicit synchronisation is not acceptable.  sbg_reduce_noalloc runs
// the same FP64 reduction kernels as sbg_reduce, but its per-CTA partial
// records live in the fixed array below instead of a buffer owned by the
// grid, and its result goes to a device buffer the caller owns.
//
// The array is `kNoAllocRecords` records of SBG_NRED doubles (256 KiB); every
// GPU that loads this library keeps it until the process exits.  One record
// covers up to `kNoAllocSlotsPerCta` voxel slots, so one call reduces at most
// kNoAllocRecords * kNoAllocSlotsPerCta = 2^28 voxel slots (blocks x B^3);
// larger ranges are rejected.  Each call's first kernel overwrites every
// record it uses before the second kernel reads it, so nothing needs
// clearing between calls; but all calls share the array, so two calls whose
// kernels overlap on the GPU (different streams, no ordering) race.
namespace sbg {

constexpr int kNoAllocRecords = 4096;
constexpr int64_t kNoAllocSlotsPerCta = 65536;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocRecords * kNumRed];

// Device address of g_noalloc_partials on the current device.  In host code
// the symbol is only a host-side stand-in; the kernels need the address that
// cudaGetSymbolAddress returns.  It is looked up on every call (a host-side
// lookup, no allocation) rather than cached, so that a device reset or a
// re-created context, which reloads the module at another address, never
// leaves a stale pointer behind, and concurrent first calls from several host
// threads share no mutable table.  The first lookup on a device loads the
// library's device code there.
static sbg_status noalloc_scratch(double **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress (no-allocation reduction scratch)");
    *out = (double *)p;
    return SBG_OK;
}

}  // namespace sbg

extern "C" sbg_status sbg_reduce_noalloc(sbg_grid g, sbg_state st, const sbg_params *p, int32_t geom,
                                         int32_t species, double *out_dev, void *stream) {
    TraceRange trace_range("sbg_reduce_noalloc");
    sbg_status rc = check_common(g, st, p, geom);
    if (rc != SBG_OK) return rc;
    if (!out_dev) return fail(SBG_ERR_INVALID_ARG, "sbg_reduce_noalloc: null output");
    if (species < 0 || species >= st->ns) return fail(SBG_ERR_INVALID_ARG, "sbg_reduce_noalloc: bad species");
    const int64_t b_begin = geom < 0 ? 0 : g->geom_begin[geom];
    const int64_t b_count = geom < 0 ? g->nb : g->geom_count[geom];
    const int64_t work = b_count * g->b3();
    if (work > (int64_t)kNoAllocRecords * kNoAllocSlotsPerCta)
        return fail(SBG_ERR_INVALID_ARG,
                    "sbg_reduce_noalloc: " + std::to_string(work) + " voxel slots exceed the limit of " +
                        std::to_string((int64_t)kNoAllocRecords * kNoAllocSlotsPerCta) +
                        " (use sbg_reduce for larger grids)");
    double *scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc != SBG_OK) return rc;

    RedArgs a;
    fill_red_args(g, st, p, geom, species, st->cur, scratch, a);  // a.rout stays null: read-only
    int nctas = (int)((work + kNoAllocSlotsPerCta - 1) / kNoAllocSlotsPerCta);
    if (nctas < 1) nctas = 1;
    cudaStream_t s = (cudaStream_t)stream;
    dispatch_reduce(g, st, a, nctas, s);
    k_reduce_final<<<1, 256, 0, s>>>(scratch, nctas, out_dev);
    SBG_LAUNCH_CHECK("no-allocation reduction launch");
    return SBG_OK;
}
