// One x-row of four voxels with its neighbour values, and the adjoint of the
// step on one species for such a row (shared by the ring and streaming
// kernels, which must give bitwise the same lambda).
#pragma once
#include "sbg_step.cuh"

namespace sbg {

__device__ __forceinline__ float rv4(const float4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

struct RowVals {
    float4 u;
    float xm, xp;
    float4 ym, yp, zm, zp;
};

// x differences along a row (R = xm, the four values, xp: Dx[j] = R[j+1] - R[j]).
__device__ __forceinline__ void row_dx(const RowVals &v, float Dx[5]) {
    const float R[6] = {v.xm, v.u.x, v.u.y, v.u.z, v.u.w, v.xp};
#pragma unroll
    for (int jj = 0; jj < 5; ++jj) Dx[jj] = __fsub_rn(R[jj + 1], R[jj]);
}

// Adjoint of one species (lambda^{n+1}: v0, u^n: v1): lambda^n = M^T lambda^{n+1}
// on free voxels, 0 on held ones; adds this row's terms of dL/dD (lambda dt
// g(u^n)) to qd and of dL/dk (dt w u (0 - lambda)) to qk, voxel by voxel in x
// order, as the one-row kernel does.
template <bool REACT>
__device__ __forceinline__ float4 row_adjoint1(const RowVals &v0, const RowVals &v1, const float4 w4, uint32_t hb,
                                               const StepCoef<float> &kc, float i0, float i1, float i2, float &qd,
                                               float &qk) {
    bool actx[6];
    actx[0] = !is_sent(v0.xm);
    actx[5] = !is_sent(v0.xp);
#pragma unroll
    for (int i = 0; i < 4; ++i) actx[i + 1] = !is_sent(rv4(v0.u, i));
    float D0[5], D1[5];
    row_dx(v0, D0);
    row_dx(v1, D1);
    float res[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float c = rv4(v0.u, i), u = rv4(v1.u, i);
        const float y0[4] = {rv4(v0.ym, i), rv4(v0.yp, i), rv4(v0.zm, i), rv4(v0.zp, i)};
        const float y1[4] = {rv4(v1.ym, i), rv4(v1.yp, i), rv4(v1.zm, i), rv4(v1.zp, i)};
        float n0[4], n1[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const bool out = is_sent(y0[f]);
            n0[f] = out ? c : y0[f];
            n1[f] = out ? u : y1[f];
        }
        const float dxs0 = __fsub_rn(actx[i + 2] ? D0[i + 1] : 0.f, actx[i] ? D0[i] : 0.f);
        const float dp1 = actx[i + 2] ? D1[i + 1] : 0.f, dm1 = actx[i] ? D1[i] : 0.f;
        const float kw = REACT ? __fmul_rn(kc.k, rv4(w4, i)) : 0.f;
        const float rate = REACT ? __fadd_rn(kc.decay[0], kw) : kc.decay[0];
        const float nr = fused_update_dx(c, dxs0, n0[0], n0[1], n0[2], n0[3], kc.c[0], kc.dt, rate, 0.f);
        float g = __fmul_rn(i0, __fadd_rn(-dm1, dp1));
        g = __fmaf_rn(i1, __fadd_rn(__fsub_rn(n1[0], u), __fsub_rn(n1[1], u)), g);
        g = __fmaf_rn(i2, __fadd_rn(__fsub_rn(n1[2], u), __fsub_rn(n1[3], u)), g);
        const float term = __fmul_rn(__fmul_rn(c, kc.dt), g);
        const bool act = actx[i + 1];
        const bool upd = act && !((hb >> i) & 1u);
        qd = __fadd_rn(qd, upd ? term : 0.f);
        if (REACT) {
            const float tk = __fmul_rn(__fmul_rn(__fmul_rn(kc.dt, rv4(w4, i)), u), __fsub_rn(0.f, c));
            qk = __fadd_rn(qk, upd ? tk : 0.f);
        }
        res[i] = upd ? nr : (act ? 0.f : c);
    }
    return make_float4(res[0], res[1], res[2], res[3]);
}


}  // namespace sbg
