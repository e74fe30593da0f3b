// Per-row arithmetic of the streaming step kernels (sbg_step_stream.cu,
// sbg_step_wave.cu): packed FP32 pairs, the sentinel masks and the update
// of one x-row of four voxels (Eq. 1 with the no-flux rule of Sec. 2.3 and
// the surface sink of Sec. 3.5).
#pragma once
#include "sbg_step.cuh"

namespace sbg {


// SBG_DEBUG (the libsbg_debug.so build): every face id and band-row index is
// checked against its table before it is used; an index outside records
// SBG_ERR_BOUNDS in the grid's error word and reads the ghost block (or no
// weights) instead
#ifndef SBG_DEBUG
#define SBG_DEBUG 0
#endif

__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

// Asks L2 for the line holding p (a hint: no register, no wait).  The streaming
// kernels issue it for the rows their next group will read, one sweep ahead.
__device__ __forceinline__ void prefetch_l2(const float *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ float f4at(const float4 &v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// Packed FP32 pairs (one 64-bit register pair, two lanes): the .f32x2
// arithmetic of sm_100 and later, each lane rounded exactly as the scalar
// instruction of the same name, so a pair (A, B) of species values is updated
// with half the instructions and bitwise the same results.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f32x2 r, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Mask of a stored value: all ones where it is the sentinel (outside Omega),
// else 0; and the select (v where the mask is 0, c where it is all ones) as
// one logical operation on the bits.
__device__ __forceinline__ uint32_t sent_mask(float v) { return __float_as_uint(v) == kSent32 ? ~0u : 0u; }
__device__ __forceinline__ float pick(float v, float c, uint32_t m) {
    return __uint_as_float((__float_as_uint(v) & ~m) | (__float_as_uint(c) & m));
}
__device__ __forceinline__ float zero_if(float v, uint32_t m) { return __uint_as_float(__float_as_uint(v) & ~m); }
__device__ __forceinline__ f32x2 zero_if2(f32x2 v, uint32_t m0, uint32_t m1) {
    float a, b;
    upk(v, a, b);
    return pk(zero_if(a, m0), zero_if(b, m1));
}

// Update of one row of four voxels of one species (the plain kernel's
// expression, voxel by voxel, with the rounding of every operation pinned):
//   u' = u + dt ( c_x dxx + c_y dyy + c_z dzz - decay u + t ),
//   dxx = (u~_{x+1} - u) - (u - u~_{x-1}), likewise along y and z,
// where a neighbour outside Omega (sentinel) reads as the centre value, i.e.
// its one-sided difference is +0.  The x differences between voxels of the
// row are formed once and shared; the y and z terms, the Laplacian and the
// update run on packed voxel pairs (0,1) and (2,3).  keep: mask of voxels
// that keep their value (outside Omega or held).
__device__ __forceinline__ float4 row_update(const float4 c, float xm, float xp, const float4 ym, const float4 yp,
                                             const float4 zm, const float4 zp, const float cc[3], float dt,
                                             float decay, f32x2 t01, f32x2 t23, const uint32_t keep[4]) {
    const float u[4] = {c.x, c.y, c.z, c.w};
    uint32_t mc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) mc[i] = sent_mask(u[i]);
    // one-sided x differences d[i] = u_i - u_{i-1} (i = 0..4 with u_{-1} = xm, u_4 = xp), +0 where
    // either end lies outside Omega (an inactive centre's result is discarded anyway)
    float d[5];
    d[0] = zero_if(__fsub_rn(u[0], xm), sent_mask(xm));
#pragma unroll
    for (int i = 1; i < 4; ++i) d[i] = zero_if(__fsub_rn(u[i], u[i - 1]), mc[i - 1] | mc[i]);
    d[4] = zero_if(__fsub_rn(xp, u[3]), sent_mask(xp));
    float dxx[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) dxx[i] = __fsub_rn(d[i + 1], d[i]);
    const float ya[4] = {ym.x, ym.y, ym.z, ym.w}, yb[4] = {yp.x, yp.y, yp.z, yp.w};
    const float za[4] = {zm.x, zm.y, zm.z, zm.w}, zb[4] = {zp.x, zp.y, zp.z, zp.w};
    const f32x2 cx = pk(cc[0], cc[0]), cy = pk(cc[1], cc[1]), cz = pk(cc[2], cc[2]);
    const f32x2 dt2 = pk(dt, dt), nd = pk(-decay, -decay);
    float r[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i0 = 2 * h, i1 = 2 * h + 1;
        const f32x2 uu = pk(u[i0], u[i1]);
        const f32x2 dyp = zero_if2(sub2(pk(yb[i0], yb[i1]), uu), sent_mask(yb[i0]), sent_mask(yb[i1]));
        const f32x2 dym = zero_if2(sub2(uu, pk(ya[i0], ya[i1])), sent_mask(ya[i0]), sent_mask(ya[i1]));
        const f32x2 dzp = zero_if2(sub2(pk(zb[i0], zb[i1]), uu), sent_mask(zb[i0]), sent_mask(zb[i1]));
        const f32x2 dzm = zero_if2(sub2(uu, pk(za[i0], za[i1])), sent_mask(za[i0]), sent_mask(za[i1]));
        const f32x2 lap = fma2(cz, sub2(dzp, dzm), fma2(cy, sub2(dyp, dym), mul2(cx, pk(dxx[i0], dxx[i1]))));
        const f32x2 react = fma2(nd, uu, h == 0 ? t01 : t23);
        const f32x2 v = fma2(dt2, add2(lap, react), uu);
        float v0, v1;
        upk(v, v0, v1);
        r[i0] = pick(v0, u[i0], keep[i0] | mc[i0]);
        r[i1] = pick(v1, u[i1], keep[i1] | mc[i1]);
    }
    return make_float4(r[0], r[1], r[2], r[3]);
}

}  // namespace sbg
