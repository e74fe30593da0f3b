// Sussman redistancing on the device (Sec. 2.1: the signed-distance level set
// as the steady state of d phi / d alpha = sigma(phi) (1 - |grad phi|) with
// the smoothed sign sigma = phi / sqrt(phi^2 + |grad phi|^2 h^2), first-order
// upwind differences).  The paper runs it on a dense grid on the host cores
// and names a GPU version as future work; here the dense field lives in HBM
// (4 or 8 B per voxel, 288 GB on the device) and each iteration is one
// streaming stencil pass, so the sparse block grid is then built from the
// result on the device.
//
// Scheme (per voxel, Jacobi in alpha; a neighbour beyond the box takes the
// voxel's own value):
//   D-_a = (phi_i - phi_{i-a}) / dx_a,  D+_a = (phi_{i+a} - phi_i) / dx_a,
//   phi > 0: G^2 = sum_a max(max(D-_a, 0)^2, min(D+_a, 0)^2),
//   phi < 0: G^2 = sum_a max(min(D-_a, 0)^2, max(D+_a, 0)^2),
//   phi' = phi + dalpha sigma (1 - G),  h = min(dx),  dalpha = cfl h;
// phi = 0 stays 0.  With dalpha <= h a voxel never changes sign (the decrease
// is below dalpha phi / h), so the pore set of the input is kept exactly.
#include <math.h>

#include <cstring>
#include <string>

#include "sbg_internal.cuh"

namespace sbg {

constexpr int kRdX = 32, kRdY = 8, kRdZ = 16;  // threads in x, y; planes per thread

template <typename T>
struct RedistArgs {
    const T *in;
    T *out;
    int64_t nx, ny, nz;
    T inv_dx[3];
    T h2;
    T dalpha;
    T band;                 // |phi| below this enters the residual
    unsigned int *res;      // max |sigma (1 - G)| as FP32 bits (null: not tracked)
};

// One axis of G^2: with s = sign(phi) the two one-sided upwind terms reduce to
// (max(|phi| - min(s phi_-, s phi_+), 0) / dx_a)^2 (for phi > 0 the larger of
// max(D-, 0)^2 and min(D+, 0)^2, for phi < 0 of min(D-, 0)^2 and max(D+, 0)^2;
// s v is exact, so are the differences' magnitudes).
template <typename T>
__device__ __forceinline__ T upwind_sq(T cs, T s, T vm, T vp, T inv) {
    const T t = fmax(cs - fmin(s * vm, s * vp), T(0)) * inv;
    return t * t;
}

// phi / sqrt(phi^2 + G^2 h^2) and G = sqrt(G^2): FP32 takes the hardware
// reciprocal square root (a few ulp), FP64 the correctly rounded operations
__device__ __forceinline__ float smoothed_sign(float c, float d) { return c * rsqrtf(d); }
__device__ __forceinline__ double smoothed_sign(double c, double d) { return c / sqrt(d); }
__device__ __forceinline__ float root(float g2) { return g2 > 0.f ? g2 * rsqrtf(g2) : 0.f; }
__device__ __forceinline__ double root(double g2) { return sqrt(g2); }

// One thread per (x, y) column of kRdZ planes; the z neighbours ride in
// registers, the x and y neighbours come through L1.
template <typename T>
__global__ void __launch_bounds__(kRdX * kRdY) k_sussman(const RedistArgs<T> a) {
    const int64_t x = (int64_t)blockIdx.x * kRdX + threadIdx.x;
    const int64_t y = (int64_t)blockIdx.y * kRdY + threadIdx.y;
    const int64_t z0 = (int64_t)blockIdx.z * kRdZ;
    float rmax = 0.f;
    if (x < a.nx && y < a.ny && z0 < a.nz) {
        const int64_t plane = a.nx * a.ny;
        const int xm = x > 0 ? -1 : 0, xp = x < a.nx - 1 ? 1 : 0;
        const int ym = y > 0 ? -(int)a.nx : 0, yp = y < a.ny - 1 ? (int)a.nx : 0;
        const T *p = a.in + z0 * plane + y * a.nx + x;
        T *q = a.out + z0 * plane + y * a.nx + x;
        T below = z0 > 0 ? p[-plane] : p[0];
        T c = p[0];
        const int nzl = (int)(a.nz - z0 < kRdZ ? a.nz - z0 : kRdZ);
        const bool last_chunk = z0 + nzl == a.nz;
        const bool track = a.res != nullptr;
        for (int k = 0; k < nzl; ++k, p += plane, q += plane) {
            const T above = (k + 1 < nzl || !last_chunk) ? p[plane] : c;
            T res = c;
            if (c != T(0)) {
                const T sg = c > T(0) ? T(1) : T(-1);
                const T cs = fabs(c);
                T g2 = upwind_sq(cs, sg, p[xm], p[xp], a.inv_dx[0]);
                g2 += upwind_sq(cs, sg, p[ym], p[yp], a.inv_dx[1]);
                g2 += upwind_sq(cs, sg, below, above, a.inv_dx[2]);
                const T g = root(g2);
                const T sigma = smoothed_sign(c, c * c + g2 * a.h2);
                const T rate = sigma * (T(1) - g);
                res = c + a.dalpha * rate;
                if (track && cs < a.band) rmax = fmaxf(rmax, (float)fabs(rate));
            }
            *q = res;
            below = c;
            c = above;
        }
    }
    if (a.res) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        if ((threadIdx.x & 31) == 0 && rmax > 0.f) atomicMax(a.res, __float_as_uint(rmax));
    }
}

template <typename T>
static sbg_status redistance_t(const int64_t dims[3], const double dx[3], const void *in, void *out, int on_device,
                               const sbg_redist_opts *o, int64_t *iters_out, double *res_out, cudaStream_t s) {
    const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
    const int64_t n = nx * ny * nz;
    const size_t bytes = sizeof(T) * (size_t)n;
    double h = dx[0] < dx[1] ? dx[0] : dx[1];
    h = h < dx[2] ? h : dx[2];
    T *buf[2] = {nullptr, nullptr};
    unsigned int *res = nullptr;
    unsigned int *res_host = nullptr;
    sbg_status rc = SBG_OK;
    auto done = [&](sbg_status r) {
        cudaStreamSynchronize(s);
        if (!on_device || buf[0] != out) dfree(buf[0]);
        dfree(buf[1]);
        dfree(res);
        hfree(res_host);
        return r;
    };
    cudaError_t e = cudaSuccess;
    if (on_device) {
        buf[0] = (T *)out;
        if (out != in) e = cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, s);
    } else {
        e = dmalloc((void **)&buf[0], bytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(buf[0], in, bytes, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = dmalloc((void **)&buf[1], bytes);
    if (e == cudaSuccess) e = dmalloc((void **)&res, sizeof(unsigned int));
    if (e == cudaSuccess) e = hmalloc((void **)&res_host, sizeof(unsigned int));
    if (e != cudaSuccess) return done(cuda_fail(e, "sbg_redistance: allocation or upload"));
    RedistArgs<T> a;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    for (int i = 0; i < 3; ++i) a.inv_dx[i] = (T)(1.0 / dx[i]);
    a.h2 = (T)(h * h);
    a.dalpha = (T)(o->cfl * h);
    a.band = (T)(o->band * h);
    const dim3 block(kRdX, kRdY, 1);
    const dim3 grid((unsigned)((nx + kRdX - 1) / kRdX), (unsigned)((ny + kRdY - 1) / kRdY),
                    (unsigned)((nz + kRdZ - 1) / kRdZ));
    int cur = 0;
    int64_t it = 0;
    double last = NAN;
    while (it < o->max_iter) {
        const bool check = ((it + 1) % o->check_every == 0) || (it + 1 == o->max_iter);
        if (check) {
            e = cudaMemsetAsync(res, 0, sizeof(unsigned int), s);
            if (e != cudaSuccess) return done(cuda_fail(e, "sbg_redistance: residual reset"));
        }
        a.in = buf[cur];
        a.out = buf[1 - cur];
        a.res = check ? res : nullptr;
        k_sussman<T><<<grid, block, 0, s>>>(a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return done(cuda_fail(e, "sbg_redistance: kernel launch"));
        cur = 1 - cur;
        ++it;
        if (check) {
            e = cudaMemcpyAsync(res_host, res, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return done(cuda_fail(e, "sbg_redistance: residual read"));
            float r;
            std::memcpy(&r, res_host, sizeof(r));
            last = (double)r;
            if (o->tol > 0.0 && last < o->tol) break;
        }
    }
    // the result into the caller's array
    if (on_device) {
        if (buf[cur] != out) e = cudaMemcpyAsync(out, buf[cur], bytes, cudaMemcpyDeviceToDevice, s);
    } else {
        e = cudaMemcpyAsync(out, buf[cur], bytes, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return done(cuda_fail(e, "sbg_redistance: result copy"));
    if (iters_out) *iters_out = it;
    if (res_out) *res_out = last;
    return done(rc);
}

}  // namespace sbg

using namespace sbg;

extern "C" sbg_status sbg_redistance(const int64_t dims[3], const double dx[3], const void *phi_in, void *phi_out,
                                     int32_t dtype, int32_t on_device, const sbg_redist_opts *opts,
                                     int64_t *iters_out, double *residual_out, void *stream) {
    if (!dims || !dx || !phi_in || !phi_out || !opts) return fail(SBG_ERR_INVALID_ARG, "sbg_redistance: null pointer");
    for (int i = 0; i < 3; ++i) {
        if (dims[i] < 1 || dims[i] > (int64_t)1 << 20)
            return fail(SBG_ERR_INVALID_ARG, "sbg_redistance: dims must lie in [1, 2^20]");
        if (!(dx[i] > 0.0) || !isfinite(dx[i])) return fail(SBG_ERR_INVALID_ARG, "sbg_redistance: dx > 0");
    }
    if (dtype != SBG_F32 && dtype != SBG_F64)
        return fail(SBG_ERR_INVALID_ARG, "sbg_redistance: dtype must be SBG_F32 or SBG_F64");
    if (opts->max_iter < 0 || opts->check_every < 1 || !(opts->cfl > 0.0) || !(opts->band > 0.0))
        return fail(SBG_ERR_INVALID_ARG, "sbg_redistance: max_iter >= 0, check_every >= 1, cfl > 0, band > 0");
    double h = dx[0] < dx[1] ? dx[0] : dx[1];
    h = h < dx[2] ? h : dx[2];
    const double courant = opts->cfl * h * (1.0 / dx[0] + 1.0 / dx[1] + 1.0 / dx[2]);
    if (courant > 1.0)
        return fail(SBG_ERR_INVALID_ARG, "sbg_redistance: cfl * min(dx) * sum(1/dx) = " + std::to_string(courant) +
                                             " above 1 (the upwind scheme is not monotone)");
    if ((dims[1] + kRdY - 1) / kRdY > 65535 || (dims[2] + kRdZ - 1) / kRdZ > 65535)
        return fail(SBG_ERR_INVALID_ARG, "sbg_redistance: Ny above 524280 or Nz above 1048560");
    if (!on_device && phi_in == phi_out)
        return fail(SBG_ERR_INVALID_ARG, "sbg_redistance: host input and output must differ");
    if (iters_out) *iters_out = 0;
    if (residual_out) *residual_out = NAN;
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SBG_F64)
        return redistance_t<double>(dims, dx, phi_in, phi_out, on_device, opts, iters_out, residual_out, s);
    return redistance_t<float>(dims, dx, phi_in, phi_out, on_device, opts, iters_out, residual_out, s);
}
