// Internal declarations of the sparse-block-grid library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sbg.h"

namespace sbg {

// ---------------------------------------------------------------------------
// errors
void set_error(const std::string &msg);
sbg_status fail(sbg_status s, const std::string &msg);
sbg_status cuda_fail(cudaError_t e, const char *what);

#define SBG_CUDA(call)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return sbg::cuda_fail(e_, #call); \
    } while (0)

#define SBG_LAUNCH_CHECK(what)                              \
    do {                                                    \
        cudaError_t e_ = cudaGetLastError();                \
        if (e_ != cudaSuccess) return sbg::cuda_fail(e_, what); \
    } while (0)

// Every allocation of the library (sbg_alloc.cu): the CUDA call behind a test
// hook that can make the n-th next allocation fail (sbg_debug_fail_alloc) and
// a table of the live allocations (sbg_debug_live_allocations).
cudaError_t dmalloc(void **p, size_t bytes);
cudaError_t dmalloc_async(void **p, size_t bytes, cudaStream_t s);
cudaError_t hmalloc(void **p, size_t bytes);
cudaError_t dfree(void *p);
cudaError_t dfree_async(void *p, cudaStream_t s);
cudaError_t hfree(void *p);

// ---------------------------------------------------------------------------
// inactive-voxel sentinel: a quiet NaN with a payload that arithmetic never
// produces (NVIDIA GPUs return the canonical 0x7fffffff for invalid ops), so a
// stored value is "outside Omega" iff its bits equal the sentinel.
constexpr uint32_t kSent32 = 0x7fc5b600u;
constexpr uint64_t kSent64 = 0x7ff8c5b600000000ull;

__host__ __device__ __forceinline__ float sentinel_f32() {
#ifdef __CUDA_ARCH__
    return __uint_as_float(kSent32);
#else
    union { uint32_t u; float f; } c{kSent32};
    return c.f;
#endif
}
__host__ __device__ __forceinline__ double sentinel_f64() {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)kSent64);
#else
    union { uint64_t u; double d; } c{kSent64};
    return c.d;
#endif
}
__device__ __forceinline__ bool is_sent(float v) { return __float_as_uint(v) == kSent32; }
__device__ __forceinline__ bool is_sent(double v) {
    return (uint64_t)__double_as_longlong(v) == kSent64;
}
template <typename T> __device__ __forceinline__ T sentinel();
template <> __device__ __forceinline__ float sentinel<float>() { return sentinel_f32(); }
template <> __device__ __forceinline__ double sentinel<double>() { return sentinel_f64(); }

// 26-neighbour numbering: k over (dz, dy, dx) in {-1,0,1}^3, z slowest,
// skipping the centre.  Face entries used by the 7-point stencil:
constexpr int kNbrXm = 12, kNbrXp = 13, kNbrYm = 10, kNbrYp = 15, kNbrZm = 4, kNbrZp = 21;
__host__ __device__ __forceinline__ int nbr_slot(int dx, int dy, int dz) {
    int k = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
    return k > 13 ? k - 1 : k;
}

constexpr int kNumRed = SBG_NRED;
constexpr int kRedMaxCtas = 148 * 8;

}  // namespace sbg

// ---------------------------------------------------------------------------
struct sbg_grid_s {
    int B = 8;
    int n_geoms = 1;
    float eps_mask = 0.f;
    float band_eps = 1.f;
    std::vector<int64_t> dims;              // [n_geoms * 3]
    std::vector<int64_t> geom_nactive;      // [n_geoms]
    std::vector<int64_t> geom_begin;        // [n_geoms] first block
    std::vector<int64_t> geom_count;        // [n_geoms] number of blocks
    int64_t nb = 0;
    int64_t n_active = 0;
    int64_t n_band = 0;
    // device arrays
    int4 *blocks = nullptr;        // [nb] (bx, by, bz, geometry)
    int32_t *nbr = nullptr;        // [nb * 26]
    int32_t *face_nbr = nullptr;   // [nb * 6]: -x, +x, -y, +y, -z, +z
    unsigned long long *hkeys = nullptr;
    int32_t *hvals = nullptr;
    int64_t hcap = 0;
    uint64_t *bitmap = nullptr;    // [nb * words]
    int32_t *wslab = nullptr;      // [nb] slab index or -1
    float *w = nullptr;            // [n_band * B^3]
    double *w64 = nullptr;         // same weights in FP64 (FP64 states and the reductions)
    int32_t *gdims = nullptr;      // [n_geoms * 4]: nx, ny, nz, 0
    double *partials = nullptr;    // reduction scratch [kRedMaxCtas * kNumRed]
    double *red_dev = nullptr;     // [kNumRed]
    double *red_host = nullptr;    // pinned [kNumRed]
    float *pad = nullptr;          // 16-byte-aligned page: 4 sentinels then 4 zeros (absent halo neighbours)
    float *eps = nullptr;          // [nb * B^3] diffusivity factor (inhomogeneous diffusion), FP32, preceded
                                   // by a ghost block of zeros (eps - 64, the start of its allocation)
    double *eps64 = nullptr;       // the same in FP64 (FP64 states, reductions of them)
    bool has_eps = false;
    float eps_max = 0.f;           // largest factor on an active voxel (stability limit)
    int eps_version = 0;           // bumped when the factor is set or cleared (captured graphs)
    uint64_t *heldbits = nullptr;  // [nb * words]: voxels held by the Dirichlet faces of heldbits_mask
    int heldbits_mask = -1;        // face set heldbits was computed for (-1: none yet)
    int2 *wmeta = nullptr;         // 4^3 blocks: [nb + 1] (first band row in wrow, band-row mask)
    float4 *wrow = nullptr;        // 4^3 blocks: surface weights of the band rows, in list order
    int64_t n_wrows = 0;
    int order = SBG_ORDER_TILED;   // block order of the list (sbg_build_opts.order)
    int *err = nullptr;            // device error word written by bounded waits (0 = none)
    // test hook (sbg_debug_stall_stage): the ring kernels skip the bulk copy of this group
    // (-1: none) and give up waiting after inject_wait_cycles
    int inject_stall_group = -1;
    long long inject_wait_cycles = 0;
    int inject_version = 0;        // bumped when the hook changes (captured graphs are redone)
    int *err_host = nullptr;       // pinned copy
    int64_t bytes = 0;
    int words() const { return (B * B * B + 63) / 64; }
    int b3() const { return B * B * B; }
};

struct sbg_state_s {
    sbg_grid grid = nullptr;
    int ns = 1;
    sbg_dtype dtype = SBG_F32;
    int64_t nslots = 0;            // nb * B^3
    void *base = nullptr;          // one allocation for everything below
    void *val[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [buffer][species]
    float *lo[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // F32X2 low parts
    int cur = 0;
    int64_t bytes = 0;
    // cached CUDA graph of an even number of steps
    cudaGraphExec_t graph = nullptr;
    int graph_cur = -1;
    int64_t graph_steps = 0;
    sbg_params graph_params{};
    int graph_variant = -1;
    int graph_ctas = -1;
    int graph_eps_version = -1;
    int graph_inject_version = -1;
    int variant = SBG_KERNEL_AUTO;  // step kernel choice (sbg_state_set_kernel)
    bool has_ghost = false;         // every val array is preceded by a ghost block of sentinels
                                    // (states made by sbg_state_create; not the adjoint's views)
    int ctas_per_sm = 0;
    void *wave = nullptr;           // plan of the wavefront kernel (sbg_step_stream.cu), made at first use
    // SBG_F32R (one species): val[b][0] holds the FP32 correction d; the base
    // b = bh + bl and the source r = L_h b are single arrays updated in place
    float *bh = nullptr, *bl = nullptr, *rsrc = nullptr;
    bool r_valid = false;           // r matches the base of every geometry
    int64_t since_refresh = 0;      // steps since r was recomputed and d folded
    // external space-time source a_n S_s(x) (sbg_step_source): S_s per slot in
    // the state's precision, 0 on inactive voxels; null: species without one
    void *ext[2] = {nullptr, nullptr};
    size_t elem() const { return dtype == SBG_F64 ? 8 : 4; }
};

namespace sbg {
// implemented in sbg_reduce.cu: reads and clears the grid's device error word
sbg_status check_device_error(sbg_grid g, cudaStream_t s);
// implemented in sbg_step.cu
sbg_status validate_params(sbg_grid g, const sbg_params *p, int ns);
// implemented in sbg_reduce.cu
sbg_status reduce_species(sbg_grid g, sbg_state st, const sbg_params *p, int geom, int species,
                          int which_buffer, double *out_host, cudaStream_t stream);
// one segmented reduction over several geometries (sbg_reduce.cu): the CTA
// records each geometry's reduction writes, and the reduction itself
int64_t reduce_records(sbg_grid g, sbg_state st, const sbg_params *p, int geom);
sbg_status reduce_geometries(sbg_grid g, sbg_state st, const sbg_params *p, const int *geoms, int ngeoms,
                             int species, double *records, int *seg_dev, double *out_dev, double *out_host,
                             cudaStream_t s);
// sum of one species over the active voxels of a box and their count into
// dst[0..1] (device); kernel launches only
sbg_status launch_box_sum(sbg_grid g, sbg_state st, int geom, int species, const int64_t lo[3], const int64_t hi[3],
                          double *dst, cudaStream_t s);
sbg_status check_box_args(sbg_grid g, sbg_state st, int geom, int species, const char *who);
// implemented in sbg_step.cu: one step from buffer src with the external
// source scaled by `scale` (plain kernel; no state bookkeeping)
sbg_status launch_step_ext(sbg_grid g, sbg_state st, const sbg_params *p, int src, double scale, cudaStream_t s);
// implemented in sbg_step.cu: nsteps steps (graphs, SBG_F32R refreshes); no synchronisation
sbg_status step_n(sbg_grid g, sbg_state st, const sbg_params *p, int64_t nsteps, cudaStream_t s);
// SBG_F32R: recompute r = L_h (b + d) over every geometry and fold d into b
// (kernel launches only, no synchronisation)
sbg_status refresh_source(sbg_grid g, sbg_state st, const sbg_params *p, cudaStream_t stream);
// steps between refreshes of an SBG_F32R state inside sbg_step
constexpr int64_t kRefreshSteps = 256;
// implemented in sbg_step_stream.cu: frees a state's wavefront plan (if any)
void wave_destroy(sbg_state st);
// implemented in sbg_step.cu: makes g->heldbits match the Dirichlet faces of
// p (one small kernel when they changed); call before any stream capture
sbg_status prepare_held_bits(sbg_grid g, const sbg_params *p, cudaStream_t s);
}  // namespace sbg
