/*
 * sbg.h - C ABI of the sparse-block-grid reaction-diffusion library (sm_103a).
 *
 * The library advances the reaction-diffusion PDE of Eq. 1 (Sec. 2) with the
 * FTCS / forward-Euler scheme of Sec. 2.3 on a geometry-adapted sparse block
 * grid: only the B x B x B voxel blocks that contain pore space (phi > eps,
 * Eq. 3 sign convention) are stored and updated.  Neighbours outside the pore
 * space take the centre value (the no-flux rule of Sec. 2.3), the surface
 * reaction is localised by phi (Sec. 3.5), and FP64 reductions give mass,
 * fluxes, residual, effective diffusivity and tortuosity (Eq. 2).
 *
 * Conventions (every entry point):
 *  - No exceptions cross the ABI.  Every call returns an sbg_status; on error
 *    sbg_last_error() holds a message for the calling thread.
 *  - Dense arrays are [Nz][Ny][Nx], x fastest (a contiguous [Nz, Ny, Nx]
 *    tensor), with dims[3] = {Nx, Ny, Nz}.  A dims entry need not be a
 *    multiple of the block edge; the library pads with inactive voxels.
 *  - Pointers flagged "host or device" are read (or written) during the call
 *    only; the caller keeps ownership.  Library objects (sbg_grid, sbg_state)
 *    own their device memory until the matching destroy call.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it; the call synchronises the stream only
 *    when it returns host scalars (reductions) or reads/writes host arrays.
 *  - One grid/state must not be used from two host threads at once.
 *
 * Face numbering: 0 = x-low, 1 = x-high, 2 = y-low, 3 = y-high, 4 = z-low,
 * 5 = z-high.
 */
#ifndef SBG_H
#define SBG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbg_grid_s *sbg_grid;   /* geometry: blocks, hash, neighbour table, masks */
typedef struct sbg_state_s *sbg_state; /* species fields in block layout, ping-pong pair  */
typedef struct sbg_tape_s *sbg_tape;   /* forward checkpoints for the adjoint             */

typedef enum {
    SBG_OK = 0,
    SBG_ERR_INVALID_ARG = 1,   /* bad pointer, size, dims, block edge or parameter            */
    SBG_ERR_OOM = 2,           /* a device or host allocation failed                            */
    SBG_ERR_CUDA = 3,          /* a CUDA call or kernel launch failed                           */
    SBG_ERR_UNSTABLE_DT = 4,   /* dt above sbg_stability_limit() and allow_unstable == 0       */
    SBG_ERR_NONFINITE = 5,     /* a NaN or Inf was found in the state by a reduction           */
    SBG_ERR_TIMEOUT = 6,       /* a bounded device wait gave up                                 */
    SBG_ERR_NOT_CONVERGED = 7, /* sbg_run_to_steady reached max_steps first                     */
    SBG_ERR_BOUNDS = 8         /* debug build only (libsbg_debug.so, SBG_DEBUG): a step kernel met a
                                  block, neighbour or band-row index outside its table, skipped
                                  the access and recorded this in the grid's error word         */
} sbg_status;

typedef enum {
    SBG_F32 = 0,   /* FP32 state and stencil                                                   */
    SBG_F64 = 1,   /* FP64 state and stencil                                                   */
    SBG_F32X2 = 2, /* compensated FP32: value = hi + lo, two FP32 arrays, FP32 arithmetic with
                      error-free sums, so that forward Euler keeps increments far below one
                      FP32 ulp (needed for steady states to a 1e-8 relative residual)         */
    SBG_F32R = 3   /* FP32 correction on a compensated base (one species): value = b + d with
                      b = hi + lo (FP32 pair) and d an FP32 correction.  Each step advances d
                      by forward Euler with the source r = L_h b (stored as FP32), which in
                      exact arithmetic is the forward-Euler step of b + d; every reduction and
                      every 256 steps the library recomputes r from b + d in double-float
                      arithmetic and folds d into b.  The step moves 12 B per voxel in plain
                      FP32 arithmetic; the rounding of d is relative to the change since the
                      last fold, so steady states reach residuals like SBG_F32X2's         */
} sbg_dtype;

enum { SBG_FACE_NOFLUX = 0, SBG_FACE_DIRICHLET = 1 };

/* sbg_build options. */
typedef struct {
    int32_t block;          /* block edge B: 4 or 8                                             */
    int32_t phi_on_device;  /* 1: phi is a device pointer; 0: host pointer                     */
    float eps_mask;         /* a voxel is in the pore space iff phi > eps_mask (FP32 compare);
                               0 selects FLT_EPSILON, the paper's insertion bound (Appendix B,
                               Listings 5 and 6)                                                */
    float band_eps;         /* half-width eps_b of the surface delta
                               w = (1 + cos(pi phi / eps_b)) / (2 eps_b) for 0 < phi < eps_b;
                               0 selects 1.0                                                    */
    int32_t order;          /* order of the active blocks in the list (a layout choice of this
                               library; results do not depend on it):
                               SBG_ORDER_TILED (0): tiles of 32^3 voxels, x-fastest, blocks
                               x-fastest inside a tile, so that a CTA walking a contiguous range
                               of the list meets a block's face neighbours soon after it;
                               SBG_ORDER_PLANES (1): plain x-fastest order of the box blocks
                               (z slowest), so that a kernel whose CTAs take the list's groups
                               in turn sweeps the box plane by plane and finds every face
                               neighbour in L2 (the streaming kernel, SBG_KERNEL_STREAM)        */
} sbg_build_opts;

enum { SBG_ORDER_TILED = 0, SBG_ORDER_PLANES = 1 };

/* Physics of a run (constant D per species; Eq. 1 with a linear f).
 * Species 0 (A) loses k_surf * w * A + decay[0] * A per unit time; with two
 * species, species 1 (B) gains the same k_surf * w * A and loses decay[1] * B. */
typedef struct {
    double dx[3];             /* voxel spacing along x, y, z                                   */
    double dt;                /* forward-Euler step                                             */
    int32_t nspecies;         /* 1 or 2 (must equal the state's)                               */
    int32_t face_type[6];     /* SBG_FACE_NOFLUX or SBG_FACE_DIRICHLET per face                */
    double D[2];              /* diffusion coefficient per species                             */
    double decay[2];          /* linear bulk loss rate per species                              */
    double k_surf;            /* surface reaction rate A -> B (a sink of A with one species)    */
    double face_value[6];     /* value held on Dirichlet faces (species 0); the driving
                                 difference dC of sbg_effective_D is |value[0] - value[1]|    */
    int32_t allow_unstable;   /* 1: skip the dt <= limit check                                  */
} sbg_params;

typedef struct {
    int64_t dims[3];          /* box size of geometry 0                                          */
    int32_t block;            /* B                                                              */
    int32_t n_geoms;          /* 1 for sbg_build                                                */
    int64_t n_blocks;         /* active blocks (all geometries)                                 */
    int64_t n_active;         /* active voxels (all geometries)                                 */
    int64_t n_band_blocks;    /* blocks holding a surface-weight slab                           */
    double porosity;          /* n_active / box voxels (geometry 0 for a batch)                 */
    int64_t device_bytes;     /* device memory held by the grid                                 */
} sbg_grid_info_t;

/* Reduction output layout: out[s * SBG_NRED + q] for species s. */
enum {
    SBG_RED_MASS = 0,      /* sum over active voxels of u dV (the mass curve of Sec. 3.4)      */
    SBG_RED_JIN = 1,       /* x-flux through the plane between x = 0 and x = 1:
                              sum over (y,z) with both voxels active of
                              D (u_0 - u_1) / dx * dy dz                                      */
    SBG_RED_JOUT = 2,      /* same between x = Nx-2 and x = Nx-1                               */
    SBG_RED_RESIDUAL = 3,  /* ||L_h u||_2 over free active voxels, L_h u the bracketed FTCS
                              right-hand side, evaluated in FP64                              */
    SBG_RED_MIN = 4,       /* min of u over active voxels                                       */
    SBG_RED_MAX = 5,       /* max of u over active voxels                                       */
    SBG_RED_NONFINITE = 6, /* count of NaN/Inf active voxels                                    */
    SBG_RED_NACTIVE = 7,   /* count of active voxels                                            */
    SBG_NRED = 8
};

/* ---- grid ------------------------------------------------------------------
 * Block activation and indexing (Sec. 2.3-2.4: chunks stored only if they
 * hold at least one inserted point; Appendix B Listing 5 for the insertion
 * test).  Builds, on `stream`: the compact list of active blocks in tiled
 * order (tiles of 32^3 voxels in x-fastest order, blocks x-fastest inside a
 * tile, so that face neighbours are close in the list), an open-addressing device hash from block coordinates to block
 * id, the 26-neighbour table (id or -1), one occupancy bitmap per block and
 * the surface-weight slabs of blocks that meet the band 0 < phi < eps_b.
 * phi: dense FP32 [Nz][Ny][Nx], host or device (opts->phi_on_device).
 * Returns INVALID_ARG for null pointers, dims < 1 or > 65535*B, block not
 * 4/8; OOM/CUDA on allocation or launch failure.  Synchronises `stream`. */
sbg_status sbg_build(const float *phi, const int64_t dims[3], const sbg_build_opts *opts,
                     void *stream, sbg_grid *out);

/* Batched geometries (no counterpart in the paper; a batching pattern of this
 * library): n geometries, each with its own dims and phi, concatenated into one
 * block list whose blocks carry their geometry id.  phis[g] as for sbg_build. */
sbg_status sbg_build_batch(int32_t n, const float *const *phis, const int64_t *dims /* [n][3] */,
                           const sbg_build_opts *opts, void *stream, sbg_grid *out);

sbg_status sbg_grid_info(sbg_grid grid, sbg_grid_info_t *info);

/* Per-geometry counts of a (batched) grid: n_active[g], first block and
 * number of blocks of geometry g (blocks are sorted by geometry).  Arrays of
 * length info.n_geoms, host memory; any may be NULL. */
sbg_status sbg_grid_geometry_info(sbg_grid grid, int64_t *n_active, int64_t *block_begin,
                                  int64_t *block_count);

/* Copies the 26-neighbour table ([n_blocks][26] int32, -1 = no block; entry
 * k enumerates (dz, dy, dx) in {-1,0,1}^3 z-slowest, skipping (0,0,0)) and the
 * block coordinates ([n_blocks][4] int32: bx, by, bz, geometry) to host
 * memory; either may be NULL.  For inspection and tests. */
sbg_status sbg_grid_tables(sbg_grid grid, int32_t *nbr26, int32_t *blocks);

void sbg_grid_destroy(sbg_grid grid);

/* ---- inhomogeneous diffusion (Eq. 6; the functor of Appendix B Listing 6) ----
 * A per-voxel diffusivity factor eps for single-species states: species 0
 * diffuses with D_0 * eps_i, and the flux between a voxel and a face
 * neighbour uses the arithmetic mean of their diffusivities,
 *   u'_i = u_i + dt ( sum_a 1/dx_a^2 [ D_{+a} (u~_{i+a} - u_i) - D_{-a} (u_i - u~_{i-a}) ] - decay_0 u_i ),
 *   D_{+-a} = D_0 (eps_i + eps_{i+-a}) / 2,
 * with the no-flux rule as for constant D (a neighbour outside Omega takes the
 * centre's value, so its face carries no flux).  The factor lives in the grid
 * (FP32 and FP64 copies, block layout) and applies to every SBG_F32 or
 * SBG_F64 one-species state of the grid; stepping a state of another kind,
 * with two species or with k_surf != 0 returns SBG_ERR_INVALID_ARG while a
 * factor is set.  The explicit limit becomes that of D_0 * max(eps).
 * Reductions use the same face diffusivities for fluxes and the residual.
 *
 * sbg_grid_set_diffusivity: eps from a dense array [Nz][Ny][Nx] of
 * dense_dtype (SBG_F32 or SBG_F64; host or device) for geometry `geom`;
 * values must be finite and >= 0 on active voxels (SBG_ERR_INVALID_ARG
 * otherwise; the factor is then cleared).  Synchronises `stream`. */
sbg_status sbg_grid_set_diffusivity(sbg_grid grid, int32_t geom, const void *dense, int32_t dense_dtype,
                                    int32_t on_device, void *stream);

/* eps from phi by Eq. 6, evaluated on the device in FP64 per active voxel:
 *   eps = d_min + d_max / (1 + exp(-(gamma1 + gamma2 phi))),
 * phi: FP32 [Nz][Ny][Nx] (host or device) of geometry `geom`.  Requires
 * d_min >= 0, d_max >= 0.  Synchronises `stream`. */
sbg_status sbg_grid_set_diffusivity_sigmoid(sbg_grid grid, int32_t geom, const float *phi, int32_t phi_on_device,
                                            double d_min, double d_max, double gamma1, double gamma2,
                                            void *stream);

/* Removes the factor (constant D per species again). */
sbg_status sbg_grid_clear_diffusivity(sbg_grid grid);

/* ---- state -----------------------------------------------------------------
 * nspecies fields in block layout u[s][block * B^3 + (z*B + y)*B + x] plus the
 * ping-pong partner (the two concentration properties of Appendix B Listing
 * 7).  Inactive voxels of active blocks hold a NaN sentinel and are never
 * updated. */
sbg_status sbg_state_create(sbg_grid grid, int32_t nspecies, sbg_dtype dtype, sbg_state *out);

/* Scatters a dense array into species `species`.  dense: [Nz][Ny][Nx] of
 * dense_dtype (SBG_F32 or SBG_F64), host or device (on_device).  Values of
 * inactive voxels are ignored; a NaN input is stored as a canonical NaN so
 * that reductions report it.  For SBG_F32X2 states the value is split into
 * hi = fl32(v), lo = fl32(v - hi); SBG_F32R states store that pair as the
 * base with a zero correction (the source r is recomputed before the next
 * step).  For a batch, `geom` selects the geometry (0 otherwise).
 * Synchronises `stream` when dense is host memory. */
sbg_status sbg_state_set(sbg_grid grid, sbg_state state, int32_t geom, int32_t species,
                         const void *dense, int32_t dense_dtype, int32_t on_device, void *stream);

/* Gathers species `species` into a dense array (inactive voxels -> 0).  For
 * SBG_F32X2 states an SBG_F64 output receives hi + lo, for SBG_F32R states
 * hi + lo + d. */
sbg_status sbg_state_get(sbg_grid grid, sbg_state state, int32_t geom, int32_t species,
                         void *dense, int32_t dense_dtype, int32_t on_device, void *stream);

/* External space-time source (the reaction term f(x, t) of Eq. 1 in the
 * separable form f_s(x, t_n) = a_n S_s(x); the manufactured source of the
 * verification in Sec. 3.1 and its appendix is S(r) exp(-B t)).
 * sbg_state_set_source copies the spatial part S of species `species` for
 * geometry `geom` from a dense [Nz][Ny][Nx] array (SBG_F32 or SBG_F64, host
 * or device) into a per-slot array of the state's precision (allocated on
 * first use, 0 on inactive voxels); SBG_F32 and SBG_F64 states only.
 * Synchronises `stream`.  Errors: SBG_ERR_INVALID_ARG (bad geometry,
 * species, dtypes, a non-finite value on an active voxel). */
sbg_status sbg_state_set_source(sbg_grid grid, sbg_state state, int32_t geom, int32_t species,
                                const void *dense, int32_t dense_dtype, int32_t on_device, void *stream);

/* Frees the source arrays of every species. */
sbg_status sbg_state_clear_source(sbg_state state);

/* nsteps forward-Euler steps with the source: step n (0-based) computes
 *   u' = u + dt ( L_h u - decay u -+ k w u_A + a_n S_s ),
 * a_n = factors[n] (host array of nsteps finite values; a species without a
 * source adds nothing), the source term rounded as fma(a_n, S_s, transfer).
 * One launch of the one-thread-per-voxel kernel per step (a_n is a kernel
 * argument, so no graph is replayed).  Constant D only (no diffusivity
 * factor).  Asynchronous on `stream`.  Errors: those of sbg_step, and
 * SBG_ERR_INVALID_ARG for other state types or a non-finite factor. */
sbg_status sbg_step_source(sbg_grid grid, sbg_state state, const sbg_params *params, int64_t nsteps,
                           const double *factors, void *stream);

/* Step-kernel choice for a state (this library's tuning knob; no
 * counterpart in the paper).  variant: SBG_KERNEL_AUTO (the streaming kernel
 * where it applies: SBG_F32 states of one or two species, SBG_F32R states
 * without a surface reaction, SBG_F32 states of one species with a
 * diffusivity factor, and SBG_F32X2 states, on 4^3 blocks; else
 * the pipelined kernel with cp.async halos where it exists, else the
 * one-thread-per-voxel kernel), SBG_KERNEL_PLAIN
 * (one thread per voxel, block tile in shared memory, one launch-sized grid)
 * SBG_KERNEL_PIPELINED (persistent CTAs streaming groups of blocks
 * through a bulk-copy ring: 1024-voxel groups and two z-paired rows of four
 * voxels per thread for one FP32 species and SBG_F32R states, 512-voxel
 * groups and one row per thread for the other FP32-based states; not for
 * SBG_F64) or
 * SBG_KERNEL_PIPELINED_PREFETCH (the same, with face halos prefetched one
 * group ahead in registers: fewer CTAs per SM, less exposed latency) or
 * SBG_KERNEL_PIPELINED_ASYNC (face halos copied one group ahead into shared
 * memory with per-thread cp.async: no extra registers; with it the FP32 states
 * of two species or with a diffusivity factor and SBG_F32X2 states run two
 * z-paired rows per thread too, except in batched steps).  ctas_per_sm:
 * persistent CTAs per SM for the pipelined kernel (0 = as many as fit).
 * SBG_KERNEL_STREAM (SBG_F32 states of one or two species, SBG_F32R states
 * without a surface reaction, one FP32 species with a diffusivity factor
 * (u and the factor read at the same offsets) and SBG_F32X2 states (hi and
 * lo read at the same offsets), on 4^3 blocks:
 * CTAs take groups of 16 blocks (12 for two species) in turn, one
 * x-row of four voxels per thread, every neighbour row read straight from
 * global memory through L1; best with SBG_ORDER_PLANES grids, whose plane
 * order keeps the sweep's neighbour planes in L2; states of other kinds fall
 * back to SBG_KERNEL_AUTO's choice).
 * SBG_KERNEL_WAVE / SBG_KERNEL_WAVE4 (the streaming kernel's states on an
 * SBG_ORDER_PLANES grid of one geometry): 2 / 4 steps per launch, run as a
 * wavefront over the planes of blocks (step n+1 on one plane while step n+2
 * runs a few planes behind it), the intermediate steps kept in rings of a few
 * planes that stay in L2, so that HBM sees one read and one write of the state
 * per launch; a remainder of fewer steps runs the streaming kernel.  The first
 * sbg_step of such a state builds its plan (a host synchronisation and ~5 MB
 * per ring plane and species on a 512^3 grid); a wait of one work unit on
 * another is bounded like the ring kernels' (SBG_ERR_TIMEOUT).  Other grids and
 * states fall back to SBG_KERNEL_AUTO's choice.
 * Results are bitwise identical across variants.  The pipelined kernels index
 * voxel slots with 32-bit integers: a grid of 2^31 or more slots (blocks x
 * B^3) runs the one-thread-per-voxel kernel under SBG_KERNEL_AUTO, and
 * sbg_step fails with SBG_ERR_INVALID_ARG under the explicit pipelined
 * variants (as do batched steps and the FP32 adjoint on such a grid). */
enum {
    SBG_KERNEL_AUTO = 0,
    SBG_KERNEL_PLAIN = 1,
    SBG_KERNEL_PIPELINED = 2,
    SBG_KERNEL_PIPELINED_PREFETCH = 3,
    SBG_KERNEL_PIPELINED_ASYNC = 4,
    SBG_KERNEL_STREAM = 5,
    SBG_KERNEL_WAVE = 6,
    SBG_KERNEL_WAVE4 = 7
};
sbg_status sbg_state_set_kernel(sbg_state state, int32_t variant, int32_t ctas_per_sm);

/* Copies all species of `src` into `dst` (same grid, dtype and species). */
sbg_status sbg_state_copy(sbg_state dst, sbg_state src, void *stream);

void sbg_state_destroy(sbg_state state);

/* ---- time stepping -----------------------------------------------------------
 * nsteps forward-Euler FTCS steps of Eq. 1 (Sec. 2.3; Appendix B Listing 6
 * for the per-point update):
 *   u'_i = u_i + dt ( sum_a D_s/dx_a^2 [(u~_{i+a} - u_i) - (u_i - u~_{i-a})]
 *                     - decay_s u_i -/+ k_surf w_i u_{A,i} )
 * with u~_j = u_j if j is an active voxel, else u_i (no-flux rule).  Active
 * voxels on Dirichlet faces are held.  Each step reads one buffer and writes
 * the other.  Launches are enqueued on `stream` (replayed from a captured CUDA
 * graph when nsteps is large); no synchronisation.  Returns UNSTABLE_DT when
 * dt > sbg_stability_limit() unless params->allow_unstable. */
sbg_status sbg_step(sbg_grid grid, sbg_state state, const sbg_params *params, int64_t nsteps,
                    void *stream);

/* Explicit stability limit: Eq. 10 (2-D, pure diffusion) extended to every
 * axis with more than one voxel, with each species' largest linear loss rate
 * (decay, plus k_surf / eps_b for species 0) added:
 *   dt_lim = min_s 1 / (2 D_s sum_a dx_a^-2 + r_s,max).
 * Returns the limit, or -1 on a null pointer. */
double sbg_stability_limit(const sbg_params *params, const int64_t dims[3], double band_eps);

/* ---- reductions -------------------------------------------------------------
 * Reductions over the current state, accumulated in FP64 (FP64 states) or in
 * double-float pairs per voxel and warp and FP64 above (FP32-based states;
 * ~48-bit significand, B300 runs FP64 at a small fraction of its FP32 rate);
 * per-CTA partials in a scratch buffer of the grid, then a fixed-order final
 * pass: the result is deterministic.  out: host double[nspecies * SBG_NRED]
 * (layout above); min and max are those of the stored FP32 values (hi parts
 * for compensated states).  For a batch, `geom` selects the geometry (-1 =
 * all geometries together).  For SBG_F32R states the same pass also stores
 * the source r = L_h u and folds the correction into the base (the field is
 * unchanged up to double-float rounding).  Synchronises `stream`. */
sbg_status sbg_reduce(sbg_grid grid, sbg_state state, const sbg_params *params, int32_t geom,
                      double *out, void *stream);

/* sbg_reduce without the synchronisation: enqueues the same reductions (and,
 * for SBG_F32R states, the same refresh of r and fold of the correction) on
 * `stream`, then an asynchronous copy of the results into `out`
 * (nspecies * SBG_NRED doubles, same layout; host memory, page-locked for the
 * copy to be asynchronous, or device memory).  `out` holds the results once
 * `stream` has passed this call (an event, a synchronisation); until then it
 * must stay allocated and untouched.  The device error word of bounded waits
 * is not read here: the next synchronising call reports it.  This lets a
 * solver enqueue the next steps before it reads a convergence check. */
sbg_status sbg_reduce_async(sbg_grid grid, sbg_state state, const sbg_params *params, int32_t geom, double *out,
                            void *stream);

/* The monitoring check of a transient run (the mass total of Sec. 3.4, the
 * x-face fluxes, min/max and the non-finite and active counts), enqueued like
 * sbg_reduce_async, without the residual ||L_h u||: the SBG_RED_RESIDUAL slot
 * of every species reads NaN.  Every other scalar is bitwise the value
 * sbg_reduce_async gives for the same state (same kernels' accumulation
 * order).  It reads each species' values once (plus the +x neighbours of the
 * inlet and outlet planes) instead of evaluating the stencil, so it costs a
 * memory pass rather than the residual's double-float arithmetic.  SBG_F32R
 * states: no refresh of the source and no fold (the state is not touched).
 * Same ownership, ordering and error rules as sbg_reduce_async. */
sbg_status sbg_check_async(sbg_grid grid, sbg_state state, const sbg_params *params, int32_t geom, double *out,
                           void *stream);

/* The same FP64 reduction for callers that may not allocate device memory
 * (their memory belongs to another allocator, such as a framework's caching
 * allocator or a fixed serving arena, or allocation latency is not allowed in
 * their loop).  No counterpart in the paper.  It calls no cudaMalloc or
 * cudaFree: the per-CTA partial records live in a fixed 256 KiB device array
 * inside the library, held on every GPU that loads it until exit.
 *   species  reduced species (0 or 1);
 *   out_dev  caller-owned DEVICE buffer of SBG_NRED doubles, same layout as
 *            one species of sbg_reduce; written in stream order, no host copy
 *            and no synchronisation (read it after the stream has run);
 *   limit    the reduced range (one geometry, or all with geom = -1) may hold
 *            at most 2^28 voxel slots (blocks x B^3); larger ranges return
 *            SBG_ERR_INVALID_ARG - use sbg_reduce for them.
 * Every call looks up the array's device address (cudaGetSymbolAddress, a
 * host-side lookup that allocates nothing), so a device reset or a re-created
 * context never leaves a stale address; the first call on a device loads the
 * library's device code there, so make that first call before any stream
 * capture.
 * All calls share the array: calls whose kernels may overlap on the GPU
 * (unordered streams) race and must be serialised by the caller.  Unlike
 * sbg_reduce it does not read the grid's device error word.  Results equal
 * sbg_reduce's up to the order of the FP64 sums. */
sbg_status sbg_reduce_noalloc(sbg_grid grid, sbg_state state, const sbg_params *params, int32_t geom,
                              int32_t species, double *out_dev, void *stream);
/* (For SBG_F32R states sbg_reduce_noalloc only reads the state: no source
 * update, no fold.) */

/* Sum of species `species` over the active voxels of geometry `geom` with
 * lo <= (x, y, z) < hi (voxel coordinates; the box may extend past the
 * grid), and their number: out (host, 2 doubles) = {sum u, count}.  The mass
 * of the bleached region of a simulated FRAP experiment (Sec. 3.3).
 * Double-float per voxel and warp (FP32-based states) or FP64, then FP64 per
 * CTA and a fixed-order final sum.  Synchronises `stream`. */
sbg_status sbg_reduce_box(sbg_grid grid, sbg_state state, int32_t geom, int32_t species, const int64_t lo[3],
                          const int64_t hi[3], double *out, void *stream);

/* Simulated FRAP (Sec. 3.3): advances `state` by n_samples * steps_per_sample
 * steps of `params` (exactly as sbg_step) and records the sum of species
 * `species` over the active voxels of the box lo <= (x, y, z) < hi of
 * geometry `geom` before the first step and after every steps_per_sample
 * steps.  sums (host, n_samples + 1 doubles) receives the box sums in order;
 * count (host, may be NULL) the number of active voxels in the box.  The
 * sums stay on the device until one copy at the end (no synchronisation
 * between samples); an even steps_per_sample keeps the cached step graph.
 * Synchronises `stream`.  Errors: SBG_ERR_INVALID_ARG (bad geometry, species
 * or counts), those of sbg_step. */
sbg_status sbg_frap_curve(sbg_grid grid, sbg_state state, const sbg_params *params, int32_t geom, int32_t species,
                          const int64_t lo[3], const int64_t hi[3], int64_t steps_per_sample, int32_t n_samples,
                          double *sums, int64_t *count, void *stream);

/* Least-squares fit of a reference FRAP curve to a measured one over a time
 * scale (Sec. 3.3: the bulk-box curve fitted to the porous one): the scale s
 * in [s_lo, s_hi] that minimises sum_i (f[i] - g(s t[i]))^2, g the
 * piecewise-linear interpolant of (t_ref, f_ref).  A bulk curve at D_ref
 * evaluated at s t is the bulk curve at s D_ref evaluated at t, so
 * D_eff = s D_ref.  Host arrays: t, f (n >= 1, t >= 0), t_ref strictly
 * increasing with t_ref[0] <= s_lo min t and t_ref[m-1] >= s_hi max t
 * (m >= 2).  A scan of 4001 points, then golden-section search in the best
 * scan interval.  scale (host) gets s; rss (host, may be NULL) the residual
 * sum of squares.  Pure host code; no device work. */
sbg_status sbg_frap_fit(const double *t, const double *f, int64_t n, const double *t_ref, const double *f_ref,
                        int64_t m, double s_lo, double s_hi, double *scale, double *rss);

/* The normalised recovery curve of a simulated FRAP run (Sec. 3.3): runs
 * sbg_frap_curve (n_samples * steps_per_sample steps of `params`, the box sum
 * of `species` over lo <= (x, y, z) < hi before the first step and after
 * every steps_per_sample steps) and writes, for i = 0..n_samples (host
 * arrays of n_samples + 1 doubles),
 *   t[i] = i * steps_per_sample * dt,
 *   F[i] = M_box(t_i) / (c n_box),
 * c the mean of the species over every active voxel of the geometry before
 * the first step (conserved in a closed box: the level the box recovers to)
 * and n_box the active voxels in the box (*count, may be NULL).  Each curve
 * is thus normalised by its own equilibrium, so that the pore curve and a
 * bulk reference curve both tend to 1.  Synchronises `stream`.  Errors:
 * those of sbg_frap_curve; SBG_ERR_INVALID_ARG when the box holds no active
 * voxel or the field sums to zero. */
sbg_status sbg_frap_recovery(sbg_grid grid, sbg_state state, const sbg_params *params, int32_t geom,
                             int32_t species, const int64_t lo[3], const int64_t hi[3], int64_t steps_per_sample,
                             int32_t n_samples, double *t, double *F, int64_t *count, void *stream);

/* The FRAP estimate of the pore-space effective diffusivity (Sec. 3.3 and
 * Eq. 2): fits the reference curve (t_ref, F_ref), recorded in the bulk at
 * diffusivity D_ref, to the measured curve (t, F) over a time scale s
 * (sbg_frap_fit, same arguments and bounds) and returns
 *   D_eff = s D_ref,  tau = D_ref / D_eff = 1 / s (inf when s <= 0),
 * plus s (scale) and the residual sum of squares (rss); scale and rss may be
 * NULL.  Host arrays and outputs; no device work.  Errors: those of
 * sbg_frap_fit; SBG_ERR_INVALID_ARG for D_ref not finite and > 0. */
sbg_status sbg_frap_effective_D(const double *t, const double *F, int64_t n, const double *t_ref, const double *F_ref,
                                int64_t m, double D_ref, double s_lo, double s_hi, double *D_eff, double *tau,
                                double *scale, double *rss);

/* Effective diffusivity and diffusive tortuosity (Eq. 2: tau = D / D_eff with
 * the pore-space D_eff) from the x-face fluxes of species 0:
 *   D_eff = J L / (dC A), J = (J_in + J_out) / 2, L = (Nx - 1) dx,
 *   A = Ny dy Nz dz, dC = |face_value[0] - face_value[1]|,
 *   psi = n_active / (Nx Ny Nz), tau = psi D / D_eff (inf when D_eff <= 0).
 * D_eff is the superficial value (per box cross-section).  Host outputs. */
sbg_status sbg_effective_D(sbg_grid grid, sbg_state state, const sbg_params *params, int32_t geom,
                           double *D_eff, double *tau, double *psi, void *stream);

/* Steps until the relative residual ||L_h u|| / ||L_h u^0|| of species 0 drops
 * below tol, checking every check_every steps; *steps_done and *rel_residual
 * report where it stopped.  Returns NOT_CONVERGED at max_steps and NONFINITE
 * when a check finds a NaN/Inf. */
sbg_status sbg_run_to_steady(sbg_grid grid, sbg_state state, const sbg_params *params, double tol,
                             int64_t check_every, int64_t max_steps, int64_t *steps_done,
                             double *rel_residual, void *stream);

/* Batched steady-state solve (no counterpart in the paper: this library's
 * batching pattern) for a grid from sbg_build_batch and one SBG_F32,
 * SBG_F32X2 or SBG_F32R state: every geometry not yet converged advances by one
 * persistent, pipelined launch per step over a device work list of 512-voxel
 * spans (never straddling geometries), replayed from a captured CUDA graph of
 * check_every launches (rounded up to even); after each interval each active
 * geometry's FP64 relative residual ||L_h u|| / ||L_h u^0|| (species 0) is
 * computed and geometries below tol leave the work list.  Host outputs of
 * length n_geoms: steps_done[g] (steps at which g stopped) and
 * rel_residual[g].  Returns NOT_CONVERGED when some geometry is still above
 * tol after max_steps, NONFINITE on a NaN/Inf.  Synchronises `stream`. */
sbg_status sbg_batch_run_to_steady(sbg_grid grid, sbg_state state, const sbg_params *params, double tol,
                                   int64_t check_every, int64_t max_steps, int64_t *steps_done,
                                   double *rel_residual, void *stream);

/* ---- adjoint (no counterpart in the paper: this library's differentiation) -------
 * The step is linear, u^{n+1} = M u^n, so the gradient of a loss L(u^N) runs
 * lambda^n = M^T lambda^{n+1} backwards from lambda^N = dL/du^N: the
 * transposed masked stencil (an inactive neighbour contributes nothing, a
 * Dirichlet-held neighbour counts in the diagonal but carries lambda = 0)
 * plus the transposed A -> B coupling.  Held values are not free parameters:
 * lambda is 0 on held voxels.
 *
 * sbg_forward_record advances `state` (SBG_F32 or SBG_F64) by nsteps like
 * sbg_step and keeps a device copy of the state every checkpoint_every steps
 * (ceil(nsteps / K) copies) in a new tape, which owns that memory.
 * Synchronises nothing. */
sbg_status sbg_forward_record(sbg_grid grid, sbg_state state, const sbg_params *params, int64_t nsteps,
                              int64_t checkpoint_every, void *stream, sbg_tape *out);

/* Runs the adjoint over the recorded steps: segments are taken last to first,
 * the states of a segment are recomputed from its checkpoint into a buffer of
 * K - 1 states (allocated on the first call; each recompute step writes the
 * next buffer, nothing is copied), and K adjoint steps run over them.
 * lam: in: dL/du^N (values on held voxels are ignored: set to 0); out:
 * dL/du^0 (0 on held and inactive voxels); same grid, dtype and species as
 * the recorded state.  grad (host, 3 doubles):
 *   grad[0] = dL/dD_0, grad[1] = dL/dD_1 (0 with one species),
 *   grad[2] = dL/dk_surf (also at k_surf = 0: the first-order effect of a
 *             surface sink on the loss),
 * accumulated over steps and voxels: FP64 tapes in FP64; SBG_F32 tapes (run
 * by the pipelined kernel) in double-float pairs per thread and warp and FP64
 * per CTA; each CTA adds to its own slot and the slots are summed once in a
 * fixed order.  Synchronises `stream`. */
sbg_status sbg_adjoint(sbg_grid grid, sbg_tape tape, sbg_state lam, double *grad, void *stream);

/* Device memory held by the tape (checkpoints, recompute buffer, work state)
 * and its number of checkpoints; either pointer may be NULL. */
sbg_status sbg_tape_info(sbg_tape tape, int64_t *device_bytes, int64_t *n_checkpoints);
void sbg_tape_destroy(sbg_tape tape);

/* ---- level set: Sussman redistancing --------------------------------------------- */

typedef struct {
    double cfl;               /* dalpha = cfl * min(dx); cfl * min(dx) * sum_a 1/dx_a <= 1      */
    int64_t max_iter;         /* iterations at most                                            */
    double tol;               /* stop at a test where max |sigma (1 - G)| over voxels with
                                 |phi| < band * min(dx) is below tol (<= 0: run max_iter)       */
    double band;              /* half-width of that test's band, in units of min(dx); > 0       */
    int32_t check_every;      /* iterations between tests (the last iteration always tests)     */
} sbg_redist_opts;

/* Sussman redistancing (Sec. 2.1): drives phi towards the signed distance to
 * its zero level set as the steady state of
 *   d phi / d alpha = sigma(phi) (1 - |grad phi|),
 *   sigma(phi) = phi / sqrt(phi^2 + |grad phi|^2 h^2),  h = min(dx),
 * by forward Euler in alpha with first-order upwind (Godunov) differences for
 * the sign of phi at each voxel, every voxel from the previous iterate, a
 * neighbour beyond the box taking the voxel's own value.  phi = 0 stays 0
 * and no voxel changes sign.  phi_in / phi_out: dense [Nz][Ny][Nx] of dtype
 * (SBG_F32 or SBG_F64; the arithmetic is in that precision), both host
 * (on_device 0; distinct arrays) or both device (on_device 1; may be the same
 * array).  iters_out, residual_out (host, may be NULL): iterations run and
 * the last tested max |sigma (1 - G)| (NaN when none ran).  The field lives
 * dense on the device with one ping-pong copy; one stencil pass per
 * iteration.  Synchronises `stream`.  Errors: SBG_ERR_INVALID_ARG (dims
 * outside [1, 2^20], Ny > 524280, Nz > 1048560, dx <= 0, bad options or
 * cfl), SBG_ERR_CUDA. */
sbg_status sbg_redistance(const int64_t dims[3], const double dx[3], const void *phi_in, void *phi_out,
                          int32_t dtype, int32_t on_device, const sbg_redist_opts *opts, int64_t *iters_out,
                          double *residual_out, void *stream);

/* ---- slab decomposition along x (Sec. 2.4: domain decomposition with ghost
 * layers; the multi-GPU runs of Sec. 3.6) ------------------------------------
 * A rank holds the sub-box of its slab of x planes plus one ghost plane on
 * each side where another slab lies; it holds the ghost planes fixed in its
 * steps (Dirichlet faces of its sub-box) and overwrites them after every step
 * with the neighbour's first or last owned plane, so every owned voxel gets
 * exactly its whole-box update.  The library provides the partition and the
 * plane transfers; the exchange pattern and the transport are the caller's
 * (the binding's slab module).
 *
 * sbg_slab_partition: x_bounds[0..nparts] (host, nparts + 1 entries) with
 * x_bounds[0] = 0, x_bounds[nparts] = Nx and interior bounds on block
 * boundaries (multiples of `block`), so that slab k = [x_bounds[k],
 * x_bounds[k+1]) holds about 1/nparts of the active blocks (blocks with a
 * voxel phi > eps_mask, 0 selecting FLT_EPSILON) and at least one block
 * column.  phi: dense FP32 [Nz][Ny][Nx] on the host.  Host code.  Errors:
 * SBG_ERR_INVALID_ARG for null pointers, block not 4/8, dims < 1, nparts < 1
 * or more than the block columns. */
sbg_status sbg_slab_partition(const float *phi, const int64_t dims[3], int32_t block, float eps_mask,
                              int32_t nparts, int64_t *x_bounds);

/* One x plane of species `species` of geometry `geom` between the state and a
 * dense [Nz][Ny] buffer (host or device per on_device; its dtype must be the
 * state's: SBG_F32 or SBG_F64 states only).  get writes the values of the
 * active voxels of plane x and 0 elsewhere; set writes the active voxels of
 * plane x from the buffer and leaves every other slot as it is.  Enqueued on
 * `stream`; with a host buffer the call copies through a temporary device
 * buffer and synchronises `stream`.  Errors: SBG_ERR_INVALID_ARG (null
 * pointers, bad geometry, species or x, other state types or dtypes). */
sbg_status sbg_state_get_xplane(sbg_grid grid, sbg_state state, int32_t geom, int32_t species, int64_t x,
                                void *plane, int32_t plane_dtype, int32_t on_device, void *stream);
sbg_status sbg_state_set_xplane(sbg_grid grid, sbg_state state, int32_t geom, int32_t species, int64_t x,
                                const void *plane, int32_t plane_dtype, int32_t on_device, void *stream);

/* ---- test hooks (no counterpart in the paper) ---------------------------------
 * Failure detection is tested without a fault on the device: these hooks make
 * a bounded wait run out or an allocation fail on purpose.
 *
 * sbg_debug_stall_stage: the ring-buffer step kernels (SBG_KERNEL_PIPELINED*,
 * and the adjoint) launched on `grid` after this call never copy the group of
 * blocks `group` (index of the kernel's work unit: 512 voxels for the one-row
 * kernel, 1024 for the two-row kernel), so the wait of the CTA that owns it
 * on that ring stage runs out after `wait_cycles` SM cycles (1 <= wait_cycles
 * <= 2^31; every wait of those kernels uses that bound while the hook is
 * set).  The CTA then records SBG_ERR_TIMEOUT in the grid's device error word,
 * waits (bounded) for its copies in flight and exits; the next synchronising
 * call on the grid (sbg_reduce, sbg_effective_D, ...) returns SBG_ERR_TIMEOUT
 * and clears the word.  The device context stays usable.  group < 0 clears
 * the hook.  Captured step graphs are re-captured after every change. */
sbg_status sbg_debug_stall_stage(sbg_grid grid, int64_t group, int64_t wait_cycles);

/* sbg_debug_fail_alloc: the n-th next device or page-locked host allocation
 * of the library (any entry point, any thread) fails as if the memory were
 * exhausted: the entry point returns SBG_ERR_OOM and must release what it had
 * allocated.  n = 0 disarms.  sbg_debug_live_allocations: the number and
 * total bytes of the library's live allocations (grids, states, tapes,
 * temporaries not yet freed), for a test to check that a failed call leaves
 * nothing behind.  Host-side bookkeeping; no device work. */
sbg_status sbg_debug_fail_alloc(int64_t n);

/* sbg_debug_set_face: overwrites the face-neighbour entry `face` (0..5: -x,
 * +x, -y, +y, -z, +z) of block `block` with `id` and returns the previous
 * entry in *old_id (may be NULL), so that a test can plant an index outside
 * the block list and check that the debug build (libsbg_debug.so) reports
 * SBG_ERR_BOUNDS instead of reading outside the state.  A release build does
 * not check these ids: step a grid with a planted index only with the debug
 * build, and restore the entry afterwards.  Synchronous. */
sbg_status sbg_debug_set_face(sbg_grid grid, int64_t block, int32_t face, int32_t id, int32_t *old_id);
sbg_status sbg_debug_live_allocations(int64_t *count, int64_t *bytes);

/* sbg_debug_wave_plan: the work order of a wavefront launch (SBG_KERNEL_WAVE,
 * SBG_KERNEL_WAVE4) over `nplanes` planes of blocks holding
 * blocks_per_plane[p] blocks, for K steps per launch, a lag of L planes
 * between consecutive steps, rings of R planes and tickets of up to
 * ticket_blocks consecutive blocks of one plane.  Writes up to `capacity`
 * tickets as int32 quadruples (first block, blocks, plane, step 0..K-1) in
 * the order the kernel's CTAs take them, and their number in *count.  Fails
 * with SBG_ERR_INVALID_ARG when K < 1, L < 1, R < L + 2 (some ticket would
 * then wait on a later one) or ticket_blocks outside 1..4096.  Host code only,
 * no device work: it lets a test check on the CPU that every ticket comes
 * after the tickets it waits on (step s-1 on the planes p-1..p+1, step s+1 on
 * the planes p-R-1..p-R+1), which makes the launch deadlock-free.  The kernel
 * uses L = 4, R = 7 and tickets of 32 blocks. */
sbg_status sbg_debug_wave_plan(const int32_t *blocks_per_plane, int32_t nplanes, int32_t K, int32_t L, int32_t R,
                               int32_t ticket_blocks, int32_t *tickets, int64_t capacity, int64_t *count);

/* ---- errors -------------------------------------------------------------------- */
const char *sbg_last_error(void);            /* thread-local; "" when none                      */
const char *sbg_status_string(sbg_status s);
int32_t sbg_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SBG_H */
