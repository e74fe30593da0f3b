// Wavefront step kernel (SBG_KERNEL_WAVE / SBG_KERNEL_WAVE4): K forward-Euler
// steps per launch of the streaming kernel's states (temporal blocking over
// the planes of blocks).
//
// A step of the streaming kernel reads every slot of the state from HBM once
// and writes it once (16 B per slot for two species), so its speed is that of
// HBM.  Step n+1 of a plane of blocks needs step n only on that plane and the
// planes beside it, so one launch can run step n+1 on plane p while step n+2
// runs on plane p - L, step n+3 on p - 2L, ...: the intermediate states live
// in rings of R planes (a few MB each), which stay in the 126 MB L2, and only
// the first step's input and the last step's output move through HBM.  The
// per-voxel arithmetic and the rows each thread reads are the streaming
// kernel's, so results are bitwise those of K streaming steps (tested).
//
// Work is cut into tickets: a group of up to 16 blocks of one plane (plane =
// one layer of blocks of a plane-ordered grid) at one stage (the s-th of the
// K steps).  Stage s reads the state of stage s - 1 (stage 0: the input
// buffer) and writes ring s (stage K-1: the output buffer).  A ticket waits
//  - at stage s > 0 on plane p: until stage s-1 is done on planes p-1..p+1
//    (the ring planes it reads);
//  - at stage s < K-1 on plane p: until stage s+1 is done on planes
//    p-R-1..p-R+1, the readers of the ring slot it overwrites (plane p-R).
// Tickets are numbered round by round: round i holds stage s on plane
// i - s*L for s = 0..K-1, so with L >= 1 and R >= L + 2 every ticket a
// ticket waits on has a smaller number (checked on the host for every
// plan).  Each CTA has one scheduler warp and eight compute warps.  The
// scheduler takes ticket numbers from a global counter, waits until the
// tickets it depends on are published, and hands the ticket to the compute
// warps through a ring of kWaveSlots shared-memory slots (an mbarrier per
// slot that the scheduler arrives on once the slot is written, and one the
// compute warps arrive on when they are done with it).  It publishes a
// ticket (a fence, then an atomic add on the counter of its step and plane)
// as soon as the compute warps are done with it, also while it waits on the
// dependencies of a later ticket; so while the compute warps work through
// one ticket, the next is being resolved, and a ticket that depends on the
// CTA's own previous ticket still makes progress.  The smallest unpublished
// ticket never waits on an unpublished one, so the launch makes progress
// whatever number of CTAs is resident.  Publication is a release (the
// compute warps' stores, their mbarrier arrive, the scheduler's wait on it,
// a gpu-scope fence, the atomic) and the scheduler's polls of the counters
// are followed by a fence before it arrives on the slot's barrier (acquire).
// Every wait is bounded (wait_cycles SM cycles): one that runs out records
// SBG_ERR_TIMEOUT in the grid's error word and raises the launch's abort
// flag, on which every other wait gives up at once; the last CTA to leave
// clears the counters for the next launch.
#include <algorithm>
#include <vector>

#include "sbg_ptx.cuh"
#include "sbg_row.cuh"

namespace sbg {

constexpr int kWaveComputeWarps = 8;                       // 16 blocks x 16 rows
constexpr int kWaveThreads = 32 * (kWaveComputeWarps + 1);  // warp 0 schedules
#ifndef SBG_WAVE_SLOTS
#define SBG_WAVE_SLOTS 4
#endif
constexpr int kWaveSlots = SBG_WAVE_SLOTS;
#ifndef SBG_WAVE_TICKET
#define SBG_WAVE_TICKET 32
#endif
constexpr int kWaveTicketBlocks = SBG_WAVE_TICKET;  // blocks per ticket (passes of 16)
constexpr int kWaveCtrHead = 4;  // ticket counter, CTAs gone, abort flag, unused

__device__ __forceinline__ int ld_relaxed_gpu(const int *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Loads of the ticket's source: the input buffer does not change during the
// launch (read-only path); a ring does, so its rows go through the coherent
// path (L1 lines from before the acquire fence are not used).
template <bool NC>
__device__ __forceinline__ float4 wld4(const float *p) {
    if (NC) return __ldg(reinterpret_cast<const float4 *>(p));
    return __ldca(reinterpret_cast<const float4 *>(p));
}
template <bool NC>
__device__ __forceinline__ float wld1(const float *p) {
    if (NC) return __ldg(p);
    return __ldca(p);
}

struct WaveArgs {
    const int4 *tick;   // [T]: first block, blocks in the group, plane, stage
    const int4 *plane;  // [nplanes]: first block, groups, ring shift, blocks
    int *ctr;           // [kWaveCtrHead + K * nplanes]: all 0 between launches
    float *ring;        // rings, stage-major then species, ring_elems floats each; ring block r of a ring
    int64_t ring_elems; // at 64 + r * 64 from its start (a ghost block of sentinels first)
    int T, nplanes, R;
};

// One ticket: the rows of up to 16 blocks of one plane, one step.  src[s]
// points at the ghost block of species s's source; a block b of plane q is
// block b + shift(q) there (shifts 0 for the input buffer).  dst[s] points at
// block 0 of the destination, where block b is block b + dsh.
template <int NS, bool REACT, bool HELD, bool NC>
__device__ __forceinline__ void wave_group(const StepArgs &a, const int2 *__restrict__ wmeta,
                                           const float4 *__restrict__ wrow, float negzero, const float *const *src,
                                           float *const *dst, int b0, int nblk, int sh_m, int sh_0, int sh_p,
                                           int dsh, int n_wrows, int t) {
    const int j = t >> 4, rr = t & 15, y = rr & 3, z = rr >> 2;
    const int nb = (int)a.nb;
    const bool valid = j < nblk;
    const int b = b0 + j;
    int f[4] = {-1, -1, -1, -1};
    int woff = 0;
    uint32_t wmask = 0, held = 0;
    if (valid) {
        const int32_t *fp = a.face + (int64_t)b * 6;
        f[0] = __ldg(fp + 0);
        f[1] = __ldg(fp + 1);
        f[2] = (y == 0) ? __ldg(fp + 2) : (y == 3) ? __ldg(fp + 3) : -1;
        f[3] = (z == 0) ? __ldg(fp + 4) : (z == 3) ? __ldg(fp + 5) : -1;
        if (REACT) {
            const int2 wm = __ldg(wmeta + b);
            woff = wm.x;
            wmask = (uint32_t)wm.y;
        }
        if (HELD) held = (uint32_t)(__ldg(a.heldbits + b) >> (rr * 4)) & 0xFu;
#if SBG_DEBUG
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (f[k] < -1 || f[k] >= nb) {
                atomicExch(a.err, (int)SBG_ERR_BOUNDS);
                f[k] = -1;
            }
#endif
    }
    (void)nb;
    // x and y neighbours lie in this plane, the z neighbour in the plane below (z = 0) or above (z = 3)
    const int shz = z == 0 ? sh_m : sh_p;
    const int fx0 = f[0] < 0 ? -1 : f[0] + sh_0;
    const int fx1 = f[1] < 0 ? -1 : f[1] + sh_0;
    const int fy = f[2] < 0 ? -1 : f[2] + sh_0;
    const int fz = f[3] < 0 ? -1 : f[3] + shz;
    const int row = valid ? (b + sh_0 + 1) * 64 + rr * 4 : rr * 4;
    const int o_xm = fx0 * 64 + 64 + rr * 4 + 3;
    const int o_xp = fx1 * 64 + 64 + rr * 4;
    const int o_ym = y > 0 ? row - 4 : fy * 64 + 64 + rr * 4 + 12;
    const int o_yp = y < 3 ? row + 4 : fy * 64 + 64 + rr * 4 - 12;
    const int o_zm = z > 0 ? row - 16 : fz * 64 + 64 + rr * 4 + 48;
    const int o_zp = z < 3 ? row + 16 : fz * 64 + 64 + rr * 4 - 48;
    float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (REACT && valid && ((wmask >> rr) & 1u)) {
        const int wi = woff + __popc(wmask & ((1u << rr) - 1u));
#if SBG_DEBUG
        if (wi < 0 || wi >= n_wrows) atomicExch(a.err, (int)SBG_ERR_BOUNDS);
        else
#endif
            w4 = __ldg(wrow + wi);
    }
    (void)n_wrows;
    uint32_t keep[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) keep[i] = ((held >> i) & 1u) ? ~0u : 0u;
    f32x2 tr01 = 0ull, tr23 = 0ull;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const float *q = src[s];
        const float4 c = wld4<NC>(q + row);
        const float4 ym = wld4<NC>(q + o_ym), yp = wld4<NC>(q + o_yp);
        const float4 zm = wld4<NC>(q + o_zm), zp = wld4<NC>(q + o_zp);
        const float xm = wld1<NC>(q + o_xm), xp = wld1<NC>(q + o_xp);
        if (s == 0 && REACT) {
            const f32x2 k2 = pk(a.cf.k, a.cf.k);
            tr01 = mul2(mul2(k2, pk(w4.x, w4.y)), pk(c.x, c.y));
            tr23 = mul2(mul2(k2, pk(w4.z, w4.w)), pk(c.z, c.w));
        }
        float ta, tb, tc, td;
        upk(tr01, ta, tb);
        upk(tr23, tc, td);
        const f32x2 t01 = s == 0 ? (REACT ? pk(-ta, -tb) : pk(negzero, negzero)) : tr01;
        const f32x2 t23 = s == 0 ? (REACT ? pk(-tc, -td) : pk(negzero, negzero)) : tr23;
        const float4 r = row_update(c, xm, xp, ym, yp, zm, zp, a.cf.c[s], a.cf.dt, a.cf.decay[s], t01, t23, keep);
        if (valid) *reinterpret_cast<float4 *>(dst[s] + (int64_t)(b + dsh) * 64 + rr * 4) = r;
    }
}

__device__ __forceinline__ void mbar_arrive1(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

template <int NS, bool REACT, bool HELD, int K, int MINB>
__global__ void __launch_bounds__(kWaveThreads, MINB)
k_step_wave(const StepArgs a, const WaveArgs w, const int2 *__restrict__ wmeta, const float4 *__restrict__ wrow,
            float negzero, int n_wrows) {
    // slot: first block, blocks, plane, step (-1: stop), source shifts of planes p-1, p, p+1, destination shift
    __shared__ __align__(16) int slot[kWaveSlots][8];
    __shared__ __align__(8) uint64_t full[kWaveSlots], freed[kWaveSlots];
    __shared__ int s_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int *const done = w.ctr + kWaveCtrHead;
    int *const abort_flag = w.ctr + 2;
    if (threadIdx.x == 0) {
        for (int q = 0; q < kWaveSlots; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&freed[q], kWaveComputeWarps);
        }
    }
    __syncthreads();
    if (warp == 0) {
        // ---- scheduler (every lane runs the same control flow; lane 0's values decide) ----
        const unsigned FULL = 0xffffffffu;
        const int4 kStop = make_int4(0, 0, 0, -1);
        // tickets: t0 (being prepared, its entry tk0 loaded), t1 (entry tk1 in flight in lane 0), t2 (number
        // in flight in lane 0)
        int t0 = 0, t1 = 0, t2 = 0;
        if (lane == 0) {
            t0 = atomicAdd(w.ctr, 1);
            t1 = atomicAdd(w.ctr, 1);
            t2 = atomicAdd(w.ctr, 1);
        }
        int4 tk0 = kStop, tk1 = kStop;
        if (lane == 0) {
            if (t0 < w.T) tk0 = __ldg(w.tick + t0);
            if (t1 < w.T) tk1 = __ldg(w.tick + t1);
        }
        t0 = __shfl_sync(FULL, t0, 0);
        int fl_t[kWaveSlots], fl_i[kWaveSlots];  // in-flight tickets: number, counter index
        int pub = 0;    // sequence number of the oldest unpublished ticket
        int ready = 0;  // tickets pub .. ready-1: the compute warps are done with them, not yet published
        // counts the in-flight tickets the compute warps are done with (mbarrier waits: acquire.cta)
        auto collect = [&](int k) {
            for (;;) {
                if (ready >= k) return;
                const int q = ready % kWaveSlots;
                const int r = mbar_try_wait(&freed[q], (uint32_t)((ready / kWaveSlots) & 1)) ? 1 : 0;
                if (!__shfl_sync(FULL, r, 0)) return;
                ++ready;
            }
        };
        // publishes them; a gpu-scope fence must separate the collect from the atomics (release)
        auto publish = [&]() {
            for (; pub < ready; ++pub) {
                const int q = pub % kWaveSlots;
                int ft = 0, fi = 0;
#pragma unroll
                for (int i = 0; i < kWaveSlots; ++i)
                    if (i == q) {
                        ft = fl_t[i];
                        fi = fl_i[i];
                    }
                if (lane == 0 && ft != a.stall_group) atomicAdd(done + fi, 1);
            }
        };
        auto expired = [&](long long c0) -> bool {
            const int e = (clock64() - c0 > a.wait_cycles) ? 1 : 0;
            return __shfl_sync(FULL, e, 0) != 0;
        };
        auto fail = [&]() {
            if (lane == 0) {
                atomicExch(a.err, (int)SBG_ERR_TIMEOUT);
                atomicExch(abort_flag, 1);
            }
        };
        bool stop = false;
        int k = 0;
        for (;; ++k) {
            const int q = k % kWaveSlots;
            // the slot's previous ticket (k - kWaveSlots) must be done and published
            if (k >= kWaveSlots) {
                const long long c0 = clock64();
                while (pub <= k - kWaveSlots) {
                    collect(k);
                    if (ready > pub) {
                        fence_acq_rel_gpu();
                        publish();
                    } else if (expired(c0)) {
                        stop = true;
                        break;
                    } else {
                        __nanosleep(32);
                    }
                }
                if (stop) {  // the slot is not free: leave without writing it
                    fail();
                    break;
                }
            }
            tk0.x = __shfl_sync(FULL, tk0.x, 0);
            tk0.y = __shfl_sync(FULL, tk0.y, 0);
            tk0.z = __shfl_sync(FULL, tk0.z, 0);
            tk0.w = __shfl_sync(FULL, tk0.w, 0);
            const int p = tk0.z, st = tk0.w;
            bool timed_out = false;
            int sh = 0;
            if (st >= 0) {
                // lanes 0..2: step st-1 on planes p-1..p+1; lanes 3..5: step st+1 on planes p-R-1..p-R+1;
                // lanes 6..8: the ring shifts of planes p-1..p+1
                int idx = -1, target = 0, pq = -1;
                if (lane < 3 && st > 0) {
                    pq = p - 1 + lane;
                    if (pq >= 0 && pq < w.nplanes) idx = (st - 1) * w.nplanes + pq;
                } else if (lane >= 3 && lane < 6 && st < K - 1) {
                    pq = p - w.R - 1 + (lane - 3);
                    if (pq >= 0) idx = (st + 1) * w.nplanes + pq;
                } else if (lane >= 6 && lane < 9) {
                    const int ps = p - 1 + (lane - 6);
                    if (ps >= 0 && ps < w.nplanes) sh = __ldg(&w.plane[ps].z);
                }
                int val = 0;
                if (idx >= 0) {
                    target = __ldg(&w.plane[pq].y);
                    val = ld_relaxed_gpu(done + idx);
                }
                collect(k);
                if (!__all_sync(FULL, idx < 0 || val >= target)) {
                    // not yet: publish what is done (a ticket may wait on its own CTA's previous one), poll again
                    const long long c0 = clock64();
                    for (;;) {
                        if (ready > pub) {
                            fence_acq_rel_gpu();
                            publish();
                        }
                        __nanosleep(32);
                        const bool ok = idx < 0 || ld_relaxed_gpu(done + idx) >= target;
                        if (__all_sync(FULL, ok)) break;
                        collect(k);
                        const int ab = lane == 0 ? ld_relaxed_gpu(abort_flag) : 0;
                        if (__shfl_sync(FULL, ab, 0)) {
                            stop = true;
                            break;
                        }
                        if (expired(c0)) {
                            timed_out = true;
                            break;
                        }
                    }
                }
            }
            if (timed_out) fail();
            if (stop || timed_out || st < 0) {
                stop = stop || timed_out;
                if (lane == 0) {  // the slot is free (checked above): tell the compute warps to leave
                    slot[q][3] = -1;
                    mbar_arrive1(&full[q]);
                }
                break;
            }
            // one fence: acquire for the counters polled above (the ring rows of those tickets), release for
            // the stores of the tickets collected before it
            fence_acq_rel_gpu();
            publish();
            const int shm = __shfl_sync(FULL, sh, 6), sh0 = __shfl_sync(FULL, sh, 7),
                      shp = __shfl_sync(FULL, sh, 8);
            if (lane == 0) {
                slot[q][0] = tk0.x;
                slot[q][1] = tk0.y;
                slot[q][2] = p;
                slot[q][3] = st;
                slot[q][4] = st == 0 ? 0 : shm;
                slot[q][5] = st == 0 ? 0 : sh0;
                slot[q][6] = st == 0 ? 0 : shp;
                slot[q][7] = st == K - 1 ? 0 : sh0;
                mbar_arrive1(&full[q]);  // release: the slot's contents
            }
            const int tcur = __shfl_sync(FULL, t0, 0);
#pragma unroll
            for (int i = 0; i < kWaveSlots; ++i)
                if (i == q) {
                    fl_t[i] = tcur;
                    fl_i[i] = st * w.nplanes + p;
                }
            // next tickets: t1 becomes t0 (its entry was loaded an iteration ago), t2 becomes t1
            if (lane == 0) {
                t0 = t1;
                tk0 = tk1;
                t1 = t2;
                tk1 = t1 < w.T ? __ldg(w.tick + t1) : kStop;
                t2 = atomicAdd(w.ctr, 1);
            }
        }
        // publish the tickets still in flight (sequence numbers pub .. k-1)
        if (!stop) {
            const long long c0 = clock64();
            while (pub < k) {
                collect(k);
                if (ready > pub) {
                    fence_acq_rel_gpu();
                    publish();
                } else if (expired(c0)) {
                    fail();
                    break;
                } else {
                    __nanosleep(32);
                }
            }
        }
    } else {
        // ---- compute warps: each takes 2 of the 16 blocks of a pass, passes of 16 blocks over the ticket ----
        const int t = threadIdx.x - 32;
        for (int k = 0;; ++k) {
            const int q = k % kWaveSlots;
            if (!mbar_wait_bounded(&full[q], (uint32_t)((k / kWaveSlots) & 1), 4 * a.wait_cycles)) {
                if (lane == 0) {
                    atomicExch(a.err, (int)SBG_ERR_TIMEOUT);
                    atomicExch(abort_flag, 1);
                }
                break;
            }
            int v[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) v[i] = slot[q][i];
            const int stg = v[3];
            if (stg >= 0) {
                const float *src[NS];
                float *dst[NS];
#pragma unroll
                for (int sp = 0; sp < NS; ++sp) {
                    src[sp] = stg == 0 ? (const float *)a.in[sp] - 64
                                       : w.ring + ((int64_t)(stg - 1) * NS + sp) * w.ring_elems;
                    dst[sp] = stg == K - 1 ? (float *)a.out[sp] : w.ring + ((int64_t)stg * NS + sp) * w.ring_elems + 64;
                }
                for (int b0 = 0; b0 < v[1]; b0 += 16) {
                    const int nblk = min(16, v[1] - b0);
                    if (stg == 0)
                        wave_group<NS, REACT, HELD, true>(a, wmeta, wrow, negzero, src, dst, v[0] + b0, nblk, v[4],
                                                          v[5], v[6], v[7], n_wrows, t);
                    else
                        wave_group<NS, REACT, HELD, false>(a, wmeta, wrow, negzero, src, dst, v[0] + b0, nblk, v[4],
                                                           v[5], v[6], v[7], n_wrows, t);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive1(&freed[q]);  // release: this warp's stores of the ticket
            if (stg < 0) break;
        }
    }
    __syncthreads();
    // the last CTA to leave clears the counters for the next launch on the stream
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(w.ctr + 1, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (int i = threadIdx.x; i < K * w.nplanes; i += kWaveThreads) done[i] = 0;
        if (threadIdx.x == 0) {
            w.ctr[0] = 0;
            w.ctr[2] = 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            w.ctr[1] = 0;
        }
    }
}

__global__ void k_fill_sentinel(float *p, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = sentinel_f32();
}

__global__ void k_plane_count(const int4 *__restrict__ blocks, int64_t nb, int *count) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) atomicAdd(count + blocks[b].z, 1);
}

bool wave_plan_tickets(const std::vector<int> &blocks_per_plane, int K, int L, int R, int TB,
                       std::vector<int4> &tick, std::vector<int4> &plane, int &maxplane) {
    const int np = (int)blocks_per_plane.size();
    if (K < 1 || L < 1 || R < L + 2 || TB < 1 || TB > 4096) return false;
    plane.assign(np, make_int4(0, 0, 0, 0));
    maxplane = 0;
    int64_t start = 0;
    for (int p = 0; p < np; ++p) {
        const int n = blocks_per_plane[p];
        if (n < 0) return false;
        maxplane = std::max(maxplane, n);
        plane[p].x = (int)start;
        plane[p].y = (n + TB - 1) / TB;
        plane[p].w = n;
        start += n;
    }
    if (start + 2 >= (int64_t(1) << 25)) return false;
    for (int p = 0; p < np; ++p) plane[p].z = (p % R) * maxplane - plane[p].x;
    tick.clear();
    for (int it = 0; it < np + (K - 1) * L; ++it)
        for (int s = 0; s < K; ++s) {
            const int p = it - s * L;
            if (p < 0 || p >= np) continue;
            for (int gi = 0; gi < plane[p].y; ++gi)
                tick.push_back(make_int4(plane[p].x + TB * gi, std::min(TB, plane[p].w - TB * gi), p, s));
        }
    // every ticket a ticket waits on must come earlier: last ticket index of (stage, plane)
    std::vector<int64_t> last((size_t)K * std::max(np, 1), -1);
    for (int64_t i = 0; i < (int64_t)tick.size(); ++i) {
        const int p = tick[i].z, s = tick[i].w;
        auto before = [&](int ss, int q) { return q < 0 || q >= np || plane[q].y == 0 || last[(size_t)ss * np + q] >= 0; };
        if (s > 0)
            for (int q = p - 1; q <= p + 1; ++q)
                if (!before(s - 1, q)) return false;
        if (s < K - 1)
            for (int q = p - R - 1; q <= p - R + 1; ++q)
                if (!before(s + 1, q)) return false;
        last[(size_t)s * np + p] = i;
    }
    return true;
}

// Plan of a state's wavefront launches: tickets, plane table, counters and rings.
struct WavePlan {
    int K = 0, L = 0, R = 0, ns = 0, nplanes = 0, maxplane = 0, T = 0;
    int4 *tick = nullptr;
    int4 *plane = nullptr;
    int *ctr = nullptr;
    float *ring = nullptr;  // (K - 1) * ns rings of ring_elems floats, each starting with its ghost block
    size_t ring_elems = 0;
};

// planes between consecutive steps of one launch, and planes per ring (>= lag + 2)
#ifndef SBG_WAVE_LAG
#define SBG_WAVE_LAG 4
#endif
#ifndef SBG_WAVE_RING
#define SBG_WAVE_RING 7
#endif
constexpr int kWaveLag = SBG_WAVE_LAG;
constexpr int kWaveRing = SBG_WAVE_RING;

bool wave_kernel_applies(sbg_grid g, sbg_state st) {
    return st->dtype == SBG_F32 && stream_kernel_applies(g, st) && g->order == SBG_ORDER_PLANES && g->n_geoms == 1 &&
           g->nb > 0;
}

void wave_destroy(sbg_state st) {
    WavePlan *w = (WavePlan *)st->wave;
    if (!w) return;
    dfree(w->tick);
    dfree(w->plane);
    dfree(w->ctr);
    dfree(w->ring);
    delete w;
    st->wave = nullptr;
}

sbg_status prepare_wave(sbg_grid g, sbg_state st, int K, cudaStream_t s) {
    WavePlan *old = (WavePlan *)st->wave;
    if (old && old->K == K && old->ns == st->ns) return SBG_OK;
    wave_destroy(st);
    const int nplanes = (int)((g->dims[2] + g->B - 1) / g->B);
    int *dcount = nullptr;
    SBG_CUDA(dmalloc((void **)&dcount, sizeof(int) * std::max(nplanes, 1)));
    std::vector<int> counts(nplanes, 0);
    cudaError_t e = cudaMemsetAsync(dcount, 0, sizeof(int) * nplanes, s);
    if (e == cudaSuccess) {
        k_plane_count<<<(unsigned)((g->nb + 255) / 256), 256, 0, s>>>(g->blocks, g->nb, dcount);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts.data(), dcount, sizeof(int) * nplanes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dfree(dcount);
    if (e != cudaSuccess) return cuda_fail(e, "wavefront plan (plane counts)");
    WavePlan *w = new WavePlan();
    w->K = K;
    w->L = kWaveLag;
    w->R = kWaveRing;
    w->ns = st->ns;
    w->nplanes = nplanes;
    std::vector<int4> tick, plane;
    if (!wave_plan_tickets(counts, K, w->L, w->R, kWaveTicketBlocks, tick, plane, w->maxplane) || tick.size() >= (size_t)INT32_MAX) {
        delete w;
        return fail(SBG_ERR_INVALID_ARG, "internal: no valid wavefront ticket order for this grid");
    }
    w->T = (int)tick.size();
    w->ring_elems = ((size_t)(w->R * (int64_t)w->maxplane + 1) * 64 + 63) / 64 * 64;
    const size_t nring = (size_t)(K - 1) * st->ns * w->ring_elems;
    st->wave = w;
    e = dmalloc((void **)&w->tick, sizeof(int4) * std::max<size_t>(tick.size(), 1));
    if (e == cudaSuccess) e = dmalloc((void **)&w->plane, sizeof(int4) * std::max(nplanes, 1));
    if (e == cudaSuccess) e = dmalloc((void **)&w->ctr, sizeof(int) * (kWaveCtrHead + K * nplanes));
    if (e == cudaSuccess && nring) e = dmalloc((void **)&w->ring, sizeof(float) * nring);
    if (e != cudaSuccess) {
        wave_destroy(st);
        return cuda_fail(e, "cudaMalloc (wavefront plan)");
    }
    e = cudaMemcpyAsync(w->tick, tick.data(), sizeof(int4) * tick.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w->plane, plane.data(), sizeof(int4) * nplanes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->ctr, 0, sizeof(int) * (kWaveCtrHead + K * nplanes), s);
    if (e == cudaSuccess && nring) {
        // every ring slot holds the sentinel until written; the ghost blocks keep it
        k_fill_sentinel<<<(unsigned)((nring + 255) / 256), 256, 0, s>>>(w->ring, (int64_t)nring);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        wave_destroy(st);
        return cuda_fail(e, "wavefront plan upload");
    }
    return SBG_OK;
}

template <int NS, bool REACT, bool HELD, int K>
static cudaError_t launch_wave_t(const StepArgs &a, const WaveArgs &w, const int2 *wmeta, const float4 *wrow,
                                 int n_wrows, int ctas_per_sm, cudaStream_t s) {
    constexpr int MINB = 3;
    auto kern = k_step_wave<NS, REACT, HELD, K, MINB>;
    static int occ = -1, nsm = 0;
    if (occ < 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWaveThreads, 0);
        if (occ < 1) occ = 1;
    }
    const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < occ) ? ctas_per_sm : occ;
    int64_t grid = (int64_t)nsm * per_sm;
    if (grid > w.T) grid = w.T;
    if (grid < 1) return cudaSuccess;
    kern<<<(unsigned)grid, kWaveThreads, 0, s>>>(a, w, wmeta, wrow, -0.0f, n_wrows);
    return cudaGetLastError();
}

template <int K>
static cudaError_t launch_wave_k(const StepArgs &a, const WaveArgs &w, sbg_grid g, int ns, bool react,
                                 int ctas_per_sm, cudaStream_t s) {
    const bool held = a.held_mask != 0;
    const int2 *wm = g->wmeta;
    const float4 *wr = g->wrow;
    const int nw = (int)std::min<int64_t>(g->n_wrows, INT32_MAX);
    if (ns == 1) {
        if (react) return held ? launch_wave_t<1, true, true, K>(a, w, wm, wr, nw, ctas_per_sm, s)
                               : launch_wave_t<1, true, false, K>(a, w, wm, wr, nw, ctas_per_sm, s);
        return held ? launch_wave_t<1, false, true, K>(a, w, wm, wr, nw, ctas_per_sm, s)
                    : launch_wave_t<1, false, false, K>(a, w, wm, wr, nw, ctas_per_sm, s);
    }
    if (react) return held ? launch_wave_t<2, true, true, K>(a, w, wm, wr, nw, ctas_per_sm, s)
                           : launch_wave_t<2, true, false, K>(a, w, wm, wr, nw, ctas_per_sm, s);
    return held ? launch_wave_t<2, false, true, K>(a, w, wm, wr, nw, ctas_per_sm, s)
                : launch_wave_t<2, false, false, K>(a, w, wm, wr, nw, ctas_per_sm, s);
}

// K steps from a.in into a.out (prepare_wave(g, st, K) first, outside any capture).
cudaError_t launch_step_wave(const StepArgs &a, sbg_grid g, sbg_state st, bool react, cudaStream_t s) {
    const WavePlan *p = (const WavePlan *)st->wave;
    WaveArgs w;
    w.tick = p->tick;
    w.plane = p->plane;
    w.ctr = p->ctr;
    w.ring = p->ring;
    w.ring_elems = (int64_t)p->ring_elems;
    w.T = p->T;
    w.nplanes = p->nplanes;
    w.R = p->R;
    if (p->K == 4) return launch_wave_k<4>(a, w, g, st->ns, react, st->ctas_per_sm, s);
    return launch_wave_k<2>(a, w, g, st->ns, react, st->ctas_per_sm, s);
}

}  // namespace sbg

extern "C" sbg_status sbg_debug_wave_plan(const int32_t *blocks_per_plane, int32_t nplanes, int32_t K, int32_t L,
                                          int32_t R, int32_t ticket_blocks, int32_t *tickets, int64_t capacity,
                                          int64_t *count) {
    if (!blocks_per_plane || nplanes < 1 || !count || capacity < 0 || (capacity > 0 && !tickets))
        return sbg::fail(SBG_ERR_INVALID_ARG, "sbg_debug_wave_plan: null pointer or bad size");
    std::vector<int> counts(blocks_per_plane, blocks_per_plane + nplanes);
    std::vector<int4> tick, plane;
    int maxplane = 0;
    if (!sbg::wave_plan_tickets(counts, K, L, R, ticket_blocks, tick, plane, maxplane))
        return sbg::fail(SBG_ERR_INVALID_ARG, "sbg_debug_wave_plan: no valid ticket order for these K, L, R");
    *count = (int64_t)tick.size();
    for (int64_t i = 0; i < (int64_t)tick.size() && i < capacity; ++i) {
        tickets[4 * i + 0] = tick[i].x;
        tickets[4 * i + 1] = tick[i].y;
        tickets[4 * i + 2] = tick[i].z;
        tickets[4 * i + 3] = tick[i].w;
    }
    return SBG_OK;
}
