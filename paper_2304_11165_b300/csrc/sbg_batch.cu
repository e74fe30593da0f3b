// Batched steady-state solve over many geometries (no counterpart in the
// paper: the batching pattern of this library).
//
// sbg_build_batch concatenates the block lists of all geometries (blocks
// sorted by geometry, each carrying its geometry id; neighbour tables never
// cross geometries).  This driver advances every unconverged geometry with
// ONE persistent pipelined launch per step over a device work list of
// 512-voxel spans that never straddle geometries, replays a captured CUDA
// graph of `check_every` such launches, and after each interval computes every
// active geometry's FP64 residual in one segmented reduction (the records of
// each geometry in a segment of their own, one final kernel over all
// segments, one copy and one synchronisation).  A geometry whose relative residual is
// below tol leaves the work list; its blocks are not touched again, and since
// check_every is even its values stay in the current buffer.
#include <algorithm>
#include <cstring>
#include <vector>

#include "sbg_internal.cuh"
#include "sbg_step.cuh"
#include "sbg_trace.cuh"

namespace sbg {
sbg_status launch_step_work(sbg_grid g, sbg_state st, const sbg_params *p, int src, const int64_t *items,
                            int64_t nitems, cudaStream_t s);
}

using namespace sbg;

extern "C" sbg_status sbg_batch_run_to_steady(sbg_grid g, sbg_state st, const sbg_params *p, double tol,
                                              int64_t check_every, int64_t max_steps, int64_t *steps_done,
                                              double *rel_residual, void *stream) {
    TraceRange trace_range("sbg_batch_run_to_steady");
    if (!g || !st || !p || !steps_done || !rel_residual)
        return fail(SBG_ERR_INVALID_ARG, "sbg_batch_run_to_steady: null pointer");
    if (st->grid != g) return fail(SBG_ERR_INVALID_ARG, "sbg_batch_run_to_steady: state of another grid");
    if (check_every < 2 || max_steps < 0 || !(tol > 0.0))
        return fail(SBG_ERR_INVALID_ARG, "sbg_batch_run_to_steady: check_every >= 2, max_steps >= 0, tol > 0");
    if (st->dtype == SBG_F64) return fail(SBG_ERR_INVALID_ARG, "sbg_batch_run_to_steady: FP32-based states");
    sbg_status rc = validate_params(g, p, st->ns);
    if (rc != SBG_OK) return rc;
    rc = prepare_held_bits(g, p, (cudaStream_t)stream);  // before the step graphs are captured
    if (rc != SBG_OK) return rc;
    check_every += check_every & 1;  // even: parity of the current buffer is kept
    cudaStream_t s = (cudaStream_t)stream;
    const int n = g->n_geoms;
    // work-list spans as large as the step kernel of this state takes
    const int G = step_work_group_voxels(st->dtype, st->ns, g->has_eps, halo_variant_of(st->variant)) / g->b3();
    std::vector<double> r0(n, 0.0), red(kNumRed);
    std::vector<char> active(n, 0);
    for (int i = 0; i < n; ++i) {
        steps_done[i] = 0;
        rel_residual[i] = 0.0;
        if (g->geom_count[i] == 0) continue;
        rc = reduce_species(g, st, p, i, 0, -1, red.data(), s);
        if (rc != SBG_OK) return rc;
        if (red[SBG_RED_NONFINITE] > 0) return fail(SBG_ERR_NONFINITE, "sbg_batch_run_to_steady: non-finite initial state");
        r0[i] = red[SBG_RED_RESIDUAL];
        if (r0[i] > 0.0) {
            active[i] = 1;
            rel_residual[i] = 1.0;
        }
    }
    int64_t max_items = 0;
    for (int i = 0; i < n; ++i) max_items += (g->geom_count[i] + G - 1) / G;
    int64_t *items = nullptr;
    SBG_CUDA(dmalloc((void **)&items, sizeof(int64_t) * 2 * std::max<int64_t>(max_items, 1)));
    // the segmented check: one record segment per geometry, one result row per geometry
    int64_t nrec = 0;
    for (int i = 0; i < n; ++i)
        if (g->geom_count[i] > 0) nrec += reduce_records(g, st, p, i);
    double *records = nullptr, *res_dev = nullptr;
    int *seg_dev = nullptr;
    cudaError_t ae = dmalloc((void **)&records, sizeof(double) * kNumRed * (size_t)std::max<int64_t>(nrec, 1));
    if (ae == cudaSuccess) ae = dmalloc((void **)&res_dev, sizeof(double) * kNumRed * (size_t)std::max(n, 1));
    if (ae == cudaSuccess) ae = dmalloc((void **)&seg_dev, sizeof(int) * 2 * (size_t)std::max(n, 1));
    if (ae != cudaSuccess) {
        dfree(items);
        dfree(records);
        dfree(res_dev);
        dfree(seg_dev);
        return cuda_fail(ae, "cudaMalloc (batch check buffers)");
    }
    std::vector<double> res_host(kNumRed * (size_t)std::max(n, 1));
    std::vector<int> ids;
    std::vector<int64_t> h;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cs = nullptr;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (cs) cudaStreamDestroy(cs);
        dfree(items);
        dfree(records);
        dfree(res_dev);
        dfree(seg_dev);
    };
    auto rebuild = [&]() -> sbg_status {
        h.clear();
        for (int i = 0; i < n; ++i) {
            if (!active[i]) continue;
            const int64_t b0 = g->geom_begin[i], cnt = g->geom_count[i];
            for (int64_t q = 0; q < cnt; q += G) {
                h.push_back(b0 + q);
                h.push_back(std::min<int64_t>(G, cnt - q));
            }
        }
        if (!h.empty())
            SBG_CUDA(cudaMemcpyAsync(items, h.data(), sizeof(int64_t) * h.size(), cudaMemcpyHostToDevice, s));
        SBG_CUDA(cudaStreamSynchronize(s));
        if (exec) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        const int64_t nitems = (int64_t)h.size() / 2;
        if (nitems == 0) return SBG_OK;
        // first call outside capture (no kernel: empty list) sets up launch attributes
        sbg_status r = launch_step_work(g, st, p, st->cur, items, 0, s);
        if (r != SBG_OK) return r;
        if (!cs) SBG_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        SBG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        int src = st->cur;
        for (int64_t k = 0; k < check_every && r == SBG_OK; ++k) {
            r = launch_step_work(g, st, p, src, items, nitems, cs);
            src = 1 - src;
        }
        cudaError_t e = cudaStreamEndCapture(cs, &graph);
        if (r != SBG_OK) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "batch graph capture");
        return SBG_OK;
    };
    rc = rebuild();
    int64_t done = 0;
    while (rc == SBG_OK && !h.empty() && done < max_steps) {
        if (cudaGraphLaunch(exec, s) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "batch graph launch");
            break;
        }
        done += check_every;
        bool changed = false;
        // every unconverged geometry's residual in one segmented reduction (one synchronisation)
        ids.clear();
        for (int i = 0; i < n; ++i)
            if (active[i]) ids.push_back(i);
        rc = reduce_geometries(g, st, p, ids.data(), (int)ids.size(), 0, records, seg_dev, res_dev, res_host.data(),
                               s);
        for (size_t k = 0; k < ids.size() && rc == SBG_OK; ++k) {
            const int i = ids[k];
            const double *r = &res_host[k * kNumRed];
            if (r[SBG_RED_NONFINITE] > 0) {
                rc = fail(SBG_ERR_NONFINITE, "sbg_batch_run_to_steady: non-finite value in geometry " + std::to_string(i));
                break;
            }
            steps_done[i] = done;
            rel_residual[i] = r[SBG_RED_RESIDUAL] / r0[i];
            if (rel_residual[i] < tol) {
                active[i] = 0;
                changed = true;
            }
        }
        if (rc == SBG_OK && changed) rc = rebuild();
    }
    cleanup();
    if (rc != SBG_OK) return rc;
    for (int i = 0; i < n; ++i)
        if (active[i]) return fail(SBG_ERR_NOT_CONVERGED, "sbg_batch_run_to_steady: max_steps reached");
    return SBG_OK;
}
