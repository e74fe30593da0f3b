// Simulated FRAP (fluorescence recovery after photobleaching, Sec. 3.3): the
// recovery curve of the mass in a bleached box, recorded on the device
// between the steps, and the least-squares fit of a reference (bulk box)
// curve to it over a time scale, whose value is D_eff / D_ref (Eq. 2 then
// gives the tortuosity).
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "sbg_internal.cuh"
#include "sbg_trace.cuh"

namespace sbg {

// piecewise-linear interpolant of (tr, fr) at t (tr strictly increasing,
// tr[0] <= t <= tr[m-1] checked by the caller)
static double interp(const double *tr, const double *fr, int64_t m, double t) {
    if (t <= tr[0]) return fr[0];
    if (t >= tr[m - 1]) return fr[m - 1];
    const int64_t k = (int64_t)(std::upper_bound(tr, tr + m, t) - tr);  // tr[k-1] <= t < tr[k]
    const double w = (t - tr[k - 1]) / (tr[k] - tr[k - 1]);
    return fr[k - 1] + w * (fr[k] - fr[k - 1]);
}

static double rss_at(double s, const double *t, const double *f, int64_t n, const double *tr, const double *fr,
                     int64_t m) {
    double acc = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double d = f[i] - interp(tr, fr, m, s * t[i]);
        acc += d * d;
    }
    return acc;
}

}  // namespace sbg

using namespace sbg;

extern "C" sbg_status sbg_frap_curve(sbg_grid g, sbg_state st, const sbg_params *p, int32_t geom, int32_t species,
                                     const int64_t lo[3], const int64_t hi[3], int64_t steps_per_sample,
                                     int32_t n_samples, double *sums, int64_t *count, void *stream) {
    TraceRange trace_range("sbg_frap_curve");
    sbg_status rc = check_box_args(g, st, geom, species, "sbg_frap_curve");
    if (rc != SBG_OK) return rc;
    if (!p || !lo || !hi || !sums) return fail(SBG_ERR_INVALID_ARG, "sbg_frap_curve: null pointer");
    if (steps_per_sample < 1 || n_samples < 0)
        return fail(SBG_ERR_INVALID_ARG, "sbg_frap_curve: steps_per_sample >= 1 and n_samples >= 0");
    if (st->dtype == SBG_F32X2 && st->ns != 1)
        return fail(SBG_ERR_INVALID_ARG, "sbg_frap_curve: SBG_F32X2 states hold one species");
    rc = validate_params(g, p, st->ns);
    if (rc != SBG_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nrec = (size_t)n_samples + 1;
    double *rec = nullptr;
    SBG_CUDA(dmalloc_async((void **)(void **)&rec, 2 * sizeof(double) * nrec, s));
    for (size_t i = 0; i < nrec && rc == SBG_OK; ++i) {
        if (i > 0) rc = step_n(g, st, p, steps_per_sample, s);
        if (rc == SBG_OK) rc = launch_box_sum(g, st, geom, species, lo, hi, rec + 2 * i, s);
    }
    std::vector<double> host(2 * nrec);
    cudaError_t ce = cudaSuccess;
    if (rc == SBG_OK) ce = cudaMemcpyAsync(host.data(), rec, 2 * sizeof(double) * nrec, cudaMemcpyDeviceToHost, s);
    dfree_async(rec, s);
    cudaError_t se = cudaStreamSynchronize(s);
    if (rc != SBG_OK) return rc;
    if (ce != cudaSuccess) return cuda_fail(ce, "sbg_frap_curve: copy of the curve");
    if (se != cudaSuccess) return cuda_fail(se, "sbg_frap_curve");
    rc = check_device_error(g, s);
    if (rc != SBG_OK) return rc;
    for (size_t i = 0; i < nrec; ++i) sums[i] = host[2 * i];
    if (count) *count = (int64_t)host[1];
    return SBG_OK;
}

extern "C" sbg_status sbg_frap_fit(const double *t, const double *f, int64_t n, const double *t_ref,
                                   const double *f_ref, int64_t m, double s_lo, double s_hi, double *scale,
                                   double *rss) {
    if (!t || !f || !t_ref || !f_ref || !scale) return fail(SBG_ERR_INVALID_ARG, "sbg_frap_fit: null pointer");
    if (n < 1 || m < 2) return fail(SBG_ERR_INVALID_ARG, "sbg_frap_fit: n >= 1 and m >= 2 samples");
    if (!(s_lo > 0.0) || !(s_hi > s_lo) || !isfinite(s_hi))
        return fail(SBG_ERR_INVALID_ARG, "sbg_frap_fit: 0 < s_lo < s_hi finite");
    double tmax = 0.0, tmin = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        if (!isfinite(t[i]) || !isfinite(f[i]) || t[i] < 0.0)
            return fail(SBG_ERR_INVALID_ARG, "sbg_frap_fit: times >= 0 and finite values");
        tmax = std::max(tmax, t[i]);
        tmin = std::min(tmin, t[i]);
    }
    for (int64_t j = 0; j < m; ++j) {
        if (!isfinite(t_ref[j]) || !isfinite(f_ref[j]))
            return fail(SBG_ERR_INVALID_ARG, "sbg_frap_fit: non-finite reference sample");
        if (j > 0 && !(t_ref[j] > t_ref[j - 1]))
            return fail(SBG_ERR_INVALID_ARG, "sbg_frap_fit: reference times must increase strictly");
    }
    if (t_ref[0] > s_lo * tmin || t_ref[m - 1] < s_hi * tmax)
        return fail(SBG_ERR_INVALID_ARG, "sbg_frap_fit: the reference curve must cover [s_lo t_min, s_hi t_max]");
    // coarse scan, then golden-section search inside the best scan interval
    constexpr int kScan = 4000;
    int best = 0;
    double best_r = INFINITY;
    for (int k = 0; k <= kScan; ++k) {
        const double sk = s_lo + (s_hi - s_lo) * k / kScan;
        const double r = rss_at(sk, t, f, n, t_ref, f_ref, m);
        if (r < best_r) {
            best_r = r;
            best = k;
        }
    }
    double a = s_lo + (s_hi - s_lo) * std::max(best - 1, 0) / kScan;
    double b = s_lo + (s_hi - s_lo) * std::min(best + 1, kScan) / kScan;
    const double gr = 0.5 * (sqrt(5.0) - 1.0);
    double c = b - gr * (b - a), d = a + gr * (b - a);
    double fc = rss_at(c, t, f, n, t_ref, f_ref, m), fd = rss_at(d, t, f, n, t_ref, f_ref, m);
    for (int it = 0; it < 200 && (b - a) > 1e-15 * s_hi; ++it) {
        if (fc <= fd) {
            b = d;
            d = c;
            fd = fc;
            c = b - gr * (b - a);
            fc = rss_at(c, t, f, n, t_ref, f_ref, m);
        } else {
            a = c;
            c = d;
            fc = fd;
            d = a + gr * (b - a);
            fd = rss_at(d, t, f, n, t_ref, f_ref, m);
        }
    }
    double sbest = 0.5 * (a + b);
    double rbest = rss_at(sbest, t, f, n, t_ref, f_ref, m);
    const double s_scan = s_lo + (s_hi - s_lo) * best / kScan;
    if (best_r < rbest) {  // a scan point the refinement did not improve on
        sbest = s_scan;
        rbest = best_r;
    }
    *scale = sbest;
    if (rss) *rss = rbest;
    return SBG_OK;
}

extern "C" sbg_status sbg_frap_recovery(sbg_grid g, sbg_state st, const sbg_params *p, int32_t geom,
                                        int32_t species, const int64_t lo[3], const int64_t hi[3],
                                        int64_t steps_per_sample, int32_t n_samples, double *t, double *F,
                                        int64_t *count, void *stream) {
    TraceRange trace_range("sbg_frap_recovery");
    if (!t || !F) return fail(SBG_ERR_INVALID_ARG, "sbg_frap_recovery: null output");
    sbg_status rc = check_box_args(g, st, geom, species, "sbg_frap_recovery");
    if (rc != SBG_OK) return rc;
    if (!p) return fail(SBG_ERR_INVALID_ARG, "sbg_frap_recovery: null params");
    // the equilibrium level: the mean of the species over every active voxel of the
    // geometry (conserved in a closed box), from the state before the first step
    const int64_t all_lo[3] = {0, 0, 0};
    const int64_t all_hi[3] = {g->dims[3 * geom], g->dims[3 * geom + 1], g->dims[3 * geom + 2]};
    double tot[2] = {0.0, 0.0};
    rc = sbg_reduce_box(g, st, geom, species, all_lo, all_hi, tot, stream);
    if (rc != SBG_OK) return rc;
    int64_t n_box = 0;
    rc = sbg_frap_curve(g, st, p, geom, species, lo, hi, steps_per_sample, n_samples, F, &n_box, stream);
    if (rc != SBG_OK) return rc;
    if (count) *count = n_box;
    if (n_box == 0 || tot[1] == 0.0 || tot[0] == 0.0)
        return fail(SBG_ERR_INVALID_ARG, "sbg_frap_recovery: the box holds no active voxel or the field is zero");
    const double level = tot[0] / tot[1] * (double)n_box;  // mean u x active voxels in the box
    for (int32_t i = 0; i <= n_samples; ++i) {
        t[i] = p->dt * (double)steps_per_sample * (double)i;
        F[i] = F[i] / level;
    }
    return SBG_OK;
}

extern "C" sbg_status sbg_frap_effective_D(const double *t, const double *F, int64_t n, const double *t_ref,
                                           const double *F_ref, int64_t m, double D_ref, double s_lo, double s_hi,
                                           double *D_eff, double *tau, double *scale, double *rss) {
    if (!D_eff || !tau) return fail(SBG_ERR_INVALID_ARG, "sbg_frap_effective_D: null output");
    if (!(D_ref > 0.0) || !isfinite(D_ref)) return fail(SBG_ERR_INVALID_ARG, "sbg_frap_effective_D: D_ref > 0");
    double s = 0.0, r = 0.0;
    sbg_status rc = sbg_frap_fit(t, F, n, t_ref, F_ref, m, s_lo, s_hi, &s, &r);
    if (rc != SBG_OK) return rc;
    *D_eff = s * D_ref;                        // the reference curve at s D_ref matches the measured one
    *tau = s > 0.0 ? 1.0 / s : INFINITY;        // tau = D / D_eff (Eq. 2)
    if (scale) *scale = s;
    if (rss) *rss = r;
    return SBG_OK;
}
