// sweep.cpp -- the TTC-threshold sweep: collision probability with a 95 %
// Wilson interval at each threshold (aeb_wilson, stats.cpp), pooled over
// scenarios, from batched launches that share one resident parameter block.
#include <cmath>
#include <cstring>
#include <vector>

#include "aeb_internal.h"
#include "host_util.h"

extern "C" aeb_status aeb_ttc_sweep(const aeb_model *model, const aeb_scenario *scenarios,
                                    uint32_t n_scen, uint64_t n_per, const double *thresholds,
                                    uint32_t n_thr, aeb_precision precision,
                                    aeb_sweep_result *per_threshold, aeb_job_stats *per_job,
                                    void *stream)
{
    using namespace aeb;
    clear_error();
    if (!model || !scenarios || !thresholds || !per_threshold || n_scen == 0 || n_thr == 0 ||
        n_per == 0)
        return fail(AEB_EINVAL, "aeb_ttc_sweep: NULL argument or empty sweep");
    for (uint32_t t = 0; t < n_thr; ++t)
        if (!std::isfinite(thresholds[t])) return fail(AEB_EINVAL, "aeb_ttc_sweep: threshold not finite");
    aeb_model m = *model;
    m.trigger = AEB_TRIGGER_TTC;
    ModelDev md;
    aeb_status st = check_model(&m, &md);
    if (st != AEB_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint64_t P = (uint64_t)n_scen * n_per;

    // outputs for `chunk` thresholds at a time: <= 2.0e8 rows (~4.2 GB)
    const uint64_t max_rows = 200'000'000ull;
    uint32_t chunk = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(n_thr, max_rows / P));
    const uint64_t out_rows = (uint64_t)chunk * P;

    std::vector<void *> allocs;
    auto cleanup = [&] {
        for (void *p : allocs) cudaFree(p);
    };
    auto dalloc = [&](size_t bytes, void **p) {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) allocs.push_back(*p);
        return e;
    };
    // parameters: sample on the host (pinned), upload once
    double *hbuf = nullptr;
    cudaError_t e = cudaHostAlloc(&hbuf, sizeof(double) * AEB_NFIELDS * P, cudaHostAllocDefault);
    if (e != cudaSuccess) return cuda_fail(e, "aeb_ttc_sweep: pinned staging");
    void *dpar = nullptr;
    e = dalloc(sizeof(double) * AEB_NFIELDS * P, &dpar);
    if (e != cudaSuccess) {
        cudaFreeHost(hbuf);
        return cuda_fail(e, "aeb_ttc_sweep: parameter buffer");
    }
    aeb_params hp, dp;
    double **hc[AEB_NFIELDS] = {&hp.v0, &hp.d0, &hp.mu, &hp.gs, &hp.gc, &hp.mass, &hp.cd, &hp.tau, &hp.t_delay, &hp.noise};
    double **dc[AEB_NFIELDS] = {&dp.v0, &dp.d0, &dp.mu, &dp.gs, &dp.gc, &dp.mass, &dp.cd, &dp.tau, &dp.t_delay, &dp.noise};
    for (int f = 0; f < AEB_NFIELDS; ++f) {
        *hc[f] = hbuf + (uint64_t)f * P;
        *dc[f] = static_cast<double *>(dpar) + (uint64_t)f * P;
    }
    for (uint32_t sc = 0; sc < n_scen && st == AEB_OK; ++sc) {
        aeb_params part;
        double **pc[AEB_NFIELDS] = {&part.v0, &part.d0, &part.mu, &part.gs, &part.gc, &part.mass, &part.cd, &part.tau, &part.t_delay, &part.noise};
        for (int f = 0; f < AEB_NFIELDS; ++f) *pc[f] = *hc[f] + (uint64_t)sc * n_per;
        st = aeb_sample_params(&m, &scenarios[sc], 0, n_per, &part, 0);
    }
    if (st == AEB_OK) {
        e = cudaMemcpyAsync(dpar, hbuf, sizeof(double) * AEB_NFIELDS * P, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "aeb_ttc_sweep: parameter upload");
    }
    cudaFreeHost(hbuf);
    if (st != AEB_OK) {
        cleanup();
        return st;
    }
    // outputs and per-job statistics of one chunk
    void *dout = nullptr, *dstats = nullptr;
    e = dalloc((1 + 8 + 8 + 4) * out_rows + 4096, &dout);
    if (e == cudaSuccess) e = dalloc(sizeof(aeb_job_stats) * (size_t)chunk * n_scen, &dstats);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "aeb_ttc_sweep: output buffers");
    }
    aeb_outputs out{};
    char *o = static_cast<char *>(dout);
    out.x_ref = reinterpret_cast<double *>(o);
    out.v_imp = reinterpret_cast<double *>(o + 8 * out_rows);
    out.n_steps = reinterpret_cast<int32_t *>(o + 16 * out_rows);
    out.status = reinterpret_cast<uint8_t *>(o + 20 * out_rows);
    std::vector<aeb_job_stats> hstats((size_t)chunk * n_scen);
    std::vector<aeb_job> jobs;
    for (uint32_t t0 = 0; t0 < n_thr && st == AEB_OK; t0 += chunk) {
        const uint32_t nt = std::min(chunk, n_thr - t0);
        jobs.clear();
        for (uint32_t t = 0; t < nt; ++t)
            for (uint32_t sc = 0; sc < n_scen; ++sc)
                jobs.push_back(aeb_job{(uint64_t)sc * n_per, ((uint64_t)t * n_scen + sc) * n_per,
                                       n_per, thresholds[t0 + t], (uint64_t)sc * n_per});
        st = aeb_rollout_batched(&m, jobs.data(), (uint32_t)jobs.size(), &dp, precision, &out,
                                 static_cast<aeb_job_stats *>(dstats), stream);
        if (st != AEB_OK) break;
        e = cudaMemcpy(hstats.data(), dstats, sizeof(aeb_job_stats) * jobs.size(),
                       cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "aeb_ttc_sweep: statistics copy");
            break;
        }
        for (uint32_t t = 0; t < nt; ++t) {
            aeb_sweep_result &r = per_threshold[t0 + t];
            std::memset(&r, 0, sizeof r);
            r.threshold = thresholds[t0 + t];
            for (uint32_t sc = 0; sc < n_scen; ++sc) {
                const aeb_job_stats &j = hstats[(size_t)t * n_scen + sc];
                r.n += j.n;
                r.n_contact += j.n_contact;
                r.n_stop += j.n_stop;
                r.n_horizon += j.n_horizon;
                r.n_invalid += j.n_invalid;
                if (per_job) per_job[(size_t)(t0 + t) * n_scen + sc] = j;
            }
            const uint64_t valid = r.n - r.n_invalid;
            r.p_contact = valid ? (double)r.n_contact / (double)valid : 0.0;
            aeb_wilson(r.n_contact, valid, 1.959963984540054, &r.ci_lo, &r.ci_hi);
        }
    }
    cleanup();
    return st;
}
