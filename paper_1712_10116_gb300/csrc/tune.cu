// tune.cu -- tg_autotune: the leaf size (n_crit of Sec. 2.3) and the launch shapes of the float32
// P2P and M2L kernels, picked by timing FMM evaluations of the caller's own system on this GPU.
//
// The search is a coordinate descent: n_crit first (it changes the tree, hence the balance between
// M2L and P2P work), then the P2P rows per lane and the M2L grid at the chosen n_crit (these change
// launch shapes only, not results).  Each setting is timed with CUDA events on the context's stream.
// Evaluation objective (the caller's particles): one all-from-all evaluation plus, when a fast set is
// given, one kick-pair evaluation; one warm-up round, then the best of two.  Step objective (no
// particles given, a system bound by tg_hhs_init): one rung-0 HOLD step of the bound system after one
// untimed step at the same setting (which sizes the buffers and captures the graph of a batched step);
// the integrator state is saved before the search and put back before every step and at the end.  A
// step holds evaluations of every rung's system, from the whole system down to the deepest rung's few
// particles, so its best leaf size can differ from that of the largest evaluation alone.
#include <algorithm>

#include "tg_common.cuh"

namespace tg {

namespace {

struct TuneRun {
    tg_ctx *c;
    int n;
    const double *pos, *mass;
    const uint8_t *fast;
    double *acc;
    cudaEvent_t e0, e1;
    int timed = 0;
    bool steps = false;   // step objective on the bound system
};

tg_status objective_step(TuneRun &r, double *ms_out)
{
    tg_ctx *c = r.c;
    tg_status st;
    if ((st = hhs_load(c, B_TUNE_SNAP)) || (st = hhs_step(c)) || (st = hhs_load(c, B_TUNE_SNAP))) return st;
    cudaEventRecord(r.e0, c->stream);
    if ((st = hhs_step(c))) return st;
    cudaEventRecord(r.e1, c->stream);
    if ((st = cuda_check(c, cudaEventSynchronize(r.e1), "autotune timing"))) return st;
    float ms = 0.f;
    if ((st = cuda_check(c, cudaEventElapsedTime(&ms, r.e0, r.e1), "autotune timing"))) return st;
    r.timed += 1;
    *ms_out = ms;
    return TG_OK;
}

tg_status objective(TuneRun &r, double *ms_out)
{
    if (r.steps) return objective_step(r, ms_out);
    tg_ctx *c = r.c;
    tg_status st;
    double best = 1e300;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(r.e0, c->stream);
        if ((st = fmm_eval(c, r.n, r.pos, r.n, nullptr, r.mass, nullptr, r.acc, r.n, nullptr, false))) return st;
        if (r.fast && (st = fmm_eval(c, r.n, r.pos, r.n, nullptr, r.mass, r.fast, r.acc, r.n, nullptr, false)))
            return st;
        cudaEventRecord(r.e1, c->stream);
        if ((st = cuda_check(c, cudaEventSynchronize(r.e1), "autotune timing"))) return st;
        float ms = 0.f;
        if ((st = cuda_check(c, cudaEventElapsedTime(&ms, r.e0, r.e1), "autotune timing"))) return st;
        if (rep > 0) best = std::min(best, (double)ms);   // rep 0 warms up buffers and caches
    }
    r.timed += 1;
    *ms_out = best;
    return TG_OK;
}

}  // namespace

tg_status autotune(tg_ctx *c, int n, const double *pos, const double *mass, const uint8_t *fast, tg_tuning *out)
{
    tg_status st;
    TuneRun r{c, n, pos, mass, fast, nullptr, nullptr, nullptr, 0, pos == nullptr};
    const double time0 = c->hhs_time;
    if (r.steps) {
        if ((st = hhs_save(c, B_TUNE_SNAP))) return st;
    } else if ((st = ensure_t(c, B_TUNE_ACC, (size_t)3 * n, &r.acc))) {
        return st;
    }
    if (cudaEventCreate(&r.e0) != cudaSuccess || cudaEventCreate(&r.e1) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, TG_ERR_CUDA, "autotune: cannot create events");
    }
    // the tuning evaluations are not the caller's work: counters and event timing are left as they were
    const tg_stats stats0 = c->stats;
    unsigned long long dev0[12];
    if ((st = cuda_check(c, cudaMemcpy(dev0, c->d_counters, sizeof dev0, cudaMemcpyDeviceToHost), "autotune"))) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
        return st;
    }
    const int prof0 = c->prof_level;
    c->prof_level = 0;
    const tg_params prm0 = c->prm;
    const tg_tuning tune0 = c->tune;
    auto finish = [&](tg_status s) {
        const int64_t regrow = c->stats.list_regrowths, syncs = c->stats.host_syncs;
        c->stats = stats0;
        c->stats.list_regrowths = regrow;
        c->stats.host_syncs = syncs;
        c->prof_level = prof0;
        if (r.steps) {
            // the bound system as it was before the search (also after a failed step)
            const tg_status sl = hhs_load(c, B_TUNE_SNAP);
            if (!s) s = sl;
            c->hhs_time = time0;
        }
        cudaStreamSynchronize(c->stream);
        cudaMemcpy(c->d_counters, dev0, sizeof dev0, cudaMemcpyHostToDevice);
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
        if (s) {
            c->prm = prm0;
            c->tune = tune0;
        }
        return s;
    };
    double initial = 0.0, best = 0.0;
    if ((st = objective(r, &initial))) return finish(st);
    best = initial;
    tg_tuning choice = c->tune;
    choice.n_crit = c->prm.n_crit;
    const int ncrit_cand[] = {48, 64, 80, 96, 112, 128, 160, 192};
    for (int nc : ncrit_cand) {
        if (nc == prm0.n_crit) continue;
        c->prm.n_crit = nc;
        double ms;
        if ((st = objective(r, &ms))) return finish(st);
        if (ms < best) {
            best = ms;
            choice.n_crit = nc;
        }
    }
    c->prm.n_crit = choice.n_crit;
    if (c->prm.precision == TG_PREC_FP32) {
        // the objective at the chosen n_crit with the current shapes, then the other shapes
        if ((st = objective(r, &best))) return finish(st);
        const int rows_cand[] = {1, 2, 3};
        const int rows0 = choice.p2p_rows;   // timed already
        for (int rows : rows_cand) {
            if (rows == rows0) continue;
            c->tune.p2p_rows = rows;
            double ms;
            if ((st = objective(r, &ms))) return finish(st);
            if (ms < best) {
                best = ms;
                choice.p2p_rows = rows;
            }
        }
        c->tune.p2p_rows = choice.p2p_rows;
        const int grid_cand[] = {4, 8, 16, 32};
        const int grid0 = choice.m2l_blocks_per_sm;
        for (int g : grid_cand) {
            if (g == grid0) continue;
            c->tune.m2l_blocks_per_sm = g;
            double ms;
            if ((st = objective(r, &ms))) return finish(st);
            if (ms < best) {
                best = ms;
                choice.m2l_blocks_per_sm = g;
            }
        }
        c->tune.m2l_blocks_per_sm = choice.m2l_blocks_per_sm;
        if (c->prm.kernel == TG_KERNEL_WENDLAND_C2 && c->prm.p <= 6) {
            // the mutual and the directed form of the harmonic M2L
            const int form0 = choice.m2l_form;
            for (int form = 0; form <= 1; ++form) {
                if (form == form0) continue;
                c->tune.m2l_form = form;
                double ms;
                if ((st = objective(r, &ms))) return finish(st);
                if (ms < best) {
                    best = ms;
                    choice.m2l_form = form;
                }
            }
            c->tune.m2l_form = choice.m2l_form;
        }
    }
    choice.candidates = r.timed;
    choice.objective_ms = best;
    choice.objective_ms_initial = initial;
    c->tune = choice;
    c->tune.n_crit = c->prm.n_crit;
    if (out) *out = c->tune;
    return finish(TG_OK);
}

}  // namespace tg
