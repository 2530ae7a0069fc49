// capi.cu -- the extern "C" entry points declared in include/taichi_gb.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tg_common.cuh"
#include "m2l_sym.cuh"

using namespace tg;

namespace {

tg_status validate(const tg_params *p, std::string &why)
{
    if (!p) {
        why = "params is NULL";
        return TG_ERR_ARG;
    }
    if (p->p < 1 || p->p > kPHigh) why = "p must be in [1, 20]";
    else if (p->n_crit < 1 || p->n_crit > 2 * kMaxNcrit) why = "n_crit must be in [1, 256]";
    else if (p->kernel != TG_KERNEL_WENDLAND_C2 && p->kernel != TG_KERNEL_PLUMMER) why = "unknown kernel";
    else if (p->precision != TG_PREC_FP64 && p->precision != TG_PREC_FP32) why = "unknown precision";
    else if (p->max_level < 1 || p->max_level > kMaxLevel) why = "max_level must be in [1, 21]";
    else if (p->k_max < 0 || p->k_max > 30) why = "k_max must be in [0, 30]";
    else if (!(p->theta > 0.0) || !std::isfinite(p->theta)) why = "theta must be > 0";
    else if (!(p->kappa > 0.0) || !std::isfinite(p->kappa)) why = "kappa must be > 0";
    else if (!(p->eps > 0.0) || !std::isfinite(p->eps)) why = "eps must be > 0";
    else if (!(p->eta > 0.0) || !std::isfinite(p->eta)) why = "eta must be > 0";
    else if (!(p->dt_max > 0.0) || !std::isfinite(p->dt_max)) why = "dt_max must be > 0";
    else if (!(p->eta_tot >= 0.0) || !std::isfinite(p->eta_tot)) why = "eta_tot must be >= 0";
    else if (p->mac != TG_MAC_SIDE && p->mac != TG_MAC_SPHERE) why = "unknown mac";
    else if (p->batched != 0 && p->batched != 1) why = "batched must be 0 or 1";
    else if (p->batched && (p->p < 4 || p->p > 6 || p->mac != TG_MAC_SIDE))
        why = "the batched step needs 4 <= p <= 6 and the side criterion (TG_MAC_SIDE)";
    return why.empty() ? TG_OK : TG_ERR_ARG;
}

tg_status begin(tg_ctx *c)
{
    if (!c) return TG_ERR_ARG;
    c->err = Err{};
    return TG_OK;
}

// Device memory of the current device (managed memory is reachable from any device).  Memory of
// another GPU is refused: the kernels run on the current one.
int check_device_ptr(const void *p)
{
    if (!p) return 0;
    cudaPointerAttributes a;
    int dev = -1;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeManaged) return 1;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" {

tg_status tg_create(const tg_params *params, void *cuda_stream, tg_ctx **out)
{
    if (!out) return TG_ERR_ARG;
    *out = nullptr;
    std::string why;
    tg_status st = validate(params, why);
    if (st) return st;
    tg_ctx *c = new (std::nothrow) tg_ctx();
    if (!c) return TG_ERR_OOM;
    c->prm = *params;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return TG_ERR_CUDA;
    }
    if (cudaMalloc(&c->d_counters, 32 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return TG_ERR_OOM;
    }
    if (cudaMallocHost(&c->h_pinned, 64 * sizeof(int64_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(c->d_counters);
        delete c;
        return TG_ERR_OOM;
    }
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_walk, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (c->side) cudaStreamDestroy(c->side);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->ev_walk) cudaEventDestroy(c->ev_walk);
        cudaFreeHost(c->h_pinned);
        cudaFree(c->d_counters);
        delete c;
        return TG_ERR_CUDA;
    }
    cudaMemset(c->d_counters, 0, 32 * sizeof(unsigned long long));
    std::memset(c->h_pinned, 0, 64 * sizeof(int64_t));
    *out = c;
    return TG_OK;
}

tg_status tg_destroy(tg_ctx *c)
{
    if (!c) return TG_ERR_ARG;
    cudaStreamSynchronize(c->stream);
    if (c->side) cudaStreamSynchronize(c->side);
    hold_graph_destroy(c);
    for (auto &b : c->buf)
        if (b.p) cudaFree(b.p);
    for (cudaEvent_t e : c->prof_events) cudaEventDestroy(e);
    if (c->d_counters) cudaFree(c->d_counters);
    if (c->h_pinned) cudaFreeHost(c->h_pinned);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_walk) cudaEventDestroy(c->ev_walk);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    delete c;
    return TG_OK;
}

const char *tg_last_error(const tg_ctx *c)
{
    if (!c) return "null context";
    return c->err.msg.c_str();
}

tg_status tg_get_stats(const tg_ctx *c, tg_stats *out)
{
    if (!c || !out) return TG_ERR_ARG;
    tg_ctx *m = const_cast<tg_ctx *>(c);
    unsigned long long dev[12] = {0};
    cudaStreamSynchronize(m->stream);
    if (cudaMemcpy(dev, m->d_counters, sizeof dev, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return TG_ERR_CUDA;
    }
    *out = c->stats;
    out->p2p_pairs = (int64_t)dev[0];
    // side contractions counted by the float32 M2L kernels: two per (cell pair, class) with both sides
    out->m2l_class_pairs += (int64_t)(dev[11] / 2);
    return TG_OK;
}

tg_status tg_set_profiling(tg_ctx *c, int level)
{
    if (!c || level < 0 || level > 2) return TG_ERR_ARG;
    prof_collect(c);
    c->prof_level = level;
    return TG_OK;
}

tg_status tg_get_profile(tg_ctx *c, tg_profile *out)
{
    if (!c || !out) return TG_ERR_ARG;
    tg_status st = prof_collect(c);
    if (st) return st;
    for (int k = 0; k < TG_K_COUNT; ++k) {
        out->ms[k] = c->prof_ms[k];
        out->launches[k] = c->prof_launches[k];
    }
    return TG_OK;
}

tg_status tg_reset_stats(tg_ctx *c)
{
    if (!c) return TG_ERR_ARG;
    prof_collect(c);
    for (int k = 0; k < TG_K_COUNT; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_launches[k] = 0;
    }
    c->stats = tg_stats{};
    cudaMemsetAsync(c->d_counters, 0, sizeof(unsigned long long), c->stream);
    cudaMemsetAsync(c->d_counters + 11, 0, sizeof(unsigned long long), c->stream);
    return TG_OK;
}

tg_status tg_build_tree(tg_ctx *c, int64_t n, const double *pos)
{
    tg_status st = begin(c);
    if (st) return st;
    if (n <= 0 || n > INT32_MAX / 4 || !check_device_ptr(pos))
        return set_err(c, TG_ERR_ARG, "tg_build_tree: need n > 0 and a device pointer");
    Geom *g;
    if ((st = ensure_t(c, B_GEOM, 1, &g)) || (st = root_cube(c, (int)n, pos, n, nullptr, g))) return st;
    // masses are not needed for the tree; gather reads a dummy unit array
    double *ones;
    if ((st = ensure_t(c, B_DIAG_POT, n, &ones))) return st;
    cudaMemsetAsync(ones, 0, sizeof(double) * n, c->stream);
    if ((st = keys_sort_gather(c, (int)n, pos, n, nullptr, ones, nullptr, g))) return st;
    int ncell = 0;
    if ((st = build_octree(c, (int)n, &ncell))) return st;
    c->last_n = n;
    c->last_ncell = ncell;
    c->last_nm2l = c->last_np2p = 0;
    return cuda_check(c, cudaStreamSynchronize(c->stream), "tg_build_tree");
}

tg_status tg_fmm_forces(tg_ctx *c, int64_t n, const double *pos, const double *mass, const uint8_t *is_fast,
                        double *acc, double *pot)
{
    tg_status st = begin(c);
    if (st) return st;
    if (n < 0 || n > INT32_MAX / 4) return set_err(c, TG_ERR_ARG, "tg_fmm_forces: n out of range");
    if (n == 0) return TG_OK;
    if (!check_device_ptr(pos) || !check_device_ptr(mass) || !check_device_ptr(acc) ||
        (is_fast && !check_device_ptr(is_fast)) || (pot && !check_device_ptr(pot)))
        return set_err(c, TG_ERR_ARG, "tg_fmm_forces: arrays must be device memory");
    if ((st = check_finite(c, n, pos, n, nullptr, mass))) return st;
    return fmm_eval(c, (int)n, pos, n, nullptr, mass, is_fast, acc, n, pot, true);
}

tg_status tg_direct_forces(tg_ctx *c, int64_t n, const double *pos, const double *mass, const uint8_t *is_fast,
                           int64_t n_sink, const int64_t *sink_idx, double *acc, double *pot)
{
    tg_status st = begin(c);
    if (st) return st;
    if (n < 0 || n_sink < 0 || (sink_idx == nullptr && n_sink > n))
        return set_err(c, TG_ERR_ARG, "tg_direct_forces: bad sizes");
    if (n_sink == 0) return TG_OK;
    if (!check_device_ptr(pos) || !check_device_ptr(mass) || !check_device_ptr(acc) ||
        (sink_idx && !check_device_ptr(sink_idx)) || (is_fast && !check_device_ptr(is_fast)))
        return set_err(c, TG_ERR_ARG, "tg_direct_forces: arrays must be device memory");
    return direct_eval(c, n, pos, mass, is_fast, n_sink, sink_idx, acc, pot);
}

tg_status tg_hhs_init(tg_ctx *c, int64_t n, double *pos, double *vel, const double *mass)
{
    tg_status st = begin(c);
    if (st) return st;
    if (n <= 0 || n > INT32_MAX / 4 || !check_device_ptr(pos) || !check_device_ptr(vel) || !check_device_ptr(mass))
        return set_err(c, TG_ERR_ARG, "tg_hhs_init: need n > 0 and device arrays");
    if ((st = check_finite(c, n, pos, n, nullptr, mass)) || (st = check_finite(c, n, vel, n, nullptr, nullptr)))
        return st;
    c->hhs_n = n;
    c->hhs_pos = pos;
    c->hhs_vel = vel;
    c->hhs_mass = mass;
    c->bound_integrator = 1;
    st = hhs_init(c);
    if (st) {
        c->hhs_n = 0;
        c->bound_integrator = 0;
    }
    return st;
}

tg_status tg_hhs_step(tg_ctx *c)
{
    tg_status st = begin(c);
    if (st) return st;
    if (c->hhs_n <= 0 || c->bound_integrator != 1) return set_err(c, TG_ERR_STATE, "tg_hhs_step before tg_hhs_init");
    return hhs_step(c);
}

tg_status tg_ensemble_step(tg_ctx **cs, int count)
{
    if (!cs || count < 1 || !cs[0]) return TG_ERR_ARG;
    tg_ctx *c0 = cs[0];
    tg_status st = begin(c0);
    if (st) return st;
    for (int i = 0; i < count; ++i) {
        if (!cs[i]) return set_err(c0, TG_ERR_ARG, "tg_ensemble_step: member %d is NULL", i);
        if (cs[i]->hhs_n <= 0 || cs[i]->bound_integrator != 1)
            return set_err(c0, TG_ERR_STATE, "tg_ensemble_step: member %d has no HHS system bound", i);
        if (!cs[i]->prm.batched || cs[i]->stream != c0->stream || cs[i]->device != c0->device)
            return set_err(c0, TG_ERR_ARG, "tg_ensemble_step: member %d is not batched on the first member's stream", i);
        for (int j = 0; j < i; ++j)
            if (cs[j] == cs[i]) return set_err(c0, TG_ERR_ARG, "tg_ensemble_step: member %d appears twice", i);
        cs[i]->err = Err{};
    }
    return ensemble_step(cs, count);
}

tg_status tg_trad_init(tg_ctx *c, int64_t n, double *pos, double *vel, const double *mass)
{
    tg_status st = begin(c);
    if (st) return st;
    if (n <= 0 || n > INT32_MAX / 4 || !check_device_ptr(pos) || !check_device_ptr(vel) || !check_device_ptr(mass))
        return set_err(c, TG_ERR_ARG, "tg_trad_init: need n > 0 and device arrays");
    c->hhs_n = n;
    c->hhs_pos = pos;
    c->hhs_vel = vel;
    c->hhs_mass = mass;
    c->bound_integrator = 2;
    st = trad_init(c);
    if (st) {
        c->hhs_n = 0;
        c->bound_integrator = 0;
    }
    return st;
}

tg_status tg_trad_step(tg_ctx *c)
{
    tg_status st = begin(c);
    if (st) return st;
    if (c->hhs_n <= 0 || c->bound_integrator != 2) return set_err(c, TG_ERR_STATE, "tg_trad_step before tg_trad_init");
    return trad_step(c);
}

tg_status tg_hhs_state(tg_ctx *c, int32_t *rung, double *a_old, double *a_cur, double *a_tot)
{
    tg_status st = begin(c);
    if (st) return st;
    if (c->hhs_n <= 0) return set_err(c, TG_ERR_STATE, "tg_hhs_state before tg_hhs_init");
    const size_t n = (size_t)c->hhs_n;
    // arrays the bound integrator does not keep (|a_old|, |a_cur|, |a|_tot of a traditional run) read as zero
    auto out = [&](void *dst, int slot, size_t bytes) -> cudaError_t {
        if (!dst) return cudaSuccess;
        if (!c->buf[slot].p) return cudaMemsetAsync(dst, 0, bytes, c->stream);
        return cudaMemcpyAsync(dst, c->buf[slot].p, bytes, cudaMemcpyDeviceToDevice, c->stream);
    };
    cudaError_t e = out(rung, B_HHS_RUNG, n * sizeof(int32_t));
    if (e == cudaSuccess) e = out(a_old, B_HHS_AOLD, n * sizeof(double));
    if (e == cudaSuccess) e = out(a_cur, B_HHS_ACUR, n * sizeof(double));
    if (e == cudaSuccess) e = out(a_tot, B_HHS_ATOT, n * sizeof(double));
    if (e != cudaSuccess) return cuda_check(c, e, "tg_hhs_state");
    return cuda_check(c, cudaStreamSynchronize(c->stream), "tg_hhs_state");
}

tg_status tg_hhs_set_accel(tg_ctx *c, const double *a_old, const double *a_cur, const double *a_tot)
{
    tg_status st = begin(c);
    if (st) return st;
    if (c->hhs_n <= 0) return set_err(c, TG_ERR_STATE, "tg_hhs_set_accel before tg_hhs_init");
    if (!check_device_ptr(a_old) || !check_device_ptr(a_cur) || (a_tot && !check_device_ptr(a_tot)))
        return set_err(c, TG_ERR_ARG, "device arrays expected");
    const size_t n = (size_t)c->hhs_n;
    cudaMemcpyAsync(c->buf[B_HHS_AOLD].p, a_old, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->buf[B_HHS_ACUR].p, a_cur, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (a_tot) cudaMemcpyAsync(c->buf[B_HHS_ATOT].p, a_tot, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    return cuda_check(c, cudaGetLastError(), "tg_hhs_set_accel");
}

tg_status tg_diagnostics(tg_ctx *c, double out[8])
{
    tg_status st = begin(c);
    if (st) return st;
    if (!out) return set_err(c, TG_ERR_ARG, "out is NULL");
    if (c->hhs_n <= 0) return set_err(c, TG_ERR_STATE, "tg_diagnostics before tg_hhs_init");
    return hhs_diagnostics(c, out);
}

tg_status tg_debug_control(tg_ctx *c, int what, int64_t value)
{
    tg_status st = begin(c);
    if (st) return st;
    switch (what) {
    case TG_DEBUG_FAIL_ALLOC:
        c->debug_fail_alloc_after = value < 0 ? -1 : value;
        return TG_OK;
    case TG_DEBUG_QUEUE_LIMIT:
        if (value < 0 || value > 0x7fffffff) return set_err(c, TG_ERR_ARG, "tg_debug_control: queue limit out of range");
        c->debug_queue_limit = (unsigned)value;
        return TG_OK;
    case TG_DEBUG_QUEUE_HOLD:
        c->debug_queue_hold = value != 0;
        return TG_OK;
    case TG_DEBUG_BATCH_CAPS:
        c->debug_batch_caps = value < 0 ? 0 : value;
        if (c->hold) hold_graph_reset_sizes(c);
        return TG_OK;
    case TG_DEBUG_LIST_CAPACITY:
        if (value <= 0) return set_err(c, TG_ERR_ARG, "tg_debug_control: list capacity estimate must be > 0");
        c->walk_front_per_cell = c->walk_blocks_per_cell = c->walk_p2p_per_cell = (double)value / 1000.0;
        return TG_OK;
    default:
        return set_err(c, TG_ERR_ARG, "tg_debug_control: unknown control %d", what);
    }
}

tg_status tg_autotune(tg_ctx *c, int64_t n, const double *pos, const double *mass, const uint8_t *is_fast,
                      tg_tuning *out)
{
    tg_status st = begin(c);
    if (st) return st;
    if (!pos && !mass) {
        // step objective on the system bound by tg_hhs_init
        if (is_fast) return set_err(c, TG_ERR_ARG, "tg_autotune: is_fast needs pos and mass");
        if (c->bound_integrator != 1) return set_err(c, TG_ERR_STATE, "tg_autotune: no system bound by tg_hhs_init");
        if (n != 0 && n != c->hhs_n) return set_err(c, TG_ERR_ARG, "tg_autotune: n differs from the bound system");
        if ((st = check_finite(c, c->hhs_n, c->hhs_pos, c->hhs_n, nullptr, c->hhs_mass))) return st;
        return autotune(c, (int)c->hhs_n, nullptr, nullptr, nullptr, out);
    }
    if (n <= 0 || n > INT32_MAX / 4) return set_err(c, TG_ERR_ARG, "tg_autotune: n out of range");
    if (!check_device_ptr(pos) || !check_device_ptr(mass) || (is_fast && !check_device_ptr(is_fast)))
        return set_err(c, TG_ERR_ARG, "tg_autotune: arrays must be device memory");
    if ((st = check_finite(c, n, pos, n, nullptr, mass))) return st;
    return autotune(c, (int)n, pos, mass, is_fast, out);
}

tg_status tg_set_tuning(tg_ctx *c, const tg_tuning *in)
{
    tg_status st = begin(c);
    if (st) return st;
    if (!in || in->n_crit < 1 || in->n_crit > 2 * kMaxNcrit || in->p2p_rows < 1 || in->p2p_rows > 3 ||
        in->m2l_blocks_per_sm < 1 || in->m2l_blocks_per_sm > 64 || in->m2l_form < 0 || in->m2l_form > 1)
        return set_err(c, TG_ERR_ARG, "tg_set_tuning: settings out of range");
    c->prm.n_crit = in->n_crit;
    c->tune.n_crit = in->n_crit;
    c->tune.p2p_rows = in->p2p_rows;
    c->tune.m2l_blocks_per_sm = in->m2l_blocks_per_sm;
    c->tune.m2l_form = in->m2l_form;
    return TG_OK;
}

tg_status tg_get_tuning(const tg_ctx *c, tg_tuning *out)
{
    if (!c || !out) return TG_ERR_ARG;
    *out = c->tune;
    out->n_crit = c->prm.n_crit;
    return TG_OK;
}

tg_status tg_tree_info(tg_ctx *c, double lo[3], double *L, int64_t *n, int64_t *n_cells)
{
    tg_status st = begin(c);
    if (st) return st;
    if (c->last_n <= 0) return set_err(c, TG_ERR_STATE, "no tree built yet");
    Geom g;
    cudaError_t e = cudaMemcpyAsync(&g, c->buf[B_GEOM].p, sizeof g, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "tg_tree_info");
    if (lo) {
        lo[0] = g.lo[0];
        lo[1] = g.lo[1];
        lo[2] = g.lo[2];
    }
    if (L) *L = g.L;
    if (n) *n = c->last_n;
    if (n_cells) *n_cells = c->last_ncell;
    return TG_OK;
}

tg_status tg_get_tree(tg_ctx *c, uint64_t *keys, int64_t *perm, int32_t *level, int64_t *coords, int64_t *first,
                      int64_t *count, int32_t *nchild)
{
    tg_status st = begin(c);
    if (st) return st;
    if (c->last_n <= 0) return set_err(c, TG_ERR_STATE, "no tree built yet");
    const size_t n = (size_t)c->last_n, nc = (size_t)c->last_ncell;
    std::vector<uint32_t> p32(n), cx(nc), cy(nc), cz(nc);
    std::vector<uint8_t> lv(nc), nch(nc);
    std::vector<int32_t> f(nc), cnt(nc);
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *dst, int slot, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, c->buf[slot].p, bytes, cudaMemcpyDeviceToHost, c->stream);
    };
    if (keys) cp(keys, B_KEYS0, n * sizeof(uint64_t));
    cp(p32.data(), B_VALS0, n * sizeof(uint32_t));
    cp(lv.data(), B_C_LEVEL, nc);
    cp(cx.data(), B_C_X, nc * 4);
    cp(cy.data(), B_C_Y, nc * 4);
    cp(cz.data(), B_C_Z, nc * 4);
    cp(f.data(), B_C_FIRST, nc * 4);
    cp(cnt.data(), B_C_COUNT, nc * 4);
    cp(nch.data(), B_C_NCHILD, nc);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "tg_get_tree");
    for (size_t s = 0; s < n; ++s)
        if (perm) perm[s] = p32[s];
    for (size_t i = 0; i < nc; ++i) {
        if (level) level[i] = lv[i];
        if (coords) {
            coords[i] = cx[i];
            coords[nc + i] = cy[i];
            coords[2 * nc + i] = cz[i];
        }
        if (first) first[i] = f[i];
        if (count) count[i] = cnt[i];
        if (nchild) nchild[i] = nch[i];
    }
    return TG_OK;
}

tg_status tg_list_counts(tg_ctx *c, int64_t *n_m2l, int64_t *n_p2p)
{
    tg_status st = begin(c);
    if (st) return st;
    if (n_m2l) *n_m2l = c->last_nm2l;
    if (n_p2p) *n_p2p = c->last_np2p;
    return TG_OK;
}

tg_status tg_get_lists(tg_ctx *c, int64_t *m2l_a, int64_t *m2l_b, int64_t *p2p_a, int64_t *p2p_b)
{
    tg_status st = begin(c);
    if (st) return st;
    const size_t nc = (size_t)c->last_ncell;
    std::vector<M2LBlock> blk(c->last_nblocks);
    std::vector<uint2> p(c->last_np2p);
    std::vector<uint8_t> nch(nc);
    std::vector<int32_t> chf(nc);
    cudaError_t e = cudaSuccess;
    auto cp = [&](void *dst, int slot, size_t bytes) {
        if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(dst, c->buf[slot].p, bytes, cudaMemcpyDeviceToHost, c->stream);
    };
    cp(blk.data(), B_M2L, blk.size() * sizeof(M2LBlock));
    {
        // pairs A != B from the front of the buffer, self pairs from its end
        const size_t nself = (size_t)c->last_np2p_self, nother = p.size() - nself;
        if (e == cudaSuccess && nother)
            e = cudaMemcpyAsync(p.data(), c->buf[B_P2P].p, nother * sizeof(uint2), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && nself)
            e = cudaMemcpyAsync(p.data() + nother, static_cast<uint2 *>(c->buf[B_P2P].p) + (c->p2p_cap - nself),
                                nself * sizeof(uint2), cudaMemcpyDeviceToHost, c->stream);
    }
    cp(nch.data(), B_C_NCHILD, nc);
    cp(chf.data(), B_C_CHILD, nc * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "tg_get_lists");
    // expand the M2L blocks into unordered cell pairs
    size_t q = 0;
    for (const M2LBlock &b : blk) {
        const bool oa = nch[b.a] != 0, ob = nch[b.b] != 0;
        const int ni = oa ? nch[b.a] : 1, nj = ob ? nch[b.b] : 1;
        const int ba = oa ? chf[b.a] : (int)b.a, bb = ob ? chf[b.b] : (int)b.b;
        for (int i = 0; i < ni; ++i)
            for (int j = 0; j < nj; ++j)
                if ((b.mask >> (8 * i + j)) & 1ull) {
                    if ((int64_t)q < c->last_nm2l) {
                        if (m2l_a) m2l_a[q] = ba + i;
                        if (m2l_b) m2l_b[q] = bb + j;
                    }
                    ++q;
                }
    }
    if ((int64_t)q != c->last_nm2l) return set_err(c, TG_ERR_STATE, "M2L block expansion mismatch");
    for (size_t i = 0; i < p.size(); ++i) {
        if (p2p_a) p2p_a[i] = p[i].x;
        if (p2p_b) p2p_b[i] = p[i].y;
    }
    return TG_OK;
}

tg_status tg_timesteps(tg_ctx *c, int64_t n, const double *a_old, const double *a_cur, const double *a_tot, double *dt,
                       int32_t *rung)
{
    tg_status st = begin(c);
    if (st) return st;
    if (n < 0) return set_err(c, TG_ERR_ARG, "n < 0");
    if (n == 0) return TG_OK;
    if (!check_device_ptr(a_old) || !check_device_ptr(a_cur) || !check_device_ptr(dt) || !check_device_ptr(rung) ||
        (a_tot && !check_device_ptr(a_tot)))
        return set_err(c, TG_ERR_ARG, "device arrays expected");
    return timesteps(c, n, a_old, a_cur, a_tot, dt, rung);
}

}  // extern "C"

// ------------------------------------------------------------------ checkpoint / restore
namespace {

const char kCkptMagic[8] = {'T', 'G', 'C', 'K', 'P', 'T', '0', '3'};

struct Fnv64 {
    uint64_t h = 1469598103934665603ull;
    void add(const void *p, size_t n)
    {
        const unsigned char *b = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
};

bool same_params(const tg_params &a, const tg_params &b)
{
    return a.p == b.p && a.n_crit == b.n_crit && a.kernel == b.kernel && a.precision == b.precision &&
           a.max_level == b.max_level && a.k_max == b.k_max && a.theta == b.theta && a.kappa == b.kappa &&
           a.eps == b.eps && a.eta == b.eta && a.dt_max == b.dt_max && a.eta_tot == b.eta_tot && a.mac == b.mac;
}

}  // namespace

extern "C" {

tg_status tg_checkpoint(tg_ctx *c, const char *path)
{
    tg_status st = begin(c);
    if (st) return st;
    if (!path) return set_err(c, TG_ERR_ARG, "tg_checkpoint: path is NULL");
    if (c->hhs_n <= 0 || c->bound_integrator != 1) return set_err(c, TG_ERR_STATE, "tg_checkpoint before tg_hhs_init");
    const size_t n = (size_t)c->hhs_n;
    std::vector<double> pos(3 * n), vel(3 * n), mass(n), a_old(n), a_cur(n), a_tot(n);
    std::vector<int32_t> rung(n);
    cudaMemcpyAsync(pos.data(), c->hhs_pos, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(vel.data(), c->hhs_vel, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(mass.data(), c->hhs_mass, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(a_old.data(), c->buf[B_HHS_AOLD].p, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(a_cur.data(), c->buf[B_HHS_ACUR].p, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(a_tot.data(), c->buf[B_HHS_ATOT].p, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(rung.data(), c->buf[B_HHS_RUNG].p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if ((st = cuda_check(c, cudaStreamSynchronize(c->stream), "tg_checkpoint"))) return st;
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = std::fopen(tmp.c_str(), "wb");
    if (!f) return set_err(c, TG_ERR_IO, "tg_checkpoint: cannot open %s", tmp.c_str());
    Fnv64 h;
    bool ok = true;
    auto put = [&](const void *p, size_t bytes) {
        if (!ok) return;
        h.add(p, bytes);
        ok = std::fwrite(p, 1, bytes, f) == bytes;
    };
    const int64_t n64 = (int64_t)n;
    put(kCkptMagic, sizeof(kCkptMagic));
    put(&n64, sizeof(n64));
    put(&c->prm, sizeof(c->prm));
    put(&c->hhs_time, sizeof(double));
    put(pos.data(), pos.size() * sizeof(double));
    put(vel.data(), vel.size() * sizeof(double));
    put(mass.data(), mass.size() * sizeof(double));
    put(a_old.data(), a_old.size() * sizeof(double));
    put(a_cur.data(), a_cur.size() * sizeof(double));
    put(a_tot.data(), a_tot.size() * sizeof(double));
    put(rung.data(), rung.size() * sizeof(int32_t));
    const uint64_t sum = h.h;
    ok = ok && std::fwrite(&sum, 1, sizeof(sum), f) == sizeof(sum);
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return set_err(c, TG_ERR_IO, "tg_checkpoint: cannot write %s", path);
    }
    return TG_OK;
}

tg_status tg_restore(tg_ctx *c, const char *path)
{
    tg_status st = begin(c);
    if (st) return st;
    if (!path) return set_err(c, TG_ERR_ARG, "tg_restore: path is NULL");
    if (c->hhs_n <= 0 || c->bound_integrator != 1) return set_err(c, TG_ERR_STATE, "tg_restore before tg_hhs_init");
    FILE *f = std::fopen(path, "rb");
    if (!f) return set_err(c, TG_ERR_IO, "tg_restore: cannot open %s", path);
    std::vector<unsigned char> data;
    {
        unsigned char chunk[1 << 16];
        size_t got;
        while ((got = std::fread(chunk, 1, sizeof(chunk), f)) > 0) data.insert(data.end(), chunk, chunk + got);
        std::fclose(f);
    }
    const size_t head = sizeof(kCkptMagic) + sizeof(int64_t) + sizeof(tg_params) + sizeof(double);
    if (data.size() < head + sizeof(uint64_t) || std::memcmp(data.data(), kCkptMagic, sizeof(kCkptMagic)) != 0)
        return set_err(c, TG_ERR_IO, "tg_restore: %s is not a checkpoint", path);
    int64_t n64;
    tg_params prm;
    double time;
    std::memcpy(&n64, data.data() + 8, sizeof(n64));
    std::memcpy(&prm, data.data() + 16, sizeof(prm));
    std::memcpy(&time, data.data() + 16 + sizeof(prm), sizeof(time));
    if (n64 <= 0 || n64 > INT32_MAX / 4) return set_err(c, TG_ERR_IO, "tg_restore: corrupt size in %s", path);
    const size_t n = (size_t)n64;
    const size_t body = n * (3 + 3 + 1 + 1 + 1 + 1) * sizeof(double) + n * sizeof(int32_t);
    if (data.size() != head + body + sizeof(uint64_t)) return set_err(c, TG_ERR_IO, "tg_restore: %s is truncated", path);
    Fnv64 h;
    h.add(data.data(), head + body);
    uint64_t sum;
    std::memcpy(&sum, data.data() + head + body, sizeof(sum));
    if (sum != h.h) return set_err(c, TG_ERR_IO, "tg_restore: checksum mismatch in %s", path);
    if (n64 != c->hhs_n) return set_err(c, TG_ERR_STATE, "tg_restore: file holds n = %lld, bound n = %lld",
                                         (long long)n64, (long long)c->hhs_n);
    if (!same_params(prm, c->prm)) return set_err(c, TG_ERR_STATE, "tg_restore: parameters differ from the context's");
    const unsigned char *p = data.data() + head;
    const double *pos = reinterpret_cast<const double *>(p);
    const double *vel = pos + 3 * n;
    const double *mass = vel + 3 * n;
    const double *a_old = mass + n;
    const double *a_cur = a_old + n;
    const double *a_tot = a_cur + n;
    std::vector<int32_t> rung(n);
    std::memcpy(rung.data(), reinterpret_cast<const unsigned char *>(a_tot + n), n * sizeof(int32_t));
    std::vector<double> bound_mass(n);
    cudaMemcpyAsync(bound_mass.data(), c->hhs_mass, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if ((st = cuda_check(c, cudaStreamSynchronize(c->stream), "tg_restore"))) return st;
    if (std::memcmp(bound_mass.data(), mass, n * sizeof(double)) != 0)
        return set_err(c, TG_ERR_STATE, "tg_restore: the bound masses differ from the file's");
    // the file body is not guaranteed to be 8-byte aligned in the vector: stage through aligned copies
    std::vector<double> pv(9 * n);
    std::memcpy(pv.data(), p, 3 * n * sizeof(double));
    std::memcpy(pv.data() + 3 * n, p + 3 * n * sizeof(double), 3 * n * sizeof(double));
    std::memcpy(pv.data() + 6 * n, p + 7 * n * sizeof(double), 3 * n * sizeof(double));
    cudaMemcpyAsync(c->hhs_pos, pv.data(), 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->hhs_vel, pv.data() + 3 * n, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->buf[B_HHS_AOLD].p, pv.data() + 6 * n, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->buf[B_HHS_ACUR].p, pv.data() + 7 * n, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->buf[B_HHS_ATOT].p, pv.data() + 8 * n, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->buf[B_HHS_RUNG].p, rung.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream);
    if ((st = cuda_check(c, cudaStreamSynchronize(c->stream), "tg_restore"))) return st;
    c->hhs_time = time;
    return TG_OK;
}

}  // extern "C"
