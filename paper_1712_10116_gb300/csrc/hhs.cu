// hhs.cu -- HOLD integrator with individual timesteps (Zhu 2017, Sec. 2.2, Algorithms 1-3):
// timestep function dt_i = sqrt(eta eps / (|a_old| + |a_current|)) (optionally capped by the
// minimum timestep of Eq. 9 from the total acceleration), stable slow/fast split at
// the pivot step of each rung, KDK with the kickS2F / kickFS2S pairs, drifts, and the
// conservation diagnostics of Sec. 3.2.
//
// Each kick pair (kickS2F on F, kickFS2S on S at the same positions) is one FMM evaluation on
// the current system with per-particle classes; this equals the paper's two masked Poisson
// calls and guarantees identical tree walks for both kicks.  Kicks with no sinks or no sources
// are skipped, which gives the (2 + 2 + 2^(k+1)) call count of Sec. 2.2.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <new>

#include "tg_common.cuh"

namespace tg {

// ------------------------------------------------------------------ timestep and split
// rung k pivot step dt_k = dt_max / 2^k; slow = {dt_i >= dt_k} (everything at k = k_max)
// dt_i of Sec. 2.2, capped by Eq. (9) when a_tot is given and eta_tot_eps > 0, with a fixed sequence of
// correctly rounded float64 operations (eta*eps on the host, one division, one square root), so
// that rungs are reproducible bit for bit
__device__ __forceinline__ double timestep_of(double a_old, double a_cur, double eta_eps, const double *a_tot,
                                              double eta_tot_eps, int64_t i)
{
    const double a = __dadd_rn(a_old, a_cur);
    double d = (a > 0.0) ? sqrt(__ddiv_rn(eta_eps, a)) : INFINITY;
    if (a_tot && eta_tot_eps > 0.0) {
        const double at = a_tot[i];
        if (at > 0.0) {
            const double dt_tot = sqrt(__ddiv_rn(eta_tot_eps, at));
            if (dt_tot < d) d = dt_tot;
        }
    }
    return d;
}

__global__ void hhs_timestep(int64_t ns, const int64_t *sys, const double *a_old, const double *a_cur, double eta_eps,
                             const double *a_tot, double eta_tot_eps, double *dt)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = sys ? sys[q] : q;
        dt[i] = timestep_of(a_old[i], a_cur[i], eta_eps, a_tot, eta_tot_eps, i);
    }
}

// |a|_tot of Eq. (9) for every member of the system from an all-masses evaluation
__global__ void hhs_record_total(int64_t ns, const int64_t *sys, const double *acc, double *a_tot)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
        const double ax = acc[q], ay = acc[ns + q], az = acc[2 * ns + q];
        a_tot[sys ? sys[q] : q] = sqrt(ax * ax + ay * ay + az * az);
    }
}

__global__ void hhs_flags(int64_t ns, const int64_t *sys, const double *dt, double dt_k, int deepest, uint32_t *flag,
                          uint8_t *fast)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = sys[q];
        const uint32_t f = (!deepest && !(dt[i] >= dt_k)) ? 1u : 0u;
        flag[q] = f;
        fast[q] = (uint8_t)f;
    }
}

__global__ void hhs_partition(int64_t ns, const int64_t *sys, const uint32_t *flag, const uint32_t *pre, int64_t *S,
                              int64_t *F, int32_t *rung, int k)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = sys[q];
        if (flag[q]) {
            F[pre[q]] = i;
        } else {
            S[q - pre[q]] = i;
            rung[i] = k;
        }
    }
}

// v += a dt for the sinks of the pair; |a| bookkeeping (kickFS2S: a_current; second kickS2F: a_old)
__global__ void hhs_kick(int64_t ns, const int64_t *sys, const uint8_t *fast, const double *acc, double half_dt,
                         int second, int64_t n_all, double *vel, double *a_old, double *a_cur)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = sys[q];
        const double ax = acc[q], ay = acc[ns + q], az = acc[2 * ns + q];
        vel[i] += ax * half_dt;
        vel[n_all + i] += ay * half_dt;
        vel[2 * n_all + i] += az * half_dt;
        const double amag = sqrt(ax * ax + ay * ay + az * az);
        if (fast && fast[q]) {
            if (second) a_old[i] = amag;
        } else {
            a_cur[i] = amag;
        }
    }
}

__global__ void hhs_drift(int64_t ns, const int64_t *S, double dt, int64_t n_all, double *pos, const double *vel)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = S[q];
        pos[i] += vel[i] * dt;
        pos[n_all + i] += vel[n_all + i] * dt;
        pos[2 * n_all + i] += vel[2 * n_all + i] * dt;
    }
}

__global__ void hhs_iota(int64_t n, int64_t *idx)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) idx[q] = q;
}

__global__ void hhs_init_accel(int64_t n, const double *acc, double *a_old, double *a_cur, double *a_tot)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double ax = acc[i], ay = acc[n + i], az = acc[2 * n + i];
        a_old[i] = 0.0;
        a_cur[i] = sqrt(ax * ax + ay * ay + az * az);
        a_tot[i] = a_cur[i];
    }
}

// ------------------------------------------------------------------ host scheduler
struct Level {
    int64_t *sys = nullptr;     // current system (global indices, ascending)
    int64_t *S = nullptr;       // slow set
    uint32_t *flag = nullptr;   // fast flag per system element (scan input)
    uint32_t *pre = nullptr;    // exclusive scan of flag
    uint8_t *fast = nullptr;    // fast flag as bytes (FMM classes)
};

struct Sched {
    tg_ctx *c;
    int64_t n;
    std::vector<Level> lv;
    double *a_old, *a_cur, *a_tot, *dt, *acc;
    int32_t *rung;
    int64_t *all;
};

static tg_status level_buffers(tg_ctx *c, int64_t n, std::vector<Level> &lv, int kmax)
{
    // per-level lists live in one allocation: sys | S (int64), flag | pre (uint32), fast (uint8)
    // each level's block starts on a 256-byte boundary (int64 lists need 8-byte alignment)
    const size_t per = ((n * (2 * sizeof(int64_t) + 2 * sizeof(uint32_t) + 1) + 64) + 255) & ~(size_t)255;
    char *base;
    tg_status st = ensure_t(c, B_HHS_IDX, per * (kmax + 2), &base);
    if (st) return st;
    lv.resize(kmax + 2);
    for (int k = 0; k <= kmax + 1; ++k) {
        char *p = base + per * k;
        lv[k].sys = reinterpret_cast<int64_t *>(p);
        lv[k].S = lv[k].sys + n;
        lv[k].flag = reinterpret_cast<uint32_t *>(lv[k].S + n);
        lv[k].pre = lv[k].flag + n;
        lv[k].fast = reinterpret_cast<uint8_t *>(lv[k].pre + n);
    }
    return TG_OK;
}

static tg_status kick_pair(Sched &s, int k, int64_t ns, int64_t nS, int64_t nF, double dt, int second)
{
    tg_ctx *c = s.c;
    if (nS == 0) return TG_OK;  // kickFS2S has no sinks, kickS2F no sources
    Level &L = s.lv[k];
    tg_status st = fmm_eval(c, (int)ns, c->hhs_pos, s.n, L.sys, c->hhs_mass, nF > 0 ? L.fast : nullptr, s.acc, ns,
                            nullptr, false);
    if (st) return st;
    {
        ProfScope ps_(c, TG_K_HHS);
        hhs_kick<<<grid_for(ns, 256), 256, 0, c->stream>>>(ns, L.sys, nF > 0 ? L.fast : nullptr, s.acc, 0.5 * dt, second,
                                                           s.n, c->hhs_vel, s.a_old, s.a_cur);
    }
    if (k == 0 && second && c->prm.eta_tot > 0.0) {
        // Eq. (9): the second kickFS2S of rung 0 passes the whole system with all masses to the
        // Poisson solver; with a fast set the kick pair above masked F-F, so evaluate once more
        if (nF > 0 && (st = fmm_eval(c, (int)ns, c->hhs_pos, s.n, L.sys, c->hhs_mass, nullptr, s.acc, ns, nullptr, false)))
            return st;
        ProfScope ps_(c, TG_K_HHS);
        hhs_record_total<<<grid_for(ns, 256), 256, 0, c->stream>>>(ns, L.sys, s.acc, s.a_tot);
    }
    return cuda_check(c, cudaGetLastError(), "kick");
}

static tg_status evolve_hold(Sched &s, int k, int64_t ns, double dt, int calc)
{
    tg_ctx *c = s.c;
    tg_status st;
    Level &L = s.lv[k];
    const int kmax = c->prm.k_max;
    if (calc)
        {
            ProfScope ps_(c, TG_K_HHS);
            hhs_timestep<<<grid_for(ns, 256), 256, 0, c->stream>>>(ns, L.sys, s.a_old, s.a_cur, c->prm.eta * c->prm.eps,
                                                                   s.a_tot, c->prm.eta_tot * c->prm.eps, s.dt);
        }
    {
        ProfScope ps_(c, TG_K_HHS);
        hhs_flags<<<grid_for(ns, 256), 256, 0, c->stream>>>(ns, L.sys, s.dt, dt, k >= kmax ? 1 : 0, L.flag, L.fast);
    }
    uint32_t *d_total = reinterpret_cast<uint32_t *>(c->d_counters + 9);
    if ((st = exclusive_scan_u32(c, L.flag, L.pre, (int)ns, d_total))) return st;
    Level &N = s.lv[k + 1];
    {
        ProfScope ps_(c, TG_K_HHS);
        hhs_partition<<<grid_for(ns, 256), 256, 0, c->stream>>>(ns, L.sys, L.flag, L.pre, L.S, N.sys, s.rung, k);
    }
    uint32_t *h = reinterpret_cast<uint32_t *>(c->h_pinned + 40);
    cudaMemcpyAsync(h, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = stream_sync(c);
    if (e != cudaSuccess) return cuda_check(c, e, "hhs split");
    const int64_t nF = (int64_t)*h, nS = ns - nF;
    if (nS > 0 && k > c->stats.max_rung) c->stats.max_rung = k;
    if (nF > 0 && (st = evolve_hold(s, k + 1, nF, 0.5 * dt, 0))) return st;
    // KDK (Algorithm 2)
    c->stats.kdk_frames += 1;
    if ((st = kick_pair(s, k, ns, nS, nF, dt, 0))) return st;
    if (nS > 0) {
        {
            ProfScope ps_(c, TG_K_HHS);
            hhs_drift<<<grid_for(nS, 256), 256, 0, c->stream>>>(nS, L.S, dt, s.n, c->hhs_pos, c->hhs_vel);
        }
        if ((st = cuda_check(c, cudaGetLastError(), "drift"))) return st;
    }
    if ((st = kick_pair(s, k, ns, nS, nF, dt, 1))) return st;
    if (nF > 0 && (st = evolve_hold(s, k + 1, nF, 0.5 * dt, 1))) return st;
    return TG_OK;
}

static tg_status make_sched(tg_ctx *c, Sched &s)
{
    tg_status st;
    s.c = c;
    s.n = c->hhs_n;
    if ((st = ensure_t(c, B_HHS_AOLD, s.n, &s.a_old)) || (st = ensure_t(c, B_HHS_ACUR, s.n, &s.a_cur)) ||
        (st = ensure_t(c, B_HHS_ATOT, s.n, &s.a_tot)) ||
        (st = ensure_t(c, B_HHS_DT, s.n, &s.dt)) || (st = ensure_t(c, B_HHS_RUNG, s.n, &s.rung)) ||
        (st = ensure_t(c, B_SUB_ACC, 3 * s.n, &s.acc)))
        return st;
    return TG_OK;
}

tg_status hhs_init(tg_ctx *c)
{
    Sched s;
    tg_status st = make_sched(c, s);
    if (st) return st;
    if ((st = fmm_eval(c, (int)s.n, c->hhs_pos, s.n, nullptr, c->hhs_mass, nullptr, s.acc, s.n, nullptr, false)))
        return st;
    {
        ProfScope ps_(c, TG_K_HHS);
        hhs_init_accel<<<grid_for(s.n, 256), 256, 0, c->stream>>>(s.n, s.acc, s.a_old, s.a_cur, s.a_tot);
    }
    cudaMemsetAsync(s.rung, 0, sizeof(int32_t) * s.n, c->stream);
    c->hhs_time = 0.0;
    return cuda_check(c, cudaGetLastError(), "hhs init");
}

// Snapshot of the integrator state (pos, vel, |a_old|, |a_cur|, |a|_tot, rungs) that makes a rung-0 step
// transactional: an error inside the step copies it back.
static tg_status snapshot_state(tg_ctx *c, const Sched &s, char **snap, int slot = B_SNAP)
{
    const size_t n = (size_t)s.n;
    tg_status st = ensure_t(c, slot, n * (9 * sizeof(double) + sizeof(int32_t)), snap);
    if (st) return st;
    double *d = reinterpret_cast<double *>(*snap);
    cudaMemcpyAsync(d, c->hhs_pos, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(d + 3 * n, c->hhs_vel, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(d + 6 * n, s.a_old, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(d + 7 * n, s.a_cur, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(d + 8 * n, s.a_tot, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(d + 9 * n, s.rung, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
    return cuda_check(c, cudaGetLastError(), "hhs snapshot");
}

static void restore_state(tg_ctx *c, const Sched &s, const char *snap)
{
    const size_t n = (size_t)s.n;
    const double *d = reinterpret_cast<const double *>(snap);
    cudaMemcpyAsync(c->hhs_pos, d, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(c->hhs_vel, d + 3 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(s.a_old, d + 6 * n, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(s.a_cur, d + 7 * n, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(s.a_tot, d + 8 * n, n * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(s.rung, d + 9 * n, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, c->stream);
    stream_sync(c);
}

// The bound integrator state (pos, vel, |a| and rungs) into / back from a scratch slot other than the
// step's own snapshot (the autotuner's step objective); the step time is saved by the caller.
tg_status hhs_save(tg_ctx *c, int slot)
{
    Sched s;
    tg_status st = make_sched(c, s);
    if (st) return st;
    char *snap = nullptr;
    return snapshot_state(c, s, &snap, slot);
}

tg_status hhs_load(tg_ctx *c, int slot)
{
    Sched s;
    tg_status st = make_sched(c, s);
    if (st) return st;
    if (!c->buf[slot].p) return set_err(c, TG_ERR_STATE, "no saved integrator state");
    restore_state(c, s, static_cast<const char *>(c->buf[slot].p));
    return cuda_check(c, cudaGetLastError(), "hhs state restore");
}

tg_status hhs_step(tg_ctx *c)
{
    if (c->prm.batched) return hhs_step_batched(c);
    Sched s;
    tg_status st = make_sched(c, s);
    if (st) return st;
    if ((st = check_finite(c, s.n, c->hhs_pos, s.n, nullptr, c->hhs_mass))) return st;
    char *snap = nullptr;
    if ((st = snapshot_state(c, s, &snap))) return st;
    const tg_stats stats0 = c->stats;
    if ((st = level_buffers(c, s.n, s.lv, c->prm.k_max)) == TG_OK) {
        {
            ProfScope ps_(c, TG_K_HHS);
            hhs_iota<<<grid_for(s.n, 256), 256, 0, c->stream>>>(s.n, s.lv[0].sys);
        }
        st = evolve_hold(s, 0, s.n, c->prm.dt_max, 1);
        if (st == TG_OK) st = cuda_check(c, stream_sync(c), "hhs step");
    }
    if (st) {
        // the buffers may have moved while growing: the snapshot slot is looked up again
        restore_state(c, s, static_cast<const char *>(c->buf[B_SNAP].p));
        const int64_t regrow = c->stats.list_regrowths;
        c->stats = stats0;
        c->stats.list_regrowths = regrow;
        return st;
    }
    c->hhs_time += c->prm.dt_max;
    return TG_OK;
}

// ------------------------------------------------------------------ batched HOLD step
// The recursion of Algorithms 1-2 becomes a device-side work queue: a stack of frames (level k, calc
// flag, phase) in device memory, advanced by a one-thread scheduler kernel that publishes the next
// operation -- a split at level k, a kick pair (with the drift after the first), or the extra
// all-masses evaluation of Eq. (9) -- and sets the conditions of a CUDA graph: a WHILE node whose body
// is the scheduler, an IF node holding the split kernels and an IF node holding one evaluation with
// its kick.  A rung-0 step is one launch of that graph; the host reads its counters once at the end.
// The operations run in exactly the order of the host-driven recursion, with the same kernels.
constexpr int kHoldLevels = 32;   // k_max <= 30, plus the level below the deepest

enum HoldOp { kOpNone = 0, kOpSplit = 1, kOpKick1 = 2, kOpKick2 = 3, kOpTotal = 4, kOpDone = 5 };

struct HoldState {
    // read by the host after the step
    int status;                     // 0: finished; 1: the loop stopped at its iteration limit
    int pad0;
    unsigned long long stats[8];    // evaluations, particle-forces, M2L pairs, M2L pairs x classes,
                                    // P2P leaf pairs, cells, KDK frames, deepest rung holding a slow particle
    unsigned long long splits, evals, iterations;
    // scheduler state
    int op, k, calc, sp;
    int stack_k[kHoldLevels], stack_calc[kHoldLevels], stack_phase[kHoldLevels];
    long long ns[kHoldLevels], nF[kHoldLevels];   // system size and fast count per level
    int cur_ns;                     // size of the system being split (device count of its scan)
    uint32_t split_total;           // fast members found by the split (scan total)
    unsigned limit;                 // iteration limit of the loop
    int hold;                       // test hook: publish no operation
};

// per-level lists (the layout of level_buffers): sys | S (int64) | flag | pre (uint32) | fast (uint8)
struct LevelLayout {
    char *base;
    size_t per;
    int64_t n;
    __device__ __forceinline__ int64_t *sys(int k) const { return reinterpret_cast<int64_t *>(base + per * k); }
    __device__ __forceinline__ int64_t *slow(int k) const { return sys(k) + n; }
    __device__ __forceinline__ uint8_t *fast(int k) const
    {
        return reinterpret_cast<uint8_t *>(reinterpret_cast<uint32_t *>(slow(k) + n) + 2 * n);
    }
};

__global__ void hold_begin(HoldState *h, DevEval *de, LevelLayout lv, int64_t n, unsigned limit, int hold)
{
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        h->status = 0;
        for (int i = 0; i < 8; ++i) h->stats[i] = 0ull;
        h->splits = h->evals = h->iterations = 0ull;
        h->op = kOpNone;
        h->sp = 1;
        h->stack_k[0] = 0;
        h->stack_calc[0] = 1;
        h->stack_phase[0] = 0;
        h->ns[0] = n;
        h->nF[0] = 0;
        h->limit = limit;
        h->hold = hold;
        de->overflow = 0u;
    }
    int64_t *sys0 = lv.sys(0);
    for (int64_t q = tid; q < n; q += (int64_t)gridDim.x * blockDim.x) sys0[q] = q;
}

// One iteration of the loop: advance the frames of Algorithm 1 to the next operation.  Phases of a
// frame: 0 split; 1 after the split (recurse into level k + 1 with calc = 0 if there is a fast set);
// 2 first kick pair and drift; 3 second kick pair; 4 the Eq. (9) evaluation at rung 0; 5 recurse with
// calc = 1; 6 return.  Kick pairs without slow sinks are skipped, as in the host recursion.
__global__ void hold_sched(HoldState *h, int k_max, int eq9, cudaGraphConditionalHandle h_loop,
                           cudaGraphConditionalHandle h_split, cudaGraphConditionalHandle h_eval)
{
    int op = kOpNone;
    h->iterations += 1ull;
    if (h->iterations > h->limit) {
        h->status = 1;   // bounded: give up, the host restores the state and reports a timeout
        op = kOpDone;
    } else if (!h->hold) {
        for (int guard = 0; guard < 8 * kHoldLevels && op == kOpNone; ++guard) {
            if (h->sp == 0) {
                op = kOpDone;
                break;
            }
            const int top = h->sp - 1, k = h->stack_k[top];
            const long long nF = h->nF[k], nS = h->ns[k] - h->nF[k];
            switch (h->stack_phase[top]) {
            case 0:
                h->stack_phase[top] = 1;
                h->k = k;
                h->calc = h->stack_calc[top];
                h->cur_ns = (int)h->ns[k];
                op = kOpSplit;
                break;
            case 1:
                h->stack_phase[top] = 2;
                if (nF > 0 && h->sp < kHoldLevels) {
                    h->stack_k[h->sp] = k + 1;
                    h->stack_calc[h->sp] = 0;
                    h->stack_phase[h->sp] = 0;
                    h->sp += 1;
                }
                break;
            case 2:
                h->stack_phase[top] = 3;
                h->stats[6] += 1ull;   // a KDK frame
                if (nS > 0) {
                    h->k = k;
                    op = kOpKick1;
                }
                break;
            case 3:
                h->stack_phase[top] = 4;
                if (nS > 0) {
                    h->k = k;
                    op = kOpKick2;
                }
                break;
            case 4:
                h->stack_phase[top] = 5;
                if (eq9 && k == 0 && nS > 0 && nF > 0) {
                    h->k = k;
                    op = kOpTotal;
                }
                break;
            case 5:
                h->stack_phase[top] = 6;
                if (nF > 0 && h->sp < kHoldLevels) {
                    h->stack_k[h->sp] = k + 1;
                    h->stack_calc[h->sp] = 1;
                    h->stack_phase[h->sp] = 0;
                    h->sp += 1;
                }
                break;
            default:
                h->sp -= 1;
            }
        }
        if (op == kOpNone) op = kOpDone;   // the guard ran out: end the step (cannot happen with k_max <= 30)
    }
    h->op = op;
    if (op == kOpSplit) h->splits += 1ull;
    if (op == kOpKick1 || op == kOpKick2 || op == kOpTotal) h->evals += 1ull;
    cudaGraphSetConditional(h_split, op == kOpSplit ? 1u : 0u);
    cudaGraphSetConditional(h_eval, (op == kOpKick1 || op == kOpKick2 || op == kOpTotal) ? 1u : 0u);
    cudaGraphSetConditional(h_loop, op == kOpDone ? 0u : 1u);
}

__global__ void hold_timestep(const HoldState *h, LevelLayout lv, const double *a_old, const double *a_cur,
                              double eta_eps, const double *a_tot, double eta_tot_eps, double *dt)
{
    if (!h->calc) return;
    const int k = h->k;
    const int64_t ns = h->ns[k];
    const int64_t *sys = lv.sys(k);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = sys[q];
        dt[i] = timestep_of(a_old[i], a_cur[i], eta_eps, a_tot, eta_tot_eps, i);
    }
}

__global__ void hold_flags(const HoldState *h, LevelLayout lv, const double *dt, double dt_max, int k_max,
                           uint32_t *flag)
{
    const int k = h->k;
    const int64_t ns = h->ns[k];
    const int64_t *sys = lv.sys(k);
    uint8_t *fast = lv.fast(k);
    const double dt_k = ldexp(dt_max, -k);   // dt_max halved k times, exactly
    const int deepest = k >= k_max;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t f = (!deepest && !(dt[sys[q]] >= dt_k)) ? 1u : 0u;
        flag[q] = f;
        fast[q] = (uint8_t)f;
    }
}

__global__ void hold_partition(const HoldState *h, LevelLayout lv, const uint32_t *flag, const uint32_t *pre,
                               int32_t *rung)
{
    const int k = h->k;
    const int64_t ns = h->ns[k];
    const int64_t *sys = lv.sys(k);
    int64_t *S = lv.slow(k), *F = lv.sys(k + 1);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = sys[q];
        if (flag[q]) {
            F[pre[q]] = i;
        } else {
            S[q - pre[q]] = i;
            rung[i] = k;
        }
    }
}

__global__ void hold_split_finish(HoldState *h)
{
    const int k = h->k;
    const long long nF = (long long)h->split_total;
    h->nF[k] = nF;
    h->ns[k + 1] = nF;
    h->nF[k + 1] = 0;
    if (h->ns[k] - nF > 0 && (unsigned long long)k > h->stats[7]) h->stats[7] = (unsigned long long)k;
}

// gather the system of the evaluation in flight into contiguous buffers (stride cap_n) and publish
// its size and class count to the device-sized evaluation
__global__ void hold_frame(const HoldState *h, LevelLayout lv, const double *pos, int64_t n_all, const double *mass,
                           double *xin, double *min, uint8_t *fin, DevEval *de, int64_t cap_n)
{
    const int k = h->k;
    const int64_t ns = h->ns[k];
    const int masked = (h->op != kOpTotal) && h->nF[k] > 0;
    const int64_t *sys = lv.sys(k);
    const uint8_t *fast = lv.fast(k);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        de->n = (int)ns;
        de->np1 = (int)ns + 1;
        de->masked = masked;
        de->sort_blocks = (int)((ns + kSortTileItems - 1) / kSortTileItems);
        de->hist_items = kSortBins * de->sort_blocks;
    }
    for (int64_t q = tid; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = sys[q];
        xin[q] = pos[i];
        xin[cap_n + q] = pos[n_all + i];
        xin[2 * cap_n + q] = pos[2 * n_all + i];
        min[q] = mass[i];
        fin[q] = masked ? fast[q] : (uint8_t)0;
    }
}

// the kick of the evaluation in flight (the same arithmetic as hhs_kick), or |a|_tot of Eq. (9)
__global__ void hold_kick(const HoldState *h, LevelLayout lv, const double *acc, int64_t cap_n, double dt_max,
                          int64_t n_all, double *vel, double *a_old, double *a_cur, double *a_tot, int eq9)
{
    const int op = h->op, k = h->k;
    const int64_t ns = h->ns[k];
    const int64_t *sys = lv.sys(k);
    const int masked = (op != kOpTotal) && h->nF[k] > 0;
    const uint8_t *fast = lv.fast(k);
    const int second = op == kOpKick2;
    const bool record = op == kOpTotal || (eq9 && second && k == 0 && !masked);
    const double half_dt = 0.5 * ldexp(dt_max, -k);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ns; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = sys[q];
        const double ax = acc[q], ay = acc[cap_n + q], az = acc[2 * cap_n + q];
        if (op != kOpTotal) {
            vel[i] += ax * half_dt;
            vel[n_all + i] += ay * half_dt;
            vel[2 * n_all + i] += az * half_dt;
            const double amag = sqrt(ax * ax + ay * ay + az * az);
            if (masked && fast[q]) {
                if (second) a_old[i] = amag;
            } else {
                a_cur[i] = amag;
            }
        }
        if (record) a_tot[i] = sqrt(ax * ax + ay * ay + az * az);
    }
}

__global__ void hold_drift(const HoldState *h, LevelLayout lv, double dt_max, int64_t n_all, double *pos,
                           const double *vel)
{
    if (h->op != kOpKick1) return;
    const int k = h->k;
    const int64_t nS = h->ns[k] - h->nF[k];
    const int64_t *S = lv.slow(k);
    const double dt = ldexp(dt_max, -k);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nS; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = S[q];
        pos[i] += vel[i] * dt;
        pos[n_all + i] += vel[n_all + i] * dt;
        pos[2 * n_all + i] += vel[2 * n_all + i] * dt;
    }
}

}  // namespace tg

// One graph holding the step loops of several contexts, and what each member was captured with.
struct EnsembleGraph {
    std::vector<tg_ctx *> members;
    std::vector<uint64_t> epochs;
    std::vector<tg_params> prms;
    std::vector<tg_tuning> tunes;
    std::vector<const void *> bound;   // pos, vel, mass per member
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// The captured graph of the batched step and what it was captured with.
struct HoldGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    tg::BatchCaps caps;
    bool sized = false;                 // caps hold estimates from a plain evaluation
    uint64_t epoch = ~0ull;             // alloc_epoch at capture
    tg_params prm{};                    // parameters at capture
    tg_tuning tune{};
    int64_t n = 0;                      // bound system size at capture
    void *bound[3] = {nullptr, nullptr, nullptr};
    int64_t launches_split[TG_K_COUNT] = {0}, launches_eval[TG_K_COUNT] = {0};
    unsigned long long *h_read = nullptr;   // pinned: HoldState head + overflow word
    struct EnsembleGraph *ens = nullptr;    // ensemble graph this context leads (tg_ensemble_step)
};

namespace tg {

void ensemble_destroy(tg_ctx *c);

void hold_graph_destroy(tg_ctx *c)
{
    HoldGraph *g = c->hold;
    if (!g) return;
    ensemble_destroy(c);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    if (g->h_read) cudaFreeHost(g->h_read);
    delete g;
    c->hold = nullptr;
}

static bool same_capture_params(const tg_params &a, const tg_params &b)
{
    return a.p == b.p && a.n_crit == b.n_crit && a.kernel == b.kernel && a.precision == b.precision &&
           a.max_level == b.max_level && a.k_max == b.k_max && a.theta == b.theta && a.kappa == b.kappa &&
           a.eps == b.eps && a.eta == b.eta && a.dt_max == b.dt_max && a.eta_tot == b.eta_tot && a.mac == b.mac;
}

static unsigned hold_limit(const tg_ctx *c)
{
    if (c->debug_queue_limit) return c->debug_queue_limit;
    // at most 2^(k+1) - 1 frames of four operations each, plus the splits; k_max is capped for the bound
    const int k = std::min(c->prm.k_max, 22);
    return (unsigned)(8u << k) + 64u;
}

// every scratch buffer the captured graph uses, at its capacity (nothing may grow inside a capture)
static tg_status hold_presize(tg_ctx *c, const Sched &s, const BatchCaps &cap, const std::vector<Level> &lv)
{
    (void)lv;
    tg_status st;
    void *p;
    const int n = cap.n, C = cap.cells, p_ = c->prm.p, ncp = (ncoef(p_) + 3) & ~3;
    const size_t rows = (size_t)C * 2;
    const int nblocks = (n + kSortTileItems - 1) / kSortTileItems;
    const int nh = (p_ + 1) * (p_ + 1), ncpr = (nh + 3) & ~3;
    const int64_t max_units = (int64_t)cap.p2p / 16 + C + 1;
    const size_t tsz = c->prm.precision == TG_PREC_FP32 ? 4 : 8;   // compute precision
    struct Need { int slot; size_t bytes; };
    const Need needs[] = {
        {B_GEOM, 64}, {B_PARTIAL, sizeof(double) * 6 * 2 * 152}, {B_KEYS0, 8ull * n}, {B_KEYS1, 8ull * n},
        {B_VALS0, 4ull * n}, {B_VALS1, 4ull * n}, {B_HIST, 4ull * ((size_t)kSortBins * nblocks + 1)},
        {B_SCAN_TMP, 4 * std::max(scan_scratch_words(std::max(kSortBins * nblocks, 1)), std::max(scan_scratch_words(C), scan_scratch_words(n + 1)))},
        {B_XS, 8ull * n}, {B_YS, 8ull * n}, {B_ZS, 8ull * n}, {B_MS, 8ull * n}, {B_FS, 1ull * n},
        {B_XS2, 8ull * n}, {B_YS2, 8ull * n}, {B_ZS2, 8ull * n}, {B_MS2, 8ull * n}, {B_FS2, 1ull * n},
        {B_PERM2, 4ull * n}, {B_NSLOW, 4ull * C}, {B_PF, 4 * tsz * n}, {B_LEAF_OF, 4ull * n},
        {B_C_LEVEL, 1ull * C}, {B_C_X, 4ull * C}, {B_C_Y, 4ull * C}, {B_C_Z, 4ull * C}, {B_C_FIRST, 4ull * C},
        {B_C_COUNT, 4ull * C}, {B_C_CHILD, 4ull * C}, {B_C_PARENT, 4ull * C}, {B_C_NCHILD, 1ull * C},
        {B_C_TMP0, 4ull * C}, {B_C_TMP1, 4ull * C},
        {B_MOM, tsz * rows * ncp}, {B_MOMF, tsz * rows * ncp}, {B_MOM01, 8 * rows * 4}, {B_LOC, tsz * rows * ncp},
        {B_ACC, 32ull * n}, {B_MOMH, 4 * rows * ncpr}, {B_LOCH, 4 * rows * ncpr},
        {B_FRONT0, 8 * cap.front}, {B_FRONT1, 8 * cap.front}, {B_M2L, 16 * cap.blocks}, {B_P2P, 8 * cap.p2p},
        {B_WALK_CNT, 8 * (8 + 24 + 1)},
        {B_OWN_CNT, 4ull * (C + 2)}, {B_OWN_FILL, 4ull * (C + 2)}, {B_OWN_OFF, 4ull * C},
        {B_OWN_LIST, 8ull * max_units}, {B_OWN_TAG, 8 * cap.p2p}, {B_OWN_PART, 4 * cap.p2p},
        {B_M2L_CNT, 4ull * C}, {B_M2L_OFF, 4ull * C}, {B_M2L_FILL, 4ull * C}, {B_M2L_SRC, 4 * cap.m2l_src},
        {B_FWORDS, 4ull * (n + 1)}, {B_FPRE, 4ull * (n + 1)}, {B_M2L_PART, 16 * cap.blocks}, {B_M2L_PCNT, 16},
        {B_SCAN_TMP2, 4 * std::max(scan_scratch_words(std::max(kSortBins * nblocks, 1)), std::max(scan_scratch_words(C), scan_scratch_words(n + 1)))},
        {B_ACC_P2P, 32ull * n},
        {B_FRAME_X, 24ull * n}, {B_FRAME_M, 8ull * n}, {B_FRAME_F, 1ull * n}, {B_SPLIT_FLAG, 4ull * n},
        {B_SPLIT_PRE, 4ull * n}, {B_HOLD, sizeof(HoldState)}, {B_DEVEVAL, sizeof(DevEval)},
    };
    for (const Need &q : needs)
        if ((st = ensure(c, q.slot, q.bytes + 16, &p))) return st;
    (void)s;
    return TG_OK;
}

// Capacities from one plain evaluation of the whole bound system (the largest evaluation of a step),
// with margins: sub-systems of deep rungs have their own, smaller root cubes.
static tg_status hold_size(tg_ctx *c, Sched &s, BatchCaps &cap)
{
    tg_status st;
    if ((st = fmm_eval(c, (int)s.n, c->hhs_pos, s.n, nullptr, c->hhs_mass, nullptr, s.acc, s.n, nullptr, false))) return st;
    if ((st = cuda_check(c, stream_sync(c), "batched sizing"))) return st;
    c->stats.evaluations -= 1;   // sizing is not the caller's work
    c->stats.sink_forces -= s.n;
    c->stats.m2l_pairs -= c->last_nm2l;
    if (!m2l_classes_on_device(c)) c->stats.m2l_class_pairs -= c->last_nm2l;
    c->stats.p2p_cell_pairs -= c->last_np2p;
    c->stats.cells -= c->last_ncell;
    const int64_t ncell = c->last_ncell;
    const int nlev = (int)c->level_begin.size() - 1;
    cap.n = (int)s.n;
    cap.cells = (int)std::min<int64_t>(INT32_MAX / 8, ncell * 3 / 2 + 4096);
    cap.levels = std::min(c->prm.max_level, nlev + 2);
    cap.front = (size_t)(cap.cells * c->walk_front_per_cell * 1.25) + 4096;
    cap.blocks = (size_t)(cap.cells * c->walk_blocks_per_cell * 1.25) + 4096;
    cap.p2p = (size_t)(cap.cells * c->walk_p2p_per_cell * 1.25) + 4096;
    cap.m2l_src = (size_t)(2.0 * c->last_nm2l * 1.5) + 4096;
    if (c->debug_batch_caps > 0) {   // test hook: start too small, so that the step must regrow
        cap.front = cap.blocks = cap.p2p = cap.m2l_src = (size_t)c->debug_batch_caps;
        cap.cells = (int)std::max<int64_t>(64, c->debug_batch_caps);
    }
    return TG_OK;
}

void hold_graph_reset_sizes(tg_ctx *c)
{
    if (c->hold) c->hold->sized = false;
}

static tg_status capture_begin(tg_ctx *c, HoldGraph *g, cudaGraph_t into)
{
    cudaError_t e = cudaStreamBeginCaptureToGraph(g->cap_stream, into, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    return cuda_check(c, e, "graph capture begin");
}

static tg_status capture_end(tg_ctx *c, HoldGraph *g)
{
    cudaGraph_t out = nullptr;
    cudaError_t e = cudaStreamEndCapture(g->cap_stream, &out);
    return cuda_check(c, e, "graph capture end");
}

// an IF node on `h` (created on `parent`) after `dep`; its body graph comes back in *body
static tg_status add_if(tg_ctx *c, cudaGraph_t parent, const cudaGraphNode_t *dep, cudaGraphNode_t *node,
                        cudaGraphConditionalHandle h, cudaGraph_t *body)
{
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaError_t e = cudaGraphAddNode(node, parent, dep, nullptr, dep ? 1 : 0, &np);
    if (e != cudaSuccess) return cuda_check(c, e, "conditional IF node");
    *body = np.conditional.phGraph_out[0];
    return TG_OK;
}

// Capture the step's graph: WHILE { scheduler; IF split { ... }; IF evaluation { ... } }.
// The step's loop, WHILE { scheduler; IF split { ... }; IF evaluation { ... } }, added to `parent` (the
// context's own graph, or an ensemble graph holding the loops of several contexts side by side).
static tg_status hold_capture_into(tg_ctx *c, HoldGraph *g, Sched &s, const std::vector<Level> &lv, size_t per,
                                   cudaGraph_t parent)
{
    tg_status st;
    if ((st = hold_presize(c, s, g->caps, lv))) return st;
    if ((st = mac_params_upload(c))) return st;
    HoldState *h = static_cast<HoldState *>(c->buf[B_HOLD].p);
    DevEval *de = static_cast<DevEval *>(c->buf[B_DEVEVAL].p);
    double *xin = static_cast<double *>(c->buf[B_FRAME_X].p), *min = static_cast<double *>(c->buf[B_FRAME_M].p);
    uint8_t *fin = static_cast<uint8_t *>(c->buf[B_FRAME_F].p);
    uint32_t *flag = static_cast<uint32_t *>(c->buf[B_SPLIT_FLAG].p), *pre = static_cast<uint32_t *>(c->buf[B_SPLIT_PRE].p);
    const LevelLayout L{reinterpret_cast<char *>(lv[0].sys), per, s.n};
    const int64_t N = s.n;
    const int cap_n = g->caps.n;
    const int grid = grid_for(N, 256, c->num_sms * 8);
    cudaError_t e;
    cudaGraphConditionalHandle h_loop;
    if ((e = cudaGraphConditionalHandleCreate(&h_loop, parent, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
        return cuda_check(c, e, "conditional handle");
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if ((e = cudaGraphAddNode(&wnode, parent, nullptr, nullptr, 0, &wp)) != cudaSuccess)
        return cuda_check(c, e, "conditional WHILE node");
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    // handles of the IF nodes belong to the body graph that holds them
    cudaGraphConditionalHandle h_split, h_eval;
    if ((e = cudaGraphConditionalHandleCreate(&h_split, body, 0, cudaGraphCondAssignDefault)) != cudaSuccess ||
        (e = cudaGraphConditionalHandleCreate(&h_eval, body, 0, cudaGraphCondAssignDefault)) != cudaSuccess)
        return cuda_check(c, e, "conditional handle");
    const int eq9 = c->prm.eta_tot > 0.0;
    // capture with every launch on the capture stream, no event timing, no scratch growth
    const cudaStream_t user_stream = c->stream;
    const int prof0 = c->prof_level;
    int64_t launches0[TG_K_COUNT];
    for (int k = 0; k < TG_K_COUNT; ++k) launches0[k] = c->prof_launches[k];
    c->stream = g->cap_stream;
    c->prof_level = 0;
    c->capturing = true;
    auto restore = [&](tg_status r) {
        c->stream = user_stream;
        c->prof_level = prof0;
        c->capturing = false;
        for (int k = 0; k < TG_K_COUNT; ++k) c->prof_launches[k] = launches0[k];
        return r;
    };
    if ((st = capture_begin(c, g, body))) return restore(st);
    hold_sched<<<1, 1, 0, c->stream>>>(h, c->prm.k_max, eq9, h_loop, h_split, h_eval);
    if ((st = capture_end(c, g))) return restore(st);
    cudaGraphNode_t sched_node;
    size_t nn = 1;
    if ((e = cudaGraphGetNodes(body, &sched_node, &nn)) != cudaSuccess || nn != 1)
        return restore(set_err(c, TG_ERR_CUDA, "graph capture: scheduler node not found"));
    cudaGraphNode_t if_split, if_eval;
    cudaGraph_t split_body, eval_body;
    if ((st = add_if(c, body, &sched_node, &if_split, h_split, &split_body))) return restore(st);
    // split at level h->k: timesteps (calc), fast flags, scan, partition, sizes
    if ((st = capture_begin(c, g, split_body))) return restore(st);
    {
        ProfScope ps_(c, TG_K_HHS);
        hold_timestep<<<grid, 256, 0, c->stream>>>(h, L, s.a_old, s.a_cur, c->prm.eta * c->prm.eps, s.a_tot,
                                                   c->prm.eta_tot * c->prm.eps, s.dt);
        hold_flags<<<grid, 256, 0, c->stream>>>(h, L, s.dt, c->prm.dt_max, c->prm.k_max, flag);
    }
    st = exclusive_scan_u32(c, flag, pre, (int)N, &h->split_total, &h->cur_ns);
    if (st == TG_OK) {
        ProfScope ps_(c, TG_K_HHS);
        hold_partition<<<grid, 256, 0, c->stream>>>(h, L, flag, pre, s.rung);
        hold_split_finish<<<1, 1, 0, c->stream>>>(h);
    }
    tg_status st2 = capture_end(c, g);
    if (st || (st = st2)) return restore(st);
    for (int k = 0; k < TG_K_COUNT; ++k) {
        g->launches_split[k] = c->prof_launches[k] - launches0[k];
        launches0[k] = c->prof_launches[k];
    }
    // evaluation in flight with its kick (and drift after the first kick pair)
    if ((st = add_if(c, body, &if_split, &if_eval, h_eval, &eval_body))) return restore(st);
    if ((st = capture_begin(c, g, eval_body))) return restore(st);
    unsigned long long *stats = h->stats;
    {
        ProfScope ps_(c, TG_K_HHS);
        hold_frame<<<grid, 256, 0, c->stream>>>(h, L, c->hhs_pos, N, c->hhs_mass, xin, min, fin, de, cap_n);
    }
    st = fmm_eval_dev(c, de, g->caps, xin, min, fin, s.acc, stats);
    if (st == TG_OK) {
        ProfScope ps_(c, TG_K_HHS);
        hold_kick<<<grid, 256, 0, c->stream>>>(h, L, s.acc, cap_n, c->prm.dt_max, N, c->hhs_vel, s.a_old, s.a_cur,
                                               s.a_tot, eq9);
        hold_drift<<<grid, 256, 0, c->stream>>>(h, L, c->prm.dt_max, N, c->hhs_pos, c->hhs_vel);
    }
    st2 = capture_end(c, g);
    if (st || (st = st2)) return restore(st);
    for (int k = 0; k < TG_K_COUNT; ++k) g->launches_eval[k] = c->prof_launches[k] - launches0[k];
    restore(TG_OK);
    return TG_OK;
}

static void hold_record_capture(tg_ctx *c, HoldGraph *g, const Sched &s)
{
    g->epoch = c->alloc_epoch;
    g->prm = c->prm;
    g->tune = c->tune;
    g->n = s.n;
    g->bound[0] = c->hhs_pos;
    g->bound[1] = c->hhs_vel;
    g->bound[2] = const_cast<double *>(c->hhs_mass);
}

static tg_status hold_capture(tg_ctx *c, HoldGraph *g, Sched &s, const std::vector<Level> &lv, size_t per)
{
    tg_status st;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    g->exec = nullptr;
    g->graph = nullptr;
    cudaError_t e = cudaGraphCreate(&g->graph, 0);
    if (e != cudaSuccess) return cuda_check(c, e, "graph create");
    if ((st = hold_capture_into(c, g, s, lv, per, g->graph))) return st;
    if ((e = cudaGraphInstantiate(&g->exec, g->graph, 0)) != cudaSuccess) return cuda_check(c, e, "graph instantiate");
    hold_record_capture(c, g, s);
    return TG_OK;
}

static bool hold_stale(const tg_ctx *c, const HoldGraph *g, const Sched &s)
{
    return g->epoch != c->alloc_epoch || !same_capture_params(g->prm, c->prm) || g->tune.p2p_rows != c->tune.p2p_rows ||
           g->tune.m2l_blocks_per_sm != c->tune.m2l_blocks_per_sm || g->tune.m2l_form != c->tune.m2l_form ||
           g->n != s.n || g->bound[0] != c->hhs_pos || g->bound[1] != c->hhs_vel || g->bound[2] != c->hhs_mass;
}

// counters of a finished step into the context (launches: the scheduler every iteration, the bodies as
// often as they ran) and the time
static void hold_commit(tg_ctx *c, const HoldGraph *g, const HoldState &head)
{
    c->prof_launches[TG_K_HHS] += 1 + (int64_t)head.iterations;
    for (int k = 0; k < TG_K_COUNT; ++k)
        c->prof_launches[k] += g->launches_split[k] * (int64_t)head.splits + g->launches_eval[k] * (int64_t)head.evals;
    c->stats.evaluations += (int64_t)head.stats[0];
    c->stats.sink_forces += (int64_t)head.stats[1];
    c->stats.m2l_pairs += (int64_t)head.stats[2];
    c->stats.m2l_class_pairs += (int64_t)head.stats[3];
    c->stats.p2p_cell_pairs += (int64_t)head.stats[4];
    c->stats.cells += (int64_t)head.stats[5];
    c->stats.kdk_frames += (int64_t)head.stats[6];
    if ((int64_t)head.stats[7] > c->stats.max_rung) c->stats.max_rung = (int64_t)head.stats[7];
    c->hhs_time += c->prm.dt_max;
}

tg_status hhs_step_batched(tg_ctx *c)
{
    Sched s;
    tg_status st = make_sched(c, s);
    if (st) return st;
    if ((st = check_finite(c, s.n, c->hhs_pos, s.n, nullptr, c->hhs_mass))) return st;
    if (!c->hold) {
        c->hold = new (std::nothrow) HoldGraph();
        if (!c->hold) return set_err(c, TG_ERR_OOM, "batched step: host allocation failed");
        cudaError_t e = cudaStreamCreateWithFlags(&c->hold->cap_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocHost(&c->hold->h_read, 4096);
        if (e != cudaSuccess) {
            hold_graph_destroy(c);
            return cuda_check(c, e, "batched step setup");
        }
    }
    HoldGraph *g = c->hold;
    char *snap = nullptr;
    if ((st = snapshot_state(c, s, &snap))) return st;
    const tg_stats stats0 = c->stats;
    auto fail = [&](tg_status r) {
        restore_state(c, s, static_cast<const char *>(c->buf[B_SNAP].p));
        const int64_t regrow = c->stats.list_regrowths, syncs = c->stats.host_syncs;
        c->stats = stats0;
        c->stats.list_regrowths = regrow;
        c->stats.host_syncs = syncs;
        return r;
    };
    if ((st = level_buffers(c, s.n, s.lv, c->prm.k_max))) return fail(st);
    const size_t per = ((s.n * (2 * sizeof(int64_t) + 2 * sizeof(uint32_t) + 1) + 64) + 255) & ~(size_t)255;
    if (!g->sized || g->caps.n != (int)s.n) {
        if ((st = hold_size(c, s, g->caps))) return fail(st);
        g->sized = true;
    }
    for (int attempt = 0; attempt < 24; ++attempt) {
        if (!g->exec || hold_stale(c, g, s)) {
            if ((st = hold_capture(c, g, s, s.lv, per))) return fail(st);
            // the capture may have grown nothing, but a stale epoch must not trigger a second capture
            g->epoch = c->alloc_epoch;
        }
        HoldState *h = static_cast<HoldState *>(c->buf[B_HOLD].p);
        DevEval *de = static_cast<DevEval *>(c->buf[B_DEVEVAL].p);
        const LevelLayout L{reinterpret_cast<char *>(s.lv[0].sys), per, s.n};
        {
            ProfScope ps_(c, TG_K_HHS);
            hold_begin<<<grid_for(s.n, 256), 256, 0, c->stream>>>(h, de, L, s.n, hold_limit(c), c->debug_queue_hold);
        }
        cudaError_t e = cudaGraphLaunch(g->exec, c->stream);
        if (e != cudaSuccess) return fail(cuda_check(c, e, "batched step launch"));
        // the step's head counters and the overflow bits, read once
        unsigned long long *hr = g->h_read;
        cudaMemcpyAsync(hr, h, offsetof(HoldState, op), cudaMemcpyDeviceToHost, c->stream);
        cudaMemcpyAsync(hr + 64, &de->overflow, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
        if ((st = cuda_check(c, stream_sync(c), "batched step"))) return fail(st);
        HoldState head;
        std::memcpy(&head, hr, offsetof(HoldState, op));
        const uint32_t overflow = *reinterpret_cast<const uint32_t *>(hr + 64);
        if (head.status != 0)
            return fail(set_err(c, TG_ERR_TIMEOUT, "batched step: the device loop stopped after %llu iterations",
                                head.iterations));
        if (overflow) {
            // restore, grow what ran out, capture again and redo the step
            restore_state(c, s, static_cast<const char *>(c->buf[B_SNAP].p));
            c->stats.list_regrowths += 1;
            if (overflow & 1u) g->caps.cells = (int)std::min<int64_t>(INT32_MAX / 8, (int64_t)g->caps.cells * 4);
            if (overflow & 2u) g->caps.levels = std::min(c->prm.max_level, g->caps.levels + 4);
            if (overflow & 4u) {
                g->caps.front *= 4;
                g->caps.blocks *= 4;
                g->caps.p2p *= 4;
                g->caps.m2l_src *= 4;
            }
            if (g->exec) cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
            continue;
        }
        hold_commit(c, g, head);
        return TG_OK;
    }
    return fail(set_err(c, TG_ERR_CAPACITY, "batched step: buffers still too small after regrowth"));
}

// ------------------------------------------------------------------ ensemble of batched steps
// Several bound systems stepped by ONE graph launch: the graph holds each system's work-queue loop side
// by side (no edges between them), so every system keeps its own rung structure and small systems run
// side by side on the GPU.  Per system the step is transactional as in hhs_step_batched; a system whose
// buffers overflow is restored and redone alone (and the ensemble graph captured again next time).
void ensemble_destroy(tg_ctx *c)
{
    if (!c->hold || !c->hold->ens) return;
    EnsembleGraph *e = c->hold->ens;
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    delete e;
    c->hold->ens = nullptr;
}

tg_status ensemble_step(tg_ctx **cs, int count)
{
    tg_status st;
    tg_ctx *c0 = cs[0];
    // per member: buffers, finiteness (one wait for all), snapshot, level lists, capacities
    std::vector<Sched> sched(count);
    std::vector<size_t> per(count);
    for (int i = 0; i < count; ++i) {
        tg_ctx *c = cs[i];
        if ((st = make_sched(c, sched[i]))) return st;
        if (!c->hold) {
            c->hold = new (std::nothrow) HoldGraph();
            if (!c->hold) return set_err(c0, TG_ERR_OOM, "ensemble step: host allocation failed");
            cudaError_t e = cudaStreamCreateWithFlags(&c->hold->cap_stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaMallocHost(&c->hold->h_read, 4096);
            if (e != cudaSuccess) {
                hold_graph_destroy(c);
                return cuda_check(c0, e, "ensemble step setup");
            }
        }
        unsigned long long *bad = c->d_counters + 10;
        cudaMemsetAsync(bad, 0, sizeof(unsigned long long), c0->stream);
        count_nonfinite<<<grid_for(sched[i].n, 256, 2 * c->num_sms), 256, 0, c0->stream>>>(
            c->hhs_pos, sched[i].n, nullptr, sched[i].n, c->hhs_mass, bad);
        cudaMemcpyAsync(c->hold->h_read + 65, bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c0->stream);
    }
    if ((st = cuda_check(c0, stream_sync(c0), "ensemble finiteness check"))) return st;
    for (int i = 0; i < count; ++i)
        if (cs[i]->hold->h_read[65])
            return set_err(c0, TG_ERR_NONFINITE, "ensemble member %d has a non-finite position or mass", i);
    for (int i = 0; i < count; ++i) {
        tg_ctx *c = cs[i];
        char *snap;
        if ((st = snapshot_state(c, sched[i], &snap)) || (st = level_buffers(c, sched[i].n, sched[i].lv, c->prm.k_max)))
            return st;
        per[i] = ((sched[i].n * (2 * sizeof(int64_t) + 2 * sizeof(uint32_t) + 1) + 64) + 255) & ~(size_t)255;
        if (!c->hold->sized || c->hold->caps.n != (int)sched[i].n) {
            if ((st = hold_size(c, sched[i], c->hold->caps))) return st;
            c->hold->sized = true;
        }
    }
    // the ensemble graph: captured again when the members or any member's buffers or parameters changed
    EnsembleGraph *eg = c0->hold->ens;
    bool stale = !eg || eg->members != std::vector<tg_ctx *>(cs, cs + count);
    for (int i = 0; i < count && !stale; ++i) {
        const tg_ctx *c = cs[i];
        stale = eg->epochs[i] != c->alloc_epoch || !same_capture_params(eg->prms[i], c->prm) ||
                eg->tunes[i].p2p_rows != c->tune.p2p_rows || eg->tunes[i].m2l_blocks_per_sm != c->tune.m2l_blocks_per_sm ||
                eg->tunes[i].m2l_form != c->tune.m2l_form || eg->bound[3 * i] != c->hhs_pos ||
                eg->bound[3 * i + 1] != c->hhs_vel || eg->bound[3 * i + 2] != c->hhs_mass;
    }
    if (stale) {
        ensemble_destroy(c0);
        eg = c0->hold->ens = new (std::nothrow) EnsembleGraph();
        if (!eg) return set_err(c0, TG_ERR_OOM, "ensemble step: host allocation failed");
        eg->members.assign(cs, cs + count);
        cudaError_t e = cudaGraphCreate(&eg->graph, 0);
        if (e != cudaSuccess) return cuda_check(c0, e, "ensemble graph create");
        for (int i = 0; i < count; ++i) {
            if ((st = hold_capture_into(cs[i], cs[i]->hold, sched[i], sched[i].lv, per[i], eg->graph))) {
                ensemble_destroy(c0);
                return st;
            }
        }
        if ((e = cudaGraphInstantiate(&eg->exec, eg->graph, 0)) != cudaSuccess) {
            ensemble_destroy(c0);
            return cuda_check(c0, e, "ensemble graph instantiate");
        }
        for (int i = 0; i < count; ++i) {
            const tg_ctx *c = cs[i];
            eg->epochs.push_back(c->alloc_epoch);
            eg->prms.push_back(c->prm);
            eg->tunes.push_back(c->tune);
            eg->bound.push_back(c->hhs_pos);
            eg->bound.push_back(c->hhs_vel);
            eg->bound.push_back(c->hhs_mass);
        }
    }
    // start every member's queue, one launch for all loops, read every member's counters with one wait
    for (int i = 0; i < count; ++i) {
        tg_ctx *c = cs[i];
        HoldState *h = static_cast<HoldState *>(c->buf[B_HOLD].p);
        DevEval *de = static_cast<DevEval *>(c->buf[B_DEVEVAL].p);
        const LevelLayout L{reinterpret_cast<char *>(sched[i].lv[0].sys), per[i], sched[i].n};
        ProfScope ps_(c, TG_K_HHS);
        hold_begin<<<grid_for(sched[i].n, 256), 256, 0, c0->stream>>>(h, de, L, sched[i].n, hold_limit(c),
                                                                       c->debug_queue_hold);
    }
    cudaError_t e = cudaGraphLaunch(eg->exec, c0->stream);
    if (e != cudaSuccess) return cuda_check(c0, e, "ensemble launch");
    for (int i = 0; i < count; ++i) {
        tg_ctx *c = cs[i];
        unsigned long long *hr = c->hold->h_read;
        cudaMemcpyAsync(hr, c->buf[B_HOLD].p, offsetof(HoldState, op), cudaMemcpyDeviceToHost, c0->stream);
        cudaMemcpyAsync(hr + 64, &static_cast<DevEval *>(c->buf[B_DEVEVAL].p)->overflow, sizeof(uint32_t),
                        cudaMemcpyDeviceToHost, c0->stream);
    }
    if ((st = cuda_check(c0, stream_sync(c0), "ensemble step"))) return st;
    tg_status first = TG_OK;
    for (int i = 0; i < count; ++i) {
        tg_ctx *c = cs[i];
        HoldState head;
        std::memcpy(&head, c->hold->h_read, offsetof(HoldState, op));
        const uint32_t overflow = *reinterpret_cast<const uint32_t *>(c->hold->h_read + 64);
        if (head.status != 0) {
            restore_state(c, sched[i], static_cast<const char *>(c->buf[B_SNAP].p));
            if (!first) first = set_err(c0, TG_ERR_TIMEOUT, "ensemble member %d: the device loop stopped after %llu "
                                                            "iterations", i, head.iterations);
            continue;
        }
        if (overflow) {
            // restore and redo this member alone; the batched step grows its buffers (and the ensemble graph
            // is captured again on the next call, since the member's buffers moved)
            restore_state(c, sched[i], static_cast<const char *>(c->buf[B_SNAP].p));
            st = hhs_step_batched(c);
            if (st && !first) first = set_err(c0, st, "ensemble member %d: %s", i, c->err.msg.c_str());
            continue;
        }
        hold_commit(c, c->hold, head);
    }
    return first;
}

__global__ void timestep_rungs(int64_t n, const double *a_old, const double *a_cur, double eta_eps, const double *a_tot,
                               double eta_tot_eps, double dt_max, int k_max, double *dt, int32_t *rung)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double d = timestep_of(a_old[i], a_cur[i], eta_eps, a_tot, eta_tot_eps, i);
        int k = 0;
        while (k < k_max && !(d >= ldexp(dt_max, -k))) ++k;
        dt[i] = d;
        rung[i] = k;
    }
}

tg_status timesteps(tg_ctx *c, int64_t n, const double *a_old, const double *a_cur, const double *a_tot, double *dt,
                    int32_t *rung)
{
    {
        ProfScope ps_(c, TG_K_HHS);
        timestep_rungs<<<grid_for(n, 256), 256, 0, c->stream>>>(n, a_old, a_cur, c->prm.eta * c->prm.eps, a_tot,
                                                              c->prm.eta_tot * c->prm.eps, c->prm.dt_max, c->prm.k_max,
                                                              dt, rung);
    }
    return cuda_check(c, cudaGetLastError(), "timesteps");
}

// ------------------------------------------------------------------ traditional individual timesteps
// The comparison integrator of Sec. 2.3: block steps dt_max / 2^rung, kick-drift-kick per particle
// over its own step.  At the end of a particle's step it drifts the whole step, gets its force from
// all masses at their stored positions (inactive particles are not synchronised), closes the step
// with a half kick, takes a new rung from dt_i = sqrt(eta eps / |a_i|) deepened until the next step
// starts on a multiple of itself, and opens it with a half kick.  Time runs on a grid of 2^k_max
// substeps per rung-0 step; end[i] is the substep where particle i's step ends.  The float64
// operations are written out in a fixed order with explicit rounding (no contraction), so that the
// rungs are reproducible bit for bit.
__device__ __forceinline__ double trad_amag(double ax, double ay, double az)
{
    return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)), __dmul_rn(az, az)));
}

__device__ __forceinline__ int trad_rung_of(double amag, double eta_eps, double dt_max, int k_max, int64_t m)
{
    const double d = (amag > 0.0) ? sqrt(__ddiv_rn(eta_eps, amag)) : INFINITY;
    int k = 0;
    while (k < k_max && !(d >= ldexp(dt_max, -k))) ++k;
    int ra = 0;   // a step starting at substep m must start on a multiple of itself
    if (m != 0) {
        int tz = 0;
        while (tz < k_max && ((m >> tz) & 1) == 0) ++tz;
        ra = k_max - tz;
    }
    return k > ra ? k : ra;
}

__global__ void trad_first_rungs(int64_t n, const double *acc, double eta_eps, double dt_max, int k_max, int32_t *rung)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        rung[i] = trad_rung_of(trad_amag(acc[i], acc[n + i], acc[2 * n + i]), eta_eps, dt_max, k_max, 0);
}

// opening half kicks at the start of a rung-0 step
__global__ void trad_open(int64_t n, const double *acc, const int32_t *rung, double dt_max, int k_max, double *vel,
                          int64_t *end, unsigned long long *max_rung)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double h = 0.5 * ldexp(dt_max, -rung[i]);
#pragma unroll
        for (int d = 0; d < 3; ++d) vel[d * n + i] = __dadd_rn(vel[d * n + i], __dmul_rn(acc[d * n + i], h));
        end[i] = (int64_t)1 << (k_max - rung[i]);
        atomicMax(max_rung, (unsigned long long)rung[i]);
    }
}

// next boundary: the smallest end (out[0], atomicMin) and how many steps end there (out[1])
__global__ void trad_next_min(int64_t n, const int64_t *end, unsigned long long *out)
{
    unsigned long long mn = ~0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        mn = min(mn, (unsigned long long)end[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0) atomicMin(out, mn);
}
__global__ void trad_next_count(int64_t n, const int64_t *end, unsigned long long *out)
{
    const unsigned long long t = out[0];
    unsigned long long c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += (unsigned long long)end[i] == t;
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out + 1, c);
}

__global__ void trad_drift(int64_t n, const int64_t *end, const unsigned long long *tnow, const int32_t *rung,
                           double dt_max, double *pos, const double *vel)
{
    const int64_t t = (int64_t)tnow[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (end[i] != t) continue;
        const double dt = ldexp(dt_max, -rung[i]);
#pragma unroll
        for (int d = 0; d < 3; ++d) pos[d * n + i] = __dadd_rn(pos[d * n + i], __dmul_rn(vel[d * n + i], dt));
    }
}

__global__ void trad_close(int64_t n, int64_t *end, const unsigned long long *tnow, int64_t m_end,
                           const double *acc_new, double *acc, int32_t *rung, double *vel, double eta_eps,
                           double dt_max, int k_max, unsigned long long *max_rung)
{
    const int64_t t = (int64_t)tnow[0];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (end[i] != t) continue;
        const double a[3] = {acc_new[i], acc_new[n + i], acc_new[2 * n + i]};
        const double h = 0.5 * ldexp(dt_max, -rung[i]);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            vel[d * n + i] = __dadd_rn(vel[d * n + i], __dmul_rn(a[d], h));   // closing half kick
            acc[d * n + i] = a[d];
        }
        const int r = trad_rung_of(trad_amag(a[0], a[1], a[2]), eta_eps, dt_max, k_max, t == m_end ? 0 : t);
        rung[i] = r;
        if (t < m_end) {
            const double h2 = 0.5 * ldexp(dt_max, -r);
#pragma unroll
            for (int d = 0; d < 3; ++d) vel[d * n + i] = __dadd_rn(vel[d * n + i], __dmul_rn(a[d], h2));
            end[i] = t + ((int64_t)1 << (k_max - r));
            atomicMax(max_rung, (unsigned long long)r);
        }
    }
}

tg_status trad_init(tg_ctx *c)
{
    tg_status st;
    const int64_t n = c->hhs_n;
    double *acc;
    int32_t *rung;
    if ((st = ensure_t(c, B_TRAD_ACC, 3 * n, &acc)) || (st = ensure_t(c, B_HHS_RUNG, n, &rung))) return st;
    if ((st = fmm_eval(c, (int)n, c->hhs_pos, n, nullptr, c->hhs_mass, nullptr, acc, n, nullptr, false))) return st;
    {
        ProfScope ps_(c, TG_K_HHS);
        trad_first_rungs<<<grid_for(n, 256), 256, 0, c->stream>>>(n, acc, c->prm.eta * c->prm.eps, c->prm.dt_max,
                                                                  c->prm.k_max, rung);
    }
    c->hhs_time = 0.0;
    return cuda_check(c, cudaGetLastError(), "traditional init");
}

tg_status trad_step(tg_ctx *c)
{
    tg_status st;
    const int64_t n = c->hhs_n;
    const int K = c->prm.k_max;
    const int64_t m_end = (int64_t)1 << K;
    const double eta_eps = c->prm.eta * c->prm.eps, dt_max = c->prm.dt_max;
    double *acc, *acc_new;
    int32_t *rung;
    int64_t *end;
    unsigned long long *ctr = c->d_counters + 16;   // [0] next boundary, [1] steps ending there, [2] deepest rung
    if ((st = ensure_t(c, B_TRAD_ACC, 3 * n, &acc)) || (st = ensure_t(c, B_HHS_RUNG, n, &rung)) ||
        (st = ensure_t(c, B_TRAD_END, n, &end)) || (st = ensure_t(c, B_SUB_ACC, 3 * n, &acc_new)))
        return st;
    const int g = grid_for(n, 256);
    cudaMemsetAsync(ctr + 2, 0, sizeof(unsigned long long), c->stream);
    {
        ProfScope ps_(c, TG_K_HHS);
        trad_open<<<g, 256, 0, c->stream>>>(n, acc, rung, dt_max, K, c->hhs_vel, end, ctr + 2);
    }
    for (;;) {
        const unsigned long long init[2] = {~0ull, 0ull};
        cudaMemcpyAsync(ctr, init, sizeof(init), cudaMemcpyHostToDevice, c->stream);
        {
            ProfScope ps_(c, TG_K_HHS);
            trad_next_min<<<g, 256, 0, c->stream>>>(n, end, ctr);
            trad_next_count<<<g, 256, 0, c->stream>>>(n, end, ctr);
        }
        unsigned long long *h = reinterpret_cast<unsigned long long *>(c->h_pinned + 48);
        cudaMemcpyAsync(h, ctr, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
        cudaError_t e = stream_sync(c);
        if (e != cudaSuccess) return cuda_check(c, e, "traditional step");
        const int64_t t = (int64_t)h[0], na = (int64_t)h[1];
        if (t > m_end || na <= 0) return set_err(c, TG_ERR_STATE, "traditional step: no boundary found");
        {
            ProfScope ps_(c, TG_K_HHS);
            trad_drift<<<g, 256, 0, c->stream>>>(n, end, ctr, rung, dt_max, c->hhs_pos, c->hhs_vel);
        }
        // forces on the active particles from all masses (the whole system is evaluated)
        if ((st = fmm_eval(c, (int)n, c->hhs_pos, n, nullptr, c->hhs_mass, nullptr, acc_new, n, nullptr, false)))
            return st;
        c->stats.sink_forces -= n - na;   // count the active particles only
        {
            ProfScope ps_(c, TG_K_HHS);
            trad_close<<<g, 256, 0, c->stream>>>(n, end, ctr, m_end, acc_new, acc, rung, c->hhs_vel, eta_eps, dt_max,
                                                 K, ctr + 2);
        }
        if ((st = cuda_check(c, cudaGetLastError(), "traditional step"))) return st;
        if (t == m_end) break;
    }
    unsigned long long *h = reinterpret_cast<unsigned long long *>(c->h_pinned + 48);
    cudaMemcpyAsync(h, ctr + 2, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
    if ((st = cuda_check(c, stream_sync(c), "traditional step"))) return st;
    if ((int64_t)h[0] > c->stats.max_rung) c->stats.max_rung = (int64_t)h[0];
    c->hhs_time += dt_max;
    return TG_OK;
}

// ------------------------------------------------------------------ diagnostics (float64)
// out: P (3), L (3), kinetic, potential sum m phi / 2
__global__ void diag_partial(int64_t n, const double *pos, const double *vel, const double *m, const double *pot,
                             double *partial)
{
    double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = pos[i], y = pos[n + i], z = pos[2 * n + i];
        const double vx = vel[i], vy = vel[n + i], vz = vel[2 * n + i], mi = m[i];
        q[0] += mi * vx;
        q[1] += mi * vy;
        q[2] += mi * vz;
        q[3] += mi * (y * vz - z * vy);
        q[4] += mi * (z * vx - x * vz);
        q[5] += mi * (x * vy - y * vx);
        q[6] += 0.5 * mi * (vx * vx + vy * vy + vz * vz);
        q[7] += 0.5 * mi * pot[i];
    }
    __shared__ double sh[8][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        double v = warp_sum(q[k]);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        double r = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[threadIdx.x][w];
        partial[blockIdx.x * 8 + threadIdx.x] = r;
    }
}

tg_status hhs_diagnostics(tg_ctx *c, double out[8])
{
    tg_status st;
    const int64_t n = c->hhs_n;
    double *pot, *acc, *partial;
    const int nb = 64;
    if ((st = ensure_t(c, B_DIAG_POT, n, &pot)) || (st = ensure_t(c, B_DIAG_ACC, 3 * n, &acc)) ||
        (st = ensure_t(c, B_RED, nb * 8, &partial)))
        return st;
    if ((st = fmm_eval(c, (int)n, c->hhs_pos, n, nullptr, c->hhs_mass, nullptr, acc, n, pot, false))) return st;
    {
        ProfScope ps_(c, TG_K_OTHER);
        diag_partial<<<nb, 256, 0, c->stream>>>(n, c->hhs_pos, c->hhs_vel, c->hhs_mass, pot, partial);
    }
    std::vector<double> h(nb * 8);
    cudaError_t e = cudaMemcpyAsync(h.data(), partial, sizeof(double) * nb * 8, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = stream_sync(c);
    if (e != cudaSuccess) return cuda_check(c, e, "diagnostics");
    double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < nb; ++b)
        for (int k = 0; k < 8; ++k) q[k] += h[b * 8 + k];
    for (int k = 0; k < 6; ++k) out[k] = q[k];
    out[6] = q[6] + q[7];
    out[7] = c->hhs_time;
    return TG_OK;
}

}  // namespace tg
