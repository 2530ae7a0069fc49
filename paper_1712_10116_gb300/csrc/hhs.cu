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
static tg_status snapshot_state(tg_ctx *c, const Sched &s, char **snap)
{
    const size_t n = (size_t)s.n;
    tg_status st = ensure_t(c, B_SNAP, n * (9 * sizeof(double) + sizeof(int32_t)), snap);
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

tg_status hhs_step(tg_ctx *c)
{
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
