// m2l.cu -- launchers of the mutual M2L kernels (Sec. 2.1): float32 fixed-order block kernels for
// p <= 6 (harmonic contraction set for the Wendland kernel, full set for Plummer softening), the
// generic kernel otherwise and in float64 up to the table order, high_order.cu above it.  Its own translation unit, so that the large
// generated contractions compile in parallel with the rest.
#include <algorithm>

#include "tg_common.cuh"
#include "m2l_sym.cuh"

namespace tg {

// zero n (+ extra) words, n from the device when dn is given (dn[0] + extra)
__global__ void zero_u32(uint32_t *p, int n, const int *dn, int extra)
{
    if (dn) n = dn[0] + extra;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0u;
}


// The walk's blocks partitioned for m2l_blocks_f32: multi-row blocks first, one-row blocks at the end
// (counts in *pcnt, on the device).  nblocks: the count, or the capacity with dnb the device count.
static tg_status m2l_partition_blocks(tg_ctx *c, const M2LBlock *blocks, int64_t nblocks,
                                      const unsigned long long *dnb, M2LBlock **part, unsigned long long **pcnt)
{
    tg_status st;
    if ((st = ensure_t(c, B_M2L_PART, (size_t)std::max<int64_t>(nblocks, 1), part)) ||
        (st = ensure_t(c, B_M2L_PCNT, 2, pcnt)))
        return st;
    ProfScope ps_(c, TG_K_M2L);
    cudaMemsetAsync(*pcnt, 0, 2 * sizeof(unsigned long long), c->stream);
    if (nblocks > 0)
        m2l_partition<<<dnb ? c->num_sms * 8 : grid_for(nblocks, 256, c->num_sms * 8), 256, 0, c->stream>>>(
            blocks, nblocks, dnb, *part, nblocks, *pcnt);
    return cuda_check(c, cudaGetLastError(), "m2l partition");
}

// Directed M2L lists from the walk's blocks: per cell the count of its sources (cnt, zeroed first), their
// offsets (exclusive scan of cnt) and the sources themselves (src, `cap` entries).
// dncell / dnb: device counts (batched path), else the host values.
static tg_status m2l_lists(tg_ctx *c, const TreeView &t, const M2LBlock *blocks, int64_t nblocks, int ncell,
                           uint32_t *cnt, uint32_t *off, uint32_t *fill, uint32_t *src, uint64_t cap,
                           const unsigned long long *dnb, const int *dncell)
{
    tg_status st;
    const int g = c->num_sms * 8;
    {
        ProfScope ps_(c, TG_K_M2L);
        zero_u32<<<g, 256, 0, c->stream>>>(cnt, ncell, dncell, 0);
        zero_u32<<<g, 256, 0, c->stream>>>(fill, ncell, dncell, 0);
        m2l_list_count<<<g, 256, 0, c->stream>>>(t, blocks, nblocks, cnt, dnb);
    }
    if ((st = exclusive_scan_u32(c, cnt, off, ncell, nullptr, dncell))) return st;
    {
        ProfScope ps_(c, TG_K_M2L);
        m2l_list_fill<<<g, 256, 0, c->stream>>>(t, blocks, nblocks, off, fill, src, cap, dnb);
    }
    return cuda_check(c, cudaGetLastError(), "m2l lists");
}

template <int P>
static void m2l_directed_launch(tg_ctx *c, const TreeView &t, const uint32_t *off, const uint32_t *cnt,
                                const uint32_t *src, uint64_t cap, const float *Mr, float *Lr, int ncpr, bool masked,
                                bool pot, const DevEval *de)
{
    const int grid = c->num_sms * c->tune.m2l_blocks_per_sm;
#define TG_DIR(MK, PT, DE) m2l_directed_h<P, MK, PT><<<grid, 128, 0, c->stream>>>(t, off, cnt, src, cap, Mr, Lr, ncpr, DE, c->d_counters + 11)
    if (de) {   // batched: both class counts launched, the other one returns at once
        TG_DIR(true, false, de);
        TG_DIR(false, false, de);
    } else if (masked) {
        if (pot) TG_DIR(true, true, nullptr);
        else TG_DIR(true, false, nullptr);
    } else {
        if (pot) TG_DIR(false, true, nullptr);
        else TG_DIR(false, false, nullptr);
    }
#undef TG_DIR
}

// Harmonic set (G = -1/|d|, P <= 6): fold the moments, contract the reduced sets into Lr, complete L.
template <int P>
static tg_status m2l_f32_harmonic(tg_ctx *c, const TreeView &t, const M2LBlock *blocks, int64_t nblocks, const float *Ms,
                                  float *L, int ncp, bool masked, bool pot, int grid, const uint32_t *fpre)
{
    if (c->tune.m2l_form == 1) {
        // directed by target cell
        constexpr int NH = M2LGenH<P>::NC;
        const int ncpr = (NH + 3) & ~3;
        const int ncell = t.ncell;
        const int64_t rows = (int64_t)ncell * 2;
        const uint64_t cap = 2ull * (uint64_t)c->last_nm2l + 16;
        float *Mr, *Lr;
        uint32_t *cnt, *off, *fill, *src;
        tg_status st;
        if ((st = ensure_t(c, B_MOMH, (size_t)rows * ncpr, &Mr)) || (st = ensure_t(c, B_LOCH, (size_t)rows * ncpr, &Lr)) ||
            (st = ensure_t(c, B_M2L_CNT, (size_t)ncell, &cnt)) || (st = ensure_t(c, B_M2L_OFF, (size_t)ncell, &off)) ||
            (st = ensure_t(c, B_M2L_FILL, (size_t)ncell, &fill)) || (st = ensure_t(c, B_M2L_SRC, cap, &src)))
            return st;
        if ((st = m2l_lists(c, t, blocks, nblocks, ncell, cnt, off, fill, src, cap, nullptr, nullptr))) return st;
        ProfScope ps_(c, TG_K_M2L);
        m2l_reduce_moments_h<P><<<grid_for(rows, 128), 128, 0, c->stream>>>(rows, Ms, ncp, Mr, ncpr, nullptr);
        cudaMemsetAsync(Lr, 0, sizeof(float) * (size_t)rows * ncpr, c->stream);
        m2l_directed_launch<P>(c, t, off, cnt, src, cap, Mr, Lr, ncpr, masked, pot, nullptr);
        m2l_complete_locals_h<P><<<grid_for(rows, 128), 128, 0, c->stream>>>(rows, Lr, ncpr, L, ncp, nullptr);
        return cuda_check(c, cudaGetLastError(), "m2l launch (directed)");
    }
    constexpr int NH = M2LGenH<P>::NC;
    const int ncpr = (NH + 3) & ~3;
    const int64_t rows = (int64_t)t.ncell * 2;
    float *Mr, *Lr;
    M2LBlock *part;
    unsigned long long *pcnt;
    tg_status st;
    if ((st = ensure_t(c, B_MOMH, (size_t)rows * ncpr, &Mr)) || (st = ensure_t(c, B_LOCH, (size_t)rows * ncpr, &Lr)))
        return st;
    if ((st = m2l_partition_blocks(c, blocks, nblocks, nullptr, &part, &pcnt))) return st;
    ProfScope ps_(c, TG_K_M2L);
    m2l_reduce_moments_h<P><<<grid_for(rows, 128), 128, 0, c->stream>>>(rows, Ms, ncp, Mr, ncpr, nullptr);
    cudaMemsetAsync(Lr, 0, sizeof(float) * (size_t)rows * ncpr, c->stream);
    using G = M2LHarm<P>;
#define TG_M2L_H(MK, PT)                                                                                          \
    do {                                                                                                          \
        m2l_blocks_f32<G, MK, PT><<<grid, 128, 0, c->stream>>>(t, part, nblocks, pcnt, Mr, Lr, ncpr, 0.f, 0, nullptr, \
                                                               nullptr, 0.0, fpre, c->d_counters + 11);            \
    } while (0)
    if (masked) {
        if (pot) TG_M2L_H(true, true);
        else TG_M2L_H(true, false);
    } else {
        if (pot) TG_M2L_H(false, true);
        else TG_M2L_H(false, false);
    }
#undef TG_M2L_H
    m2l_complete_locals_h<P><<<grid_for(rows, 128), 128, 0, c->stream>>>(rows, Lr, ncpr, L, ncp, nullptr);
    return cuda_check(c, cudaGetLastError(), "m2l launch");
}

tg_status launch_m2l_f32(tg_ctx *c, const TreeView &t, const M2LBlock *blocks, int64_t nblocks, const float *Ms,
                         float *L, int p, int nc, int ncp, bool masked, bool pot, const uint32_t *fpre)
{
    const int plummer = c->prm.kernel == TG_KERNEL_PLUMMER;
    const float eoL = (float)ldexp(c->prm.eps, -c->walk_log2L);
    if (p > TG_PMAX) return launch_m2l_hi<float>(c, t, blocks, nblocks, Ms, L, p, nc, ncp, masked, pot);
    const int grid = grid_for(nblocks * 32, 128, c->num_sms * c->tune.m2l_blocks_per_sm);
    // Wendland C2: the walk's eps gap rule leaves every M2L pair at r >= eps, where G = -1/r is harmonic
    if (!plummer && p >= 1 && p <= 6) {
        switch (p) {
        case 1: return m2l_f32_harmonic<1>(c, t, blocks, nblocks, Ms, L, ncp, masked, pot, grid, fpre);
        case 2: return m2l_f32_harmonic<2>(c, t, blocks, nblocks, Ms, L, ncp, masked, pot, grid, fpre);
        case 3: return m2l_f32_harmonic<3>(c, t, blocks, nblocks, Ms, L, ncp, masked, pot, grid, fpre);
        case 4: return m2l_f32_harmonic<4>(c, t, blocks, nblocks, Ms, L, ncp, masked, pot, grid, fpre);
        case 5: return m2l_f32_harmonic<5>(c, t, blocks, nblocks, Ms, L, ncp, masked, pot, grid, fpre);
        default: return m2l_f32_harmonic<6>(c, t, blocks, nblocks, Ms, L, ncp, masked, pot, grid, fpre);
        }
    }
    M2LBlock *part = nullptr;
    unsigned long long *pcnt = nullptr;
    if (p <= 6) {
        tg_status st;
        if ((st = m2l_partition_blocks(c, blocks, nblocks, nullptr, &part, &pcnt))) return st;
    }
    ProfScope ps_(c, TG_K_M2L);
#define TG_M2L_F32_(PP, MK, PT)                                                                                   \
    do {                                                                                                          \
        m2l_blocks_f32<M2LFull<PP>, MK, PT><<<grid, 128, 0, c->stream>>>(t, part, nblocks, pcnt, Ms, L, ncp, eoL,  \
                                                                         plummer, nullptr, nullptr, 0.0, fpre,      \
                                                                         c->d_counters + 11);                       \
    } while (0)
#define TG_M2L_F32(PP)                                                                                            \
    case PP:                                                                                                      \
        if (masked) { if (pot) TG_M2L_F32_(PP, true, true); else TG_M2L_F32_(PP, true, false); }                   \
        else { if (pot) TG_M2L_F32_(PP, false, true); else TG_M2L_F32_(PP, false, false); }                        \
        break;
    switch (p) {
        TG_M2L_F32(1)
        TG_M2L_F32(2)
        TG_M2L_F32(3)
        TG_M2L_F32(4)
        TG_M2L_F32(5)
        TG_M2L_F32(6)
    default:
        if (masked) m2l_blocks_generic<float, true><<<grid, 128, 0, c->stream>>>(t, blocks, nblocks, Ms, L, p, nc, ncp,
                                                                                ldexp(c->prm.eps, -c->walk_log2L), plummer);
        else m2l_blocks_generic<float, false><<<grid, 128, 0, c->stream>>>(t, blocks, nblocks, Ms, L, p, nc, ncp,
                                                                          ldexp(c->prm.eps, -c->walk_log2L), plummer);
    }
#undef TG_M2L_F32
#undef TG_M2L_F32_
    return cuda_check(c, cudaGetLastError(), "m2l launch");
}

// ------------------------------------------------------------------ batched path (sizes on the device)
// directed lists over capacity: flag the step (the fill and the kernel stay inside the buffer)
__global__ void m2l_list_check(const uint32_t *off, const uint32_t *cnt, DevEval *de, uint64_t cap)
{
    const int last = de->ncell - 1;
    if ((uint64_t)off[last] + cnt[last] > cap) de->overflow |= 4u;
}

template <int P>
static tg_status m2l_f32_dev_p(tg_ctx *c, const TreeView &t, const DevEval *de, const Geom *gp, const M2LBlock *blocks,
                               const unsigned long long *dnb, int64_t cap_blocks, const float *Ms, float *L, int ncp,
                               float *Mr, float *Lr, int ncpr, int rows_cap, int grid, size_t cap_src,
                               const uint32_t *fpre)
{
    const int plummer = c->prm.kernel == TG_KERNEL_PLUMMER;
    const int g = grid_for(rows_cap, 128);
    if (!plummer && c->tune.m2l_form == 1) {
        const int cap_cells = rows_cap / 2;
        uint32_t *cnt, *off, *fill, *src;
        tg_status st;
        if ((st = ensure_t(c, B_M2L_CNT, (size_t)cap_cells, &cnt)) ||
            (st = ensure_t(c, B_M2L_OFF, (size_t)cap_cells, &off)) ||
            (st = ensure_t(c, B_M2L_FILL, (size_t)cap_cells, &fill)) || (st = ensure_t(c, B_M2L_SRC, cap_src, &src)))
            return st;
        if ((st = m2l_lists(c, t, blocks, cap_blocks, cap_cells, cnt, off, fill, src, cap_src, dnb, &de->ncell)))
            return st;
        ProfScope ps_(c, TG_K_M2L);
        m2l_list_check<<<1, 1, 0, c->stream>>>(off, cnt, const_cast<DevEval *>(de), cap_src);
        m2l_reduce_moments_h<P><<<g, 128, 0, c->stream>>>(rows_cap, Ms, ncp, Mr, ncpr, &de->rows);
        zero_rows_f32<<<c->num_sms * 4, 256, 0, c->stream>>>(Lr, &de->rows, ncpr);
        m2l_directed_launch<P>(c, t, off, cnt, src, cap_src, Mr, Lr, ncpr, true, false, de);
        m2l_complete_locals_h<P><<<g, 128, 0, c->stream>>>(rows_cap, Lr, ncpr, L, ncp, &de->rows);
        return TG_OK;
    }
    M2LBlock *part;
    unsigned long long *pcnt;
    tg_status st;
    if ((st = m2l_partition_blocks(c, blocks, cap_blocks, dnb, &part, &pcnt))) return st;
    ProfScope ps_(c, TG_K_M2L);
    if (!plummer) {
        // harmonic set: fold, contract (the launch for the other class count returns at once), complete
        using G = M2LHarm<P>;
        m2l_reduce_moments_h<P><<<g, 128, 0, c->stream>>>(rows_cap, Ms, ncp, Mr, ncpr, &de->rows);
        zero_rows_f32<<<c->num_sms * 4, 256, 0, c->stream>>>(Lr, &de->rows, ncpr);
        m2l_blocks_f32<G, true, false><<<grid, 128, 0, c->stream>>>(t, part, cap_blocks, pcnt, Mr, Lr, ncpr, 0.f, 0, de,
                                                                    gp, c->prm.eps, fpre, c->d_counters + 11);
        m2l_blocks_f32<G, false, false><<<grid, 128, 0, c->stream>>>(t, part, cap_blocks, pcnt, Mr, Lr, ncpr, 0.f, 0, de,
                                                                     gp, c->prm.eps, fpre, c->d_counters + 11);
        m2l_complete_locals_h<P><<<g, 128, 0, c->stream>>>(rows_cap, Lr, ncpr, L, ncp, &de->rows);
    } else {
        using G = M2LFull<P>;
        m2l_blocks_f32<G, true, false><<<grid, 128, 0, c->stream>>>(t, part, cap_blocks, pcnt, Ms, L, ncp, 0.f, 1, de,
                                                                    gp, c->prm.eps, fpre, c->d_counters + 11);
        m2l_blocks_f32<G, false, false><<<grid, 128, 0, c->stream>>>(t, part, cap_blocks, pcnt, Ms, L, ncp, 0.f, 1, de,
                                                                     gp, c->prm.eps, fpre, c->d_counters + 11);
    }
    return TG_OK;
}

tg_status launch_m2l_f32_dev(tg_ctx *c, const TreeView &t, const DevEval *de, const Geom *gp, const M2LBlock *blocks,
                             const unsigned long long *dnb, int64_t cap_blocks, const float *Ms, float *L, int p,
                             int ncp, int cap_cells, size_t cap_src, const uint32_t *fpre)
{
    if (p < 1 || p > 6) return set_err(c, TG_ERR_ARG, "batched M2L needs 1 <= p <= 6");
    static const int nh[7] = {0, 4, 9, 16, 25, 36, 49};   // (p + 1)^2 harmonic coefficients
    const int ncpr = (nh[p] + 3) & ~3;
    const int rows_cap = 2 * cap_cells;
    float *Mr = nullptr, *Lr = nullptr;
    tg_status st;
    if (c->prm.kernel != TG_KERNEL_PLUMMER &&
        ((st = ensure_t(c, B_MOMH, (size_t)rows_cap * ncpr, &Mr)) || (st = ensure_t(c, B_LOCH, (size_t)rows_cap * ncpr, &Lr))))
        return st;
    const int grid = c->num_sms * c->tune.m2l_blocks_per_sm;
    switch (p) {
    case 1: st = m2l_f32_dev_p<1>(c, t, de, gp, blocks, dnb, cap_blocks, Ms, L, ncp, Mr, Lr, ncpr, rows_cap, grid, cap_src, fpre); break;
    case 2: st = m2l_f32_dev_p<2>(c, t, de, gp, blocks, dnb, cap_blocks, Ms, L, ncp, Mr, Lr, ncpr, rows_cap, grid, cap_src, fpre); break;
    case 3: st = m2l_f32_dev_p<3>(c, t, de, gp, blocks, dnb, cap_blocks, Ms, L, ncp, Mr, Lr, ncpr, rows_cap, grid, cap_src, fpre); break;
    case 4: st = m2l_f32_dev_p<4>(c, t, de, gp, blocks, dnb, cap_blocks, Ms, L, ncp, Mr, Lr, ncpr, rows_cap, grid, cap_src, fpre); break;
    case 5: st = m2l_f32_dev_p<5>(c, t, de, gp, blocks, dnb, cap_blocks, Ms, L, ncp, Mr, Lr, ncpr, rows_cap, grid, cap_src, fpre); break;
    default: st = m2l_f32_dev_p<6>(c, t, de, gp, blocks, dnb, cap_blocks, Ms, L, ncp, Mr, Lr, ncpr, rows_cap, grid, cap_src, fpre);
    }
    if (st) return st;
    return cuda_check(c, cudaGetLastError(), "m2l launch (device sizes)");
}

tg_status launch_m2l_f64_dev(tg_ctx *c, const TreeView &t, const DevEval *de, const Geom *gp, const M2LBlock *blocks,
                             const unsigned long long *dnb, int64_t cap_blocks, const double *Ms, double *L, int p,
                             int ncp)
{
    const int plummer = c->prm.kernel == TG_KERNEL_PLUMMER;
    const int grid = c->num_sms * 16, nc = ncoef(p);
    ProfScope ps_(c, TG_K_M2L);
    m2l_blocks_generic<double, true><<<grid, 128, 0, c->stream>>>(t, blocks, cap_blocks, Ms, L, p, nc, ncp, 0.0, plummer,
                                                                  dnb, de, gp, c->prm.eps);
    m2l_blocks_generic<double, false><<<grid, 128, 0, c->stream>>>(t, blocks, cap_blocks, Ms, L, p, nc, ncp, 0.0, plummer,
                                                                   dnb, de, gp, c->prm.eps);
    return cuda_check(c, cudaGetLastError(), "m2l launch (device sizes, float64)");
}

tg_status launch_m2l_f64(tg_ctx *c, const TreeView &t, const M2LBlock *blocks, int64_t nblocks, const double *Ms,
                         double *L, int p, int nc, int ncp, bool masked)
{
    if (p > TG_PMAX) return launch_m2l_hi<double>(c, t, blocks, nblocks, Ms, L, p, nc, ncp, masked, true);
    const int plummer = c->prm.kernel == TG_KERNEL_PLUMMER;
    const double eoL = ldexp(c->prm.eps, -c->walk_log2L);
    const int grid = grid_for(nblocks * 32, 128, c->num_sms * 16);
    ProfScope ps_(c, TG_K_M2L);
    if (masked) m2l_blocks_generic<double, true><<<grid, 128, 0, c->stream>>>(t, blocks, nblocks, Ms, L, p, nc, ncp, eoL, plummer);
    else m2l_blocks_generic<double, false><<<grid, 128, 0, c->stream>>>(t, blocks, nblocks, Ms, L, p, nc, ncp, eoL, plummer);
    return cuda_check(c, cudaGetLastError(), "m2l launch");
}

}  // namespace tg
