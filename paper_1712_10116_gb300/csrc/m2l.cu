// m2l.cu -- launchers of the mutual M2L kernels (Sec. 2.1): float32 fixed-order block kernels for
// p <= 6, the generic kernel otherwise and in float64.  Its own translation unit, so that the large
// generated contractions compile in parallel with the rest.
#include "tg_common.cuh"
#include "m2l_sym.cuh"

namespace tg {

tg_status launch_m2l_f32(tg_ctx *c, const TreeView &t, const M2LBlock *blocks, int64_t nblocks, const float *Ms,
                         float *L, int p, int nc, int ncp, bool masked, bool pot)
{
    const int plummer = c->prm.kernel == TG_KERNEL_PLUMMER;
    const float eoL = (float)ldexp(c->prm.eps, -c->walk_log2L);
    const int grid = grid_for(nblocks * 32, 128, c->num_sms * 16);
    ProfScope ps_(c, TG_K_M2L);
#define TG_M2L_F32_(PP, MK, PT) m2l_blocks_f32<PP, MK, PT><<<grid, 128, 0, c->stream>>>(t, blocks, nblocks, Ms, L, ncp, eoL, plummer)
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

tg_status launch_m2l_f64(tg_ctx *c, const TreeView &t, const M2LBlock *blocks, int64_t nblocks, const double *Ms,
                         double *L, int p, int nc, int ncp, bool masked)
{
    const int plummer = c->prm.kernel == TG_KERNEL_PLUMMER;
    const double eoL = ldexp(c->prm.eps, -c->walk_log2L);
    const int grid = grid_for(nblocks * 32, 128, c->num_sms * 16);
    ProfScope ps_(c, TG_K_M2L);
    if (masked) m2l_blocks_generic<double, true><<<grid, 128, 0, c->stream>>>(t, blocks, nblocks, Ms, L, p, nc, ncp, eoL, plummer);
    else m2l_blocks_generic<double, false><<<grid, 128, 0, c->stream>>>(t, blocks, nblocks, Ms, L, p, nc, ncp, eoL, plummer);
    return cuda_check(c, cudaGetLastError(), "m2l launch");
}

}  // namespace tg
