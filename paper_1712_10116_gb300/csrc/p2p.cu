// p2p.cu -- launchers of the mutual P2P kernels (Sec. 2.1, Eq. 2): float32 packs the rows of the
// distinct leaf pairs by owner leaf and takes the self pairs in the same launch (p2p_owner.cuh);
// float64 runs one block per leaf pair (p2p_tile.cuh).
#include "tg_common.cuh"
#include "p2p_tile.cuh"
#include "p2p_owner.cuh"

namespace tg {

tg_status launch_p2p_f32(tg_ctx *c, const TreeView &t, const uint2 *pairs, int64_t npairs, const uint2 *self_pairs,
                         int64_t nself, const float4 *pf, const int32_t *nslow, bool pot, double *acc4)
{
    return launch_p2p_owner(c, t, pairs, npairs, self_pairs, nself, pf, nslow, pot, acc4);
}

tg_status launch_p2p_f64(tg_ctx *c, const TreeView &t, const Geom *d_geom, const uint2 *pairs, int64_t npairs,
                         const uint2 *self_pairs, int64_t nself, const dbl4 *pf, const uint8_t *fs, bool masked,
                         double *acc4)
{
    tg_status st;
    if (npairs > 0 && (st = launch_p2p<double, dbl4>(c, t, d_geom, pairs, npairs, pf, fs, nullptr, masked, false, acc4)))
        return st;
    if (nself > 0 && (st = launch_p2p<double, dbl4>(c, t, d_geom, self_pairs, nself, pf, fs, nullptr, masked, true, acc4)))
        return st;
    return TG_OK;
}

}  // namespace tg
