// p2p.cu -- translation unit of the mutual P2P kernels (Sec. 2.1, Eq. 2): float32 packs the rows of
// the distinct leaf pairs by owner leaf and takes the self pairs in the same launch (p2p_owner.cuh,
// launch_p2p_f32); float64 runs one block per leaf pair (p2p_tile.cuh, launch_p2p_f64).
#include "tg_common.cuh"
#include "p2p_tile.cuh"
#include "p2p_owner.cuh"
