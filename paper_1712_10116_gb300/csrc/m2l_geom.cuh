// m2l_geom.cuh -- geometry of an M2L block: the child cells of an opened cell pair and the exact
// offset between two cell centres in units of the x cell.
#pragma once
#include "tg_common.cuh"

namespace tg {

// children of the opened cells (a cell that is not opened stands for itself)
struct BlockGeom {
    int baseA, baseB, ni, nj, lx, ly;
};

__device__ __forceinline__ BlockGeom block_geom(const TreeView &t, const M2LBlock &blk)
{
    BlockGeom bg;
    const int A = (int)blk.a, B = (int)blk.b;
    const bool openA = t.nchild[A] != 0, openB = t.nchild[B] != 0;
    bg.ni = openA ? t.nchild[A] : 1;
    bg.nj = openB ? t.nchild[B] : 1;
    bg.baseA = openA ? t.child_first[A] : A;
    bg.baseB = openB ? t.child_first[B] : B;
    bg.lx = t.level[A] + (openA ? 1 : 0);
    bg.ly = t.level[B] + (openB ? 1 : 0);
    return bg;
}

// d' = (z_x - z_y) / s_x from the integer cell coordinates: the offset in units of half the finer
// cell (exact integer) times 2^(lx - lf - 1) (exact power of two).
template <class T>
__device__ __forceinline__ void pair_offset(const TreeView &t, int x, int y, int lx, int ly, T &dx, T &dy, T &dz)
{
    const int lf = lx > ly ? lx : ly;
    // |delta| < 2^23 (both centres lie in the root cube), so int32 holds it exactly
    const T scale = (T)pow2f(lx - lf - 1);
    dx = (T)(int)centre_delta(t.cx[x], lx, t.cx[y], ly, lf) * scale;
    dy = (T)(int)centre_delta(t.cy[x], lx, t.cy[y], ly, lf) * scale;
    dz = (T)(int)centre_delta(t.cz[x], lx, t.cz[y], ly, lf) * scale;
}

}  // namespace tg
