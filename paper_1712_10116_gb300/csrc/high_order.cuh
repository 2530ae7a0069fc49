// high_order.cuh -- index arithmetic and the per-cell harmonic fold / completion of the expansion
// kernels for orders above the fixed tables (high_order.cu).  Plain functions for host and device:
// nothing here touches device memory by itself, so the host tests compile this header too.
#pragma once

namespace tg {

// position of (x, y, z) in the order by total degree, then x descending, then y descending
__host__ __device__ __forceinline__ int hi_index(int x, int y, int z)
{
    const int o = x + y + z, a = o - x;
    return o * (o + 1) * (o + 2) / 6 + a * (a + 1) / 2 + z;
}

__host__ __device__ __forceinline__ void hi_decode(int k, int &x, int &y, int &z)
{
    int o = 0;
    while ((o + 1) * (o + 2) * (o + 3) / 6 <= k) ++o;
    const int r = k - o * (o + 1) * (o + 2) / 6;
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= r) ++a;
    z = r - a * (a + 1) / 2;
    x = o - a;
    y = a - z;
}

// Moments of one (cell, class) row, orders <= p: every component with j_z >= 2 is moved onto
// (j_x + 2, j_y, j_z - 2) and (j_x, j_y + 2, j_z - 2) with a minus sign, highest j_z first, and zeroed.
// For a harmonic derivative tensor (D^{k+2e_x} + D^{k+2e_y} + D^{k+2e_z} = 0) the folded row gives
// every contraction sum_j M^j D^{n+j} unchanged.  dst may not alias src; ncp entries are copied.
template <class T>
__host__ __device__ __forceinline__ void hi_fold_row(const T *src, T *dst, int p, int ncp)
{
    for (int k = 0; k < ncp; ++k) dst[k] = src[k];
    for (int jz = p; jz >= 2; --jz)
        for (int o = jz; o <= p; ++o)
            for (int jx = o - jz; jx >= 0; --jx) {
                const int jy = o - jz - jx;
                const int k = hi_index(jx, jy, jz);
                const T v = dst[k];
                dst[hi_index(jx + 2, jy, jz - 2)] -= v;
                dst[hi_index(jx, jy + 2, jz - 2)] -= v;
                dst[k] = T(0);
            }
}

// Locals of one row: L^n for n_z >= 2 from L^{n - 2e_z + 2e_x} and L^{n - 2e_z + 2e_y} (same order, both
// earlier in the order), in place.
template <class T>
__host__ __device__ __forceinline__ void hi_complete_row(T *row, int p)
{
    for (int o = 2; o <= p; ++o)
        for (int kx = o - 2; kx >= 0; --kx)
            for (int kz = 2; kz <= o - kx; ++kz) {
                const int ky = o - kx - kz;
                row[hi_index(kx, ky, kz)] = -row[hi_index(kx + 2, ky, kz - 2)] - row[hi_index(kx, ky + 2, kz - 2)];
            }
}

}  // namespace tg
