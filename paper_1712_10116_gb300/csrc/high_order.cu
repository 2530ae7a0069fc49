// high_order.cu -- expansion kernels for orders TG_PMAX < p <= kPHigh: the order sweeps of Sec. 3.2
// (Figs. 4-7) run p up to 20.  Same normalised expansions and the same formulas as the table-driven
// kernels of fmm.cu and m2l_sym.cuh:
//   M~^j = sum m (r/s)^j,  Ms^j = M~^j / j!,  L~^n = L^n s^(|n|+1),
// but the multi-indices come from index arithmetic instead of tables, and the working sets (up to
// C(23,3) = 1771 coefficients per expansion at p = 20) live in shared memory instead of registers.
//
// M2L for the unsoftened G = -1/r uses the harmonic reduction (D^{k+2e_x} + D^{k+2e_y} + D^{k+2e_z}
// = 0): moments folded onto j_z <= 1 once per cell, locals formed for n_z <= 1 per pair and
// completed once per cell.  At p = 20 that is about 37,000 instead of 230,230 terms per side;
// the result is the same in exact arithmetic.
#include "tg_common.cuh"
#include "m2l_geom.cuh"
#include "high_order.cuh"

namespace tg {

// 1/n! for n <= 20 (n! is exact in float64 up to 22!, so each entry is the correctly rounded quotient)
__constant__ double c_hi_inv_fact[kPHigh + 1] = {
    1.0, 1.0, 1.0 / 2.0, 1.0 / 6.0, 1.0 / 24.0, 1.0 / 120.0, 1.0 / 720.0, 1.0 / 5040.0, 1.0 / 40320.0,
    1.0 / 362880.0, 1.0 / 3628800.0, 1.0 / 39916800.0, 1.0 / 479001600.0, 1.0 / 6227020800.0,
    1.0 / 87178291200.0, 1.0 / 1307674368000.0, 1.0 / 20922789888000.0, 1.0 / 355687428096000.0,
    1.0 / 6402373705728000.0, 1.0 / 121645100408832000.0, 1.0 / 2432902008176640000.0};

__device__ __forceinline__ double hi_inv_fact3(int x, int y, int z)
{
    return c_hi_inv_fact[x] * c_hi_inv_fact[y] * c_hi_inv_fact[z];
}

// ------------------------------------------------------------------ P2M (leaves)
// Warp per leaf.  Monopole and dipole in float64 from the float64 positions (M01), every order in T
// from the leaf-relative offsets: lanes over coefficients, particles staged 32 at a time as powers
// of their scaled offsets.
template <class T, class T4>
__global__ void __launch_bounds__(64) p2m_leaves_hi(TreeView t, const Geom *gp, const double *xs, const double *ys,
                                                     const double *zs, const double *ms, const uint8_t *fs,
                                                     const T4 *pf, int p, int nc, int ncp, T *M, double *M01)
{
    __shared__ T s_pw[2][3][kPHigh + 1][33];
    __shared__ T s_w[2][2][32];
    const Geom g = *gp;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < t.ncell; c += nwarps) {
        if (t.nchild[c] != 0) continue;
        const int first = t.first[c], count = t.count[c];
        const double zx = cell_centre(g, t, c, 0), zy = cell_centre(g, t, c, 1), zz = cell_centre(g, t, c, 2);
        const double inv_s = ldexp(1.0, (int)t.level[c] - g.log2L);
        double lo[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // [class * 4 + k], class 0 slow, 1 fast
        for (int s = first + lane; s < first + count; s += 32) {
            const double m = ms[s];
            const bool fast = fs[s] != 0;
            const double r[4] = {1.0, (xs[s] - zx) * inv_s, (ys[s] - zy) * inv_s, (zs[s] - zz) * inv_s};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double v = k ? m * r[k] : m;
                lo[k] += fast ? 0.0 : v;
                lo[4 + k] += fast ? v : 0.0;
            }
        }
        double mine = 0.0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const double v = warp_sum(lo[e]);
            if (lane == e) mine = v;
        }
        if (lane < 8) {
            const int cls = lane >> 2, k = lane & 3;
            M01[((size_t)c * 2 + cls) * 4 + k] = mine;
            M[((size_t)c * 2 + cls) * ncp + k] = (T)mine;
        }
        const T inv_st = (T)inv_s;
        for (int k0 = 4; k0 < ncp; k0 += 32) {
            const int k = k0 + lane;
            int kx = 0, ky = 0, kz = 0;
            if (k < nc) hi_decode(k, kx, ky, kz);
            T aS = 0, aF = 0;
            for (int s0 = 0; s0 < count; s0 += 32) {
                const int m = min(32, count - s0);
                __syncwarp();
                if (lane < m) {
                    const T4 r = pf[first + s0 + lane];
                    const T rv[3] = {r.x * inv_st, r.y * inv_st, r.z * inv_st};
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        T v = T(1);
                        s_pw[wib][a][0][lane] = v;
                        for (int e = 1; e <= p; ++e) {
                            v *= rv[a];
                            s_pw[wib][a][e][lane] = v;
                        }
                    }
                    const bool fast = fs[first + s0 + lane] != 0;
                    s_w[wib][0][lane] = fast ? T(0) : r.w;
                    s_w[wib][1][lane] = fast ? r.w : T(0);
                }
                __syncwarp();
                if (k < nc)
                    for (int i = 0; i < m; ++i) {
                        const T v = s_pw[wib][0][kx][i] * s_pw[wib][1][ky][i] * s_pw[wib][2][kz][i];
                        aS += s_w[wib][0][i] * v;
                        aF += s_w[wib][1][i] * v;
                    }
            }
            if (k < ncp) {
                M[((size_t)c * 2 + 0) * ncp + k] = k < nc ? aS : T(0);
                M[((size_t)c * 2 + 1) * ncp + k] = k < nc ? aF : T(0);
            }
        }
    }
}

// ------------------------------------------------------------------ M2M (parents of one level)
// M~_P^n = sum_children sum_{k <= n} C(n,k) 2^-(2|n-k| + |k|) (+-1)^(n-k) M~_c^k (the child centre lies
// at +-s/4 per axis, the child side is s/2).  Block per parent, threads over n; |n| <= 1 in float64.
template <class T>
__global__ void __launch_bounds__(256) m2m_level_hi(TreeView t, int lb, int le, int p, int nc, int ncp, T *M,
                                                     double *M01)
{
    __shared__ double s_binom[kPHigh + 1][kPHigh + 1];
    for (int e = threadIdx.x; e < (kPHigh + 1) * (kPHigh + 1); e += blockDim.x) {
        const int n = e / (kPHigh + 1), k = e % (kPHigh + 1);
        double b = 0.0;
        if (k <= n) {
            b = 1.0;
            for (int i = 1; i <= k; ++i) b = b * (n - k + i) / i;   // C(n-k+i, i): exact integers
        }
        s_binom[n][k] = b;
    }
    __syncthreads();
    for (int c = lb + blockIdx.x; c < le; c += gridDim.x) {
        const int nch = t.nchild[c];
        if (nch == 0) continue;
        const int cf = t.child_first[c];
        if (threadIdx.x < 8) {
            const int cls = threadIdx.x >> 2, n = threadIdx.x & 3;
            double acc = 0.0;
            for (int q = 0; q < nch; ++q) {
                const double *Mc = M01 + ((size_t)(cf + q) * 2 + cls) * 4;
                double v = Mc[n];
                if (n > 0) {
                    const uint32_t cc = n == 1 ? t.cx[cf + q] : (n == 2 ? t.cy[cf + q] : t.cz[cf + q]);
                    v = 0.5 * v + ((cc & 1u) ? 0.25 : -0.25) * Mc[0];
                }
                acc += v;
            }
            M01[((size_t)c * 2 + cls) * 4 + n] = acc;
            M[((size_t)c * 2 + cls) * ncp + n] = (T)acc;
        }
        for (int n = 4 + threadIdx.x; n < ncp; n += blockDim.x) {
            T sS = 0, sF = 0;
            if (n < nc) {
                int nx, ny, nz;
                hi_decode(n, nx, ny, nz);
                const int on = nx + ny + nz;
                for (int q = 0; q < nch; ++q) {
                    const int ch = cf + q;
                    const bool neg_x = !(t.cx[ch] & 1u), neg_y = !(t.cy[ch] & 1u), neg_z = !(t.cz[ch] & 1u);
                    const T *MS = M + (size_t)ch * 2 * ncp, *MF = MS + ncp;
                    for (int kx = 0; kx <= nx; ++kx)
                        for (int ky = 0; ky <= ny; ++ky)
                            for (int kz = 0; kz <= nz; ++kz) {
                                const int k = hi_index(kx, ky, kz), ok = kx + ky + kz;
                                const double coef = s_binom[nx][kx] * s_binom[ny][ky] * s_binom[nz][kz] *
                                                    ldexp(1.0, -(2 * (on - ok) + ok));
                                const bool neg = (neg_x && ((nx - kx) & 1)) ^ (neg_y && ((ny - ky) & 1)) ^
                                                 (neg_z && ((nz - kz) & 1));
                                const T cs = (T)(neg ? -coef : coef);
                                sS += cs * MS[k];
                                sF += cs * MF[k];
                            }
                }
            }
            M[((size_t)c * 2 + 0) * ncp + n] = n < nc ? sS : T(0);
            M[((size_t)c * 2 + 1) * ncp + n] = n < nc ? sF : T(0);
        }
    }
}

// ------------------------------------------------------------------ M2L (harmonic fold / completion)
// Moments: every component with j_z >= 2 is moved onto (j_x + 2, j_y, j_z - 2) and (j_x, j_y + 2, j_z - 2)
// with a minus sign, highest j_z first, and zeroed.  One thread per (cell, class) row.
template <class T>
__global__ void fold_moments_hi(int64_t nrows, const T *__restrict__ Ms, T *__restrict__ Mf, int p, int ncp)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nrows; w += (int64_t)gridDim.x * blockDim.x) {
        hi_fold_row<T>(Ms + w * ncp, Mf + w * ncp, p, ncp);
    }
}

// Locals: L^{n} for n_z >= 2 from L^{n - 2e_z + 2e_x} and L^{n - 2e_z + 2e_y} (same order, both earlier
// in the order), in place.  One thread per (cell, class) row.
template <class T>
__global__ void complete_locals_hi(int64_t nrows, T *L, int p, int ncp)
{
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nrows; w += (int64_t)gridDim.x * blockDim.x) {
        hi_complete_row<T>(L + w * ncp, p);
    }
}

// ------------------------------------------------------------------ M2L (mutual, block per M2L block)
// For each well-separated child pair (x, y) of the block, in turn: D^k(d'), |k| <= p, by the
// auxiliary recurrence R^(m)_{k+e_a} = d_a R^(m+1)_k + k_a R^(m+1)_{k-e_a} run level by level from
// m = p down to 0 (two shared buffers), then both sides
//   L~_x^n += sum_j (-1)^|j| rho^|j| Ms_y^j D^{n+j},   L~_y^n += (-1)^|n| rho^(|n|+1) sum_j Ms_x^j D^{n+j}
// with threads over n.  HARM: n and j restricted to z <= 1 (moments folded, locals completed after).
template <class T, bool MASKED, bool HARM>
__global__ void __launch_bounds__(256) m2l_blocks_hi(TreeView t, const M2LBlock *__restrict__ blocks, int64_t nblocks,
                                                      const T *__restrict__ Ms, T *L, int p, int nc, int ncp,
                                                      double eps_over_L, int plummer, int pot)
{
    extern __shared__ __align__(16) unsigned char hi_smem[];
    T *s_a = reinterpret_cast<T *>(hi_smem);   // auxiliary levels of even m (D at the end)
    T *s_b = s_a + ncp;                        // auxiliary levels of odd m
    T *s_mx = s_b + ncp;                       // [class][ncp] moments of x
    T *s_my = s_mx + 2 * ncp;                  // [class][ncp] moments of y
    constexpr int ncls = MASKED ? 2 : 1;
    const int nn = HARM ? (p + 1) * (p + 1) : nc;   // outputs per side
    for (int64_t w = blockIdx.x; w < nblocks; w += gridDim.x) {
        const M2LBlock blk = blocks[w];
        const BlockGeom bg = block_geom(t, blk);
        const double soft = plummer ? ldexp(eps_over_L, bg.lx) : 0.0;
        for (int ij = 0; ij < 64; ++ij) {
            const int i = ij >> 3, j = ij & 7;
            if (!((blk.mask >> ij) & 1ull) || i >= bg.ni || j >= bg.nj) continue;   // uniform over the block
            const int x = bg.baseA + i, y = bg.baseB + j;
            double dx, dy, dz;
            pair_offset<double>(t, x, y, bg.lx, bg.ly, dx, dy, dz);
            const double s2 = dx * dx + dy * dy + dz * dz + soft * soft;
            const double si = 1.0 / sqrt(s2), si2 = si * si;
            __syncthreads();   // the previous pair is done with the shared arrays
            for (int k = threadIdx.x; k < ncls * ncp; k += blockDim.x) {
                s_mx[k] = Ms[(size_t)x * 2 * ncp + k];
                s_my[k] = Ms[(size_t)y * 2 * ncp + k];
            }
            if (threadIdx.x == 0) {
                double f = -si;   // f^(m) of G = -(rho2 / 2 ...)^: f^(0) = -1/s, f^(m+1) = -(2m+1) f^(m) / s^2
                for (int m = 0; m < p; ++m) f = -f * (2 * m + 1) * si2;
                ((p & 1) ? s_b : s_a)[0] = (T)f;
            }
            __syncthreads();
            for (int m = p - 1; m >= 0; --m) {
                T *out = (m & 1) ? s_b : s_a;
                const T *in = (m & 1) ? s_a : s_b;
                double fm = -si;
                for (int q = 0; q < m; ++q) fm = -fm * (2 * q + 1) * si2;
                const int nk = ncoef_dev(p - m);
                for (int k = threadIdx.x; k < nk; k += blockDim.x) {
                    if (k == 0) {
                        out[0] = (T)fm;
                        continue;
                    }
                    int kx, ky, kz;
                    hi_decode(k, kx, ky, kz);
                    const int a = kx > 0 ? 0 : (ky > 0 ? 1 : 2);
                    const int ka = a == 0 ? kx : (a == 1 ? ky : kz);
                    const double da = a == 0 ? dx : (a == 1 ? dy : dz);
                    const int ex = a == 0, ey = a == 1, ez = a == 2;
                    T v = (T)da * in[hi_index(kx - ex, ky - ey, kz - ez)];
                    if (ka >= 2) v += (T)(ka - 1) * in[hi_index(kx - 2 * ex, ky - 2 * ey, kz - 2 * ez)];
                    out[k] = v;
                }
                __syncthreads();
            }
            const T *D = s_a;
            const T rho = (T)ldexp(1.0, bg.lx - bg.ly);
            for (int r = threadIdx.x; r < nn; r += blockDim.x) {
                int nx, ny, nz;
                if (HARM) {
                    // reduced order: total degree o, then (o,0,0), then pairs (x, o-x, 0), (x, o-x-1, 1)
                    int o = 0;
                    while ((o + 1) * (o + 1) <= r) ++o;
                    const int pos = r - o * o;
                    const int a = (pos + 1) / 2;
                    nz = pos == 0 ? 0 : pos + 1 - 2 * a;
                    nx = o - a;
                    ny = a - nz;
                } else {
                    hi_decode(r, nx, ny, nz);
                }
                const int on = nx + ny + nz;
                if (!pot && on == 0) continue;   // L^0 feeds the potential only
                T sa[ncls], sb[ncls];
#pragma unroll
                for (int cl = 0; cl < ncls; ++cl) sa[cl] = sb[cl] = T(0);
                T rp = T(1);
                for (int oj = 0; oj <= p - on; ++oj) {
                    const T sg = (oj & 1) ? -rp : rp;
                    for (int jx = oj; jx >= 0; --jx) {
                        const int zmax = HARM ? min(1, oj - jx) : oj - jx;
                        for (int jz = 0; jz <= zmax; ++jz) {
                            const int jy = oj - jx - jz;
                            const int jk = hi_index(jx, jy, jz);
                            const T Dv = D[hi_index(nx + jx, ny + jy, nz + jz)];
#pragma unroll
                            for (int cl = 0; cl < ncls; ++cl) {
                                sa[cl] += sg * s_my[cl * ncp + jk] * Dv;
                                sb[cl] += s_mx[cl * ncp + jk] * Dv;
                            }
                        }
                    }
                    rp *= rho;
                }
                T rn = rho;
                for (int o = 0; o < on; ++o) rn *= rho;
                const T sgn = (on & 1) ? -rn : rn;
                const int n = hi_index(nx, ny, nz);
#pragma unroll
                for (int cl = 0; cl < ncls; ++cl) {
                    atomicAdd(&L[((size_t)x * 2 + cl) * ncp + n], sa[cl]);
                    atomicAdd(&L[((size_t)y * 2 + cl) * ncp + n], sgn * sb[cl]);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ L2L (one level)
// L~_c^n += sum_d L~_P^(n+d) (+-1)^d 2^-(2|d| + |n| + 1) / d!  over |d| <= p - |n|; warp per cell,
// lanes over n >= n_first.
template <class T>
__global__ void __launch_bounds__(128) l2l_level_hi(TreeView t, int lb, int le, int p, int nc, int ncp, int ncls,
                                                     int n_first, T *L)
{
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = lb + warp; c < le; c += nwarps) {
        const int par = t.parent[c];
        if (par < 0) continue;
        const bool neg_x = !(t.cx[c] & 1u), neg_y = !(t.cy[c] & 1u), neg_z = !(t.cz[c] & 1u);
        const T *Lp = L + (size_t)par * 2 * ncp;
        for (int n = n_first + lane; n < nc; n += 32) {
            int nx, ny, nz;
            hi_decode(n, nx, ny, nz);
            const int on = nx + ny + nz;
            T acc0 = 0, acc1 = 0;
            for (int od = 0; od <= p - on; ++od)
                for (int dx = od; dx >= 0; --dx)
                    for (int dy = od - dx; dy >= 0; --dy) {
                        const int dz = od - dx - dy;
                        const int k = hi_index(nx + dx, ny + dy, nz + dz);
                        const bool neg = (neg_x && (dx & 1)) ^ (neg_y && (dy & 1)) ^ (neg_z && (dz & 1));
                        const double coef = hi_inv_fact3(dx, dy, dz) * ldexp(1.0, -(2 * od + on + 1));
                        const T cs = (T)(neg ? -coef : coef);
                        acc0 += Lp[k] * cs;
                        if (ncls > 1) acc1 += Lp[ncp + k] * cs;
                    }
            L[((size_t)c * 2 + 0) * ncp + n] += acc0;
            if (ncls > 1) L[((size_t)c * 2 + 1) * ncp + n] += acc1;
        }
    }
}

// ------------------------------------------------------------------ L2P
// With r = (x - z)/s:  phi = (1/s) sum_n L~^n r^n/n!,  a_e = -(1/s^2) sum_m L~^{m+e} r^m/m!.
template <class T, class T4>
__global__ void l2p_particles_hi(int n, TreeView t, int log2L, const T4 *pf, const int32_t *leaf_of, const uint8_t *fs,
                                 int masked, int p, int ncp, const T *L, double *acc4)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const T4 r = pf[s];
        const int c = leaf_of[s];
        const int cls = (masked && fs[s]) ? 1 : 0;
        const T *Lc = L + ((size_t)c * 2 + cls) * ncp;
        const T inv_s = (T)ldexp(1.0, (int)t.level[c] - log2L);
        const T rx = r.x * inv_s, ry = r.y * inv_s, rz = r.z * inv_s;
        T px[kPHigh + 1], py[kPHigh + 1], pz[kPHigh + 1];
        px[0] = py[0] = pz[0] = (T)1;
        for (int e = 1; e <= p; ++e) {
            px[e] = px[e - 1] * rx;
            py[e] = py[e - 1] * ry;
            pz[e] = pz[e - 1] * rz;
        }
        T phi = 0, gx = 0, gy = 0, gz = 0;
        int k = 0;
        for (int o = 0; o <= p; ++o)
            for (int kx = o; kx >= 0; --kx)
                for (int ky = o - kx; ky >= 0; --ky, ++k) {
                    const int kz = o - kx - ky;
                    const T mono = px[kx] * py[ky] * pz[kz] * (T)hi_inv_fact3(kx, ky, kz);
                    phi += Lc[k] * mono;
                    if (o < p) {
                        gx += Lc[hi_index(kx + 1, ky, kz)] * mono;
                        gy += Lc[hi_index(kx, ky + 1, kz)] * mono;
                        gz += Lc[hi_index(kx, ky, kz + 1)] * mono;
                    }
                }
        const T is2 = inv_s * inv_s;
        acc4[s] = (double)(-gx * is2);
        acc4[(size_t)n + s] = (double)(-gy * is2);
        acc4[2 * (size_t)n + s] = (double)(-gz * is2);
        acc4[3 * (size_t)n + s] = (double)(phi * inv_s);
    }
}

// ------------------------------------------------------------------ launchers
template <class T, class T4>
tg_status launch_p2m_hi(tg_ctx *c, const TreeView &t, const Geom *d_geom, const double *xs, const double *ys,
                        const double *zs, const double *ms, const uint8_t *fs, const T4 *pf, int p, int nc, int ncp,
                        T *M, double *M01)
{
    ProfScope ps_(c, TG_K_UP);
    p2m_leaves_hi<T, T4><<<grid_for((int64_t)t.ncell * 32, 64), 64, 0, c->stream>>>(t, d_geom, xs, ys, zs, ms, fs, pf,
                                                                                    p, nc, ncp, M, M01);
    return cuda_check(c, cudaGetLastError(), "p2m (high order)");
}

template <class T>
tg_status launch_m2m_hi(tg_ctx *c, const TreeView &t, int lb, int le, int p, int nc, int ncp, T *M, double *M01)
{
    ProfScope ps_(c, TG_K_UP);
    m2m_level_hi<T><<<std::min(le - lb, c->num_sms * 8), 256, 0, c->stream>>>(t, lb, le, p, nc, ncp, M, M01);
    return cuda_check(c, cudaGetLastError(), "m2m (high order)");
}

template <class T>
tg_status launch_m2l_hi(tg_ctx *c, const TreeView &t, const M2LBlock *blocks, int64_t nblocks, const T *Ms, T *L,
                        int p, int nc, int ncp, bool masked, bool pot)
{
    const int plummer = c->prm.kernel == TG_KERNEL_PLUMMER;
    const bool harm = !plummer;   // the eps gap rule leaves every Wendland M2L pair at r >= eps: G = -1/r
    const int64_t rows = (int64_t)t.ncell * 2;
    const T *src = Ms;
    tg_status st;
    ProfScope ps_(c, TG_K_M2L);
    if (harm) {
        T *Mf;
        if ((st = ensure_t(c, B_MOMH, (size_t)rows * ncp, &Mf))) return st;
        fold_moments_hi<T><<<grid_for(rows, 128), 128, 0, c->stream>>>(rows, Ms, Mf, p, ncp);
        src = Mf;
    }
    const size_t smem = 6 * (size_t)ncp * sizeof(T);
    const int grid = (int)std::min<int64_t>(nblocks, (int64_t)c->num_sms * 4);
    const double eoL = ldexp(c->prm.eps, -c->walk_log2L);
#define TG_M2L_HI(MK, HM)                                                                                         \
    do {                                                                                                          \
        auto kern = m2l_blocks_hi<T, MK, HM>;                                                                     \
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                       \
        kern<<<grid, 256, smem, c->stream>>>(t, blocks, nblocks, src, L, p, nc, ncp, eoL, plummer, pot ? 1 : 0);   \
    } while (0)
    if (masked) {
        if (harm) TG_M2L_HI(true, true);
        else TG_M2L_HI(true, false);
    } else {
        if (harm) TG_M2L_HI(false, true);
        else TG_M2L_HI(false, false);
    }
#undef TG_M2L_HI
    if (harm) complete_locals_hi<T><<<grid_for(rows, 128), 128, 0, c->stream>>>(rows, L, p, ncp);
    return cuda_check(c, cudaGetLastError(), "m2l (high order)");
}

template <class T>
tg_status launch_l2l_hi(tg_ctx *c, const TreeView &t, int lb, int le, int p, int nc, int ncp, int ncls, int n_first,
                        T *L)
{
    ProfScope ps_(c, TG_K_DOWN);
    l2l_level_hi<T><<<grid_for((int64_t)(le - lb) * 32, 128), 128, 0, c->stream>>>(t, lb, le, p, nc, ncp, ncls,
                                                                                     n_first, L);
    return cuda_check(c, cudaGetLastError(), "l2l (high order)");
}

template <class T, class T4>
tg_status launch_l2p_hi(tg_ctx *c, int n, const TreeView &t, const T4 *pf, const int32_t *leaf_of, const uint8_t *fs,
                        bool masked, int p, int ncp, const T *L, double *acc4)
{
    ProfScope ps_(c, TG_K_DOWN);
    l2p_particles_hi<T, T4><<<grid_for(n, 128), 128, 0, c->stream>>>(n, t, c->walk_log2L, pf, leaf_of, fs,
                                                                      masked ? 1 : 0, p, ncp, L, acc4);
    return cuda_check(c, cudaGetLastError(), "l2p (high order)");
}

#define TG_HI_INSTANTIATE(T, T4)                                                                                  \
    template tg_status launch_p2m_hi<T, T4>(tg_ctx *, const TreeView &, const Geom *, const double *,             \
                                            const double *, const double *, const double *, const uint8_t *,      \
                                            const T4 *, int, int, int, T *, double *);                            \
    template tg_status launch_m2m_hi<T>(tg_ctx *, const TreeView &, int, int, int, int, int, T *, double *);       \
    template tg_status launch_m2l_hi<T>(tg_ctx *, const TreeView &, const M2LBlock *, int64_t, const T *, T *,     \
                                        int, int, int, bool, bool);                                               \
    template tg_status launch_l2l_hi<T>(tg_ctx *, const TreeView &, int, int, int, int, int, int, int, T *);       \
    template tg_status launch_l2p_hi<T, T4>(tg_ctx *, int, const TreeView &, const T4 *, const int32_t *,          \
                                            const uint8_t *, bool, int, int, const T *, double *);
TG_HI_INSTANTIATE(float, float4)
TG_HI_INSTANTIATE(double, dbl4)
#undef TG_HI_INSTANTIATE

}  // namespace tg
