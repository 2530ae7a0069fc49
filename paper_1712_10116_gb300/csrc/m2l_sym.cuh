// m2l_sym.cuh -- mutual cell-cell interaction (M2L, Sec. 2.1).  Each unordered well-separated
// pair (A, B) is visited once: the derivative tensor D^k(z_A - z_B), |k| <= p, is built once and
// both local expansions are updated,
//   L_A^n += sum_j (-1)^|j|/j! M_B^j D^{n+j},   L_B^n += (-1)^|n| sum_j M_A^j/j! D^{n+j},
// using D^k(-d) = (-1)^|k| D^k(d).  D comes from the McMurchie-Davidson auxiliary recurrence
// R^(m)_{k+e_a} = d_a R^(m+1)_k + k_a R^(m+1)_{k-e_a}, R^(m)_0 = f_m, with f_m the m-th derivative
// of G as a function of |d|^2/2: G = -1/r (Newton, used for Wendland pairs, which are farther
// apart than eps) or -(r^2 + eps^2)^(-1/2) (Plummer).
#pragma once
#include "tg_common.cuh"
#include "tg_tables.cuh"

namespace tg {

template <class T>
struct Mom {
    const T *M;
};

template <class T>
static Mom<T> make_moments(tg_ctx *c, const double *M, size_t count, tg_status *st);

template <>
Mom<double> make_moments<double>(tg_ctx *c, const double *M, size_t count, tg_status *st)
{
    (void)c;
    (void)count;
    *st = TG_OK;
    return Mom<double>{M};
}

__global__ void convert_moments(const double *M, float *Mf, int64_t count);

template <>
Mom<float> make_moments<float>(tg_ctx *c, const double *M, size_t count, tg_status *st)
{
    float *Mf = nullptr;
    *st = ensure_t(c, B_MOMF, count, &Mf);
    if (*st) return Mom<float>{nullptr};
    {
        ProfScope ps_(c, TG_K_UP);
        convert_moments<<<grid_for((int64_t)count, 256), 256, 0, c->stream>>>(M, Mf, (int64_t)count);
    }
    return Mom<float>{Mf};
}

// D^k(d) for |k| <= p into D[0..ncoef(p)); R holds R^(m)_k packed by m.
template <class T>
__device__ __forceinline__ void dtensor_generic(int p, T dx, T dy, T dz, T soft2, T *D)
{
    T R[((TG_PMAX + 1) * (TG_PMAX + 2) * (TG_PMAX + 3) * (TG_PMAX + 4)) / 24];
    int off[TG_PMAX + 2];
    off[0] = 0;
    for (int m = 0; m <= p; ++m) off[m + 1] = off[m] + ncoef_dev(p - m);
    const T s2 = dx * dx + dy * dy + dz * dz + soft2;
    const T si = T(1) / sqrt(s2);
    const T si2 = si * si;
    T f = -si;
    for (int m = 0; m <= p; ++m) {
        R[off[m]] = f;
        f = -f * T(2 * m + 1) * si2;
    }
    const int nc = ncoef_dev(p);
    for (int k = 1; k < nc; ++k) {
        const int a = c_rec_axis[k], ka = c_rec_ka[k], km = c_rec_km[k], kmm = c_rec_kmm[k];
        const int o = c_mi_order[k];
        const T da = a == 0 ? dx : (a == 1 ? dy : dz);
        for (int m = 0; m <= p - o; ++m) {
            T v = da * R[off[m + 1] + km];
            if (kmm != 255) v += T(ka - 1) * R[off[m + 1] + kmm];
            R[off[m] + k] = v;
        }
    }
    for (int k = 0; k < nc; ++k) D[k] = R[k];
}

template <class T, bool MASKED>
__global__ void m2l_mutual(TreeView t, const Geom *gp, const uint2 *pairs, int64_t npairs, const T *M, T *L, int p,
                           int nc, T soft2)
{
    const Geom g = *gp;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < npairs; w += (int64_t)gridDim.x * blockDim.x) {
        const uint2 pr = pairs[w];
        const int a = (int)pr.x, b = (int)pr.y;
        const double sa = ldexp(g.L, -(int)t.level[a]), sb = ldexp(g.L, -(int)t.level[b]);
        const T dx = (T)(((double)t.cx[a] + 0.5) * sa - ((double)t.cx[b] + 0.5) * sb);
        const T dy = (T)(((double)t.cy[a] + 0.5) * sa - ((double)t.cy[b] + 0.5) * sb);
        const T dz = (T)(((double)t.cz[a] + 0.5) * sa - ((double)t.cz[b] + 0.5) * sb);
        T D[TG_NCOEF_MAX];
        dtensor_generic<T>(p, dx, dy, dz, soft2, D);
        const T *MaS = M + ((size_t)a * 2 + 0) * nc, *MaF = M + ((size_t)a * 2 + 1) * nc;
        const T *MbS = M + ((size_t)b * 2 + 0) * nc, *MbF = M + ((size_t)b * 2 + 1) * nc;
        T *LaA = L + ((size_t)a * 2 + 0) * nc, *LaS = L + ((size_t)a * 2 + 1) * nc;
        T *LbA = L + ((size_t)b * 2 + 0) * nc, *LbS = L + ((size_t)b * 2 + 1) * nc;
        for (int n = 0; n < nc; ++n) {
            const int nx = c_mi_x[n], ny = c_mi_y[n], nz = c_mi_z[n], on = c_mi_order[n];
            const int ncj = ncoef_dev(p - on);
            T sA0 = 0, sA1 = 0, sB0 = 0, sB1 = 0;
            for (int j = 0; j < ncj; ++j) {
                const T Dv = D[c_mi_lookup[((nx + c_mi_x[j]) * 9 + ny + c_mi_y[j]) * 9 + nz + c_mi_z[j]]];
                const T w = (T)c_inv_fact[j];
                const T wa = (c_mi_order[j] & 1) ? -w : w;
                const T mbs = MbS[j], mas = MaS[j];
                const T mball = MASKED ? mbs + MbF[j] : mbs, maall = MASKED ? mas + MaF[j] : mas;
                sA0 += wa * mball * Dv;
                sB0 += w * maall * Dv;
                if (MASKED) {
                    sA1 += wa * mbs * Dv;
                    sB1 += w * mas * Dv;
                }
            }
            const T sgn = (on & 1) ? T(-1) : T(1);
            atomicAdd(&LaA[n], sA0);
            atomicAdd(&LbA[n], sgn * sB0);
            if (MASKED) {
                atomicAdd(&LaS[n], sA1);
                atomicAdd(&LbS[n], sgn * sB1);
            }
        }
    }
}

template <class T>
static tg_status launch_m2l(tg_ctx *c, const TreeView &t, const Geom *d_geom, const uint2 *pairs, int64_t npairs,
                            const Mom<T> &mom, T *L, int p, int nc, bool masked)
{
    const T soft2 = c->prm.kernel == TG_KERNEL_PLUMMER ? (T)(c->prm.eps * c->prm.eps) : T(0);
    const int grid = grid_for(npairs, 128);
    ProfScope ps_(c, TG_K_M2L);
    if (masked) m2l_mutual<T, true><<<grid, 128, 0, c->stream>>>(t, d_geom, pairs, npairs, mom.M, L, p, nc, soft2);
    else m2l_mutual<T, false><<<grid, 128, 0, c->stream>>>(t, d_geom, pairs, npairs, mom.M, L, p, nc, soft2);
    return cuda_check(c, cudaGetLastError(), "m2l launch");
}

}  // namespace tg
