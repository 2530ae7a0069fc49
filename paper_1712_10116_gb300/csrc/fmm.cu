// fmm.cu -- one FMM evaluation (the Poisson-solver call of Algorithm 3, Zhu 2017):
// upward pass (P2M, M2M), dual tree walk (Algorithm 4) emitting unordered cell pairs, mutual
// M2L and P2P (Sec. 2.1: F_AB = -F_BA), downward pass (L2L, L2P) and the direct-summation
// reference used to measure force errors.
//
// Expansions are Cartesian Taylor series truncated at total degree p:
//   M_A^j = sum_{i in A} m_i (x_i - z_A)^j,  phi(x) = sum_n L^n (x - z)^n / n!,
//   L_A^n += sum_{|j| <= p-|n|} (-1)^|j| / j!  M_B^j  D^{n+j}(z_A - z_B),  D^k = d^k G / dz^k,
// and the same derivative tensor gives the reaction on B: L_B^n += (-1)^|n| sum_j M_A^j / j! D^{n+j}.
// With this triangular truncation the net force of A on B is exactly minus that of B on A.
//
// Each cell carries two moment classes (slow S and fast F particles) and two local
// expansions: L_all (slow sinks, sources S + F) and L_S (fast sinks, sources S only).  One walk
// and one evaluation thus serve a kickFS2S + kickS2F pair of Algorithm 2.
#include "tg_common.cuh"
#include "tg_tables.cuh"
#include "p2p_tile.cuh"
#include "m2l_sym.cuh"

namespace tg {

// ------------------------------------------------------------------ cell geometry
__device__ __forceinline__ double cell_centre(const Geom &g, const TreeView &t, int c, int axis)
{
    const uint32_t ci = axis == 0 ? t.cx[c] : (axis == 1 ? t.cy[c] : t.cz[c]);
    return g.lo[axis] + ((double)ci + 0.5) * ldexp(g.L, -(int)t.level[c]);
}

// Eq. (1) with R = kappa * side, and the rule that cell pairs closer than eps (cube gap) never use
// M2L for the Wendland kernel.  Exact: integer units of half the finer cell's side.
struct MacParams {
    double theta2, kappa2, eps;
    int log2L, wendland;
};

__device__ __forceinline__ bool well_separated(const TreeView &t, const MacParams &mp, int a, int b)
{
    const int la = t.level[a], lb = t.level[b];
    const int lf = la > lb ? la : lb;
    const int64_t ha = (int64_t)1 << (lf - la), hb = (int64_t)1 << (lf - lb);
    const uint32_t ca[3] = {t.cx[a], t.cy[a], t.cz[a]}, cb[3] = {t.cx[b], t.cy[b], t.cz[b]};
    int64_t d2 = 0, g2 = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int64_t dk = (2 * (int64_t)ca[k] + 1) * ha - (2 * (int64_t)cb[k] + 1) * hb;
        if (dk < 0) dk = -dk;
        d2 += dk * dk;
        int64_t gk = dk - (ha + hb);
        if (gk > 0) g2 += gk * gk;
    }
    const double rsum = (double)(2 * (ha + hb));
    if (!(__dmul_rn((double)d2, mp.theta2) > __dmul_rn(mp.kappa2, __dmul_rn(rsum, rsum)))) return false;
    if (mp.wendland) {
        const double eu = ldexp(mp.eps, lf + 1 - mp.log2L);
        if (!((double)g2 > __dmul_rn(eu, eu))) return false;
    }
    return true;
}

// ------------------------------------------------------------------ per-particle local data
// pf[s] = (x - z_leaf, y - z_leaf, z - z_leaf, m) in precision T; leaf_of[s] = leaf cell id.
template <class T4>
__global__ void leaf_particles(TreeView t, const Geom *gp, const double *xs, const double *ys, const double *zs,
                               const double *ms, T4 *pf, int32_t *leaf_of)
{
    const Geom g = *gp;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < t.ncell; c += nwarps) {
        if (t.nchild[c] != 0) continue;
        const double zx = cell_centre(g, t, c, 0), zy = cell_centre(g, t, c, 1), zz = cell_centre(g, t, c, 2);
        for (int s = t.first[c] + lane; s < t.first[c] + t.count[c]; s += 32) {
            T4 v;
            v.x = (decltype(v.x))(xs[s] - zx);
            v.y = (decltype(v.x))(ys[s] - zy);
            v.z = (decltype(v.x))(zs[s] - zz);
            v.w = (decltype(v.x))ms[s];
            pf[s] = v;
            leaf_of[s] = c;
        }
    }
}

// ------------------------------------------------------------------ P2M
// Warp per leaf, lanes over coefficients; classes S (fast flag 0) and F (flag 1).  Monopole and
// dipole (|k| <= 1) are accumulated in float64 from float64 offsets; higher orders in T.
template <class T>
__global__ void p2m_leaves(TreeView t, const Geom *gp, const double *xs, const double *ys, const double *zs,
                           const double *ms, const uint8_t *fs, int p, int nc, double *M)
{
    const Geom g = *gp;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < t.ncell; c += nwarps) {
        if (t.nchild[c] != 0) continue;
        const double zx = cell_centre(g, t, c, 0), zy = cell_centre(g, t, c, 1), zz = cell_centre(g, t, c, 2);
        for (int k0 = 0; k0 < nc; k0 += 32) {
            const int k = k0 + lane;
            const bool on = k < nc;
            const int ex = on ? c_mi_x[k] : 0, ey = on ? c_mi_y[k] : 0, ez = on ? c_mi_z[k] : 0;
            if (k < 4) {
                double accS = 0.0, accF = 0.0;
                for (int s = t.first[c]; s < t.first[c] + t.count[c]; ++s) {
                    double v = ms[s];
                    if (ex) v *= xs[s] - zx;
                    if (ey) v *= ys[s] - zy;
                    if (ez) v *= zs[s] - zz;
                    if (fs[s]) accF += v;
                    else accS += v;
                }
                M[((size_t)c * 2 + 0) * nc + k] = accS;
                M[((size_t)c * 2 + 1) * nc + k] = accF;
            } else {
                T accS = 0, accF = 0;
                for (int s = t.first[c]; s < t.first[c] + t.count[c]; ++s) {
                    const T rx = (T)(xs[s] - zx), ry = (T)(ys[s] - zy), rz = (T)(zs[s] - zz);
                    T v = (T)ms[s];
                    for (int e = 0; e < ex; ++e) v *= rx;
                    for (int e = 0; e < ey; ++e) v *= ry;
                    for (int e = 0; e < ez; ++e) v *= rz;
                    if (fs[s]) accF += v;
                    else accS += v;
                }
                if (on) {
                    M[((size_t)c * 2 + 0) * nc + k] = (double)accS;
                    M[((size_t)c * 2 + 1) * nc + k] = (double)accF;
                }
            }
        }
    }
}

// M2M for the parents of one level: M_P^n = sum_children sum_{k <= n} C(n,k) d^(n-k) M_c^k with
// d = z_child - z_parent = (+-q, +-q, +-q), q = side_P / 4 (exact).  Thread per (cell, class, n);
// |n| <= 1 in float64, higher orders in T.
__constant__ float c_binom_f[9][9] = {
    {1, 0, 0, 0, 0, 0, 0, 0, 0},       {1, 1, 0, 0, 0, 0, 0, 0, 0},        {1, 2, 1, 0, 0, 0, 0, 0, 0},
    {1, 3, 3, 1, 0, 0, 0, 0, 0},       {1, 4, 6, 4, 1, 0, 0, 0, 0},        {1, 5, 10, 10, 5, 1, 0, 0, 0},
    {1, 6, 15, 20, 15, 6, 1, 0, 0},    {1, 7, 21, 35, 35, 21, 7, 1, 0},    {1, 8, 28, 56, 70, 56, 28, 8, 1}};

template <class T>
__global__ void m2m_level(TreeView t, const Geom *gp, int lb, int le, int p, int nc, double *M)
{
    const Geom g = *gp;
    const int64_t total = (int64_t)(le - lb) * 2 * nc;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
        const int c = lb + (int)(w / (2 * nc));
        const int cls = (int)((w / nc) % 2);
        const int n = (int)(w % nc);
        const int nch = t.nchild[c];
        if (nch == 0) continue;
        const int nx = c_mi_x[n], ny = c_mi_y[n], nz = c_mi_z[n];
        const double q = ldexp(g.L, -(int)t.level[c] - 2);
        if (n < 4) {
            double acc = 0.0;
            for (int ch_i = 0; ch_i < nch; ++ch_i) {
                const int ch = t.child_first[c] + ch_i;
                const double *Mc = M + ((size_t)ch * 2 + cls) * nc;
                double v = Mc[n];
                if (n > 0) {
                    const uint32_t cc = nx ? t.cx[ch] : (ny ? t.cy[ch] : t.cz[ch]);
                    v += ((cc & 1u) ? q : -q) * Mc[0];
                }
                acc += v;
            }
            M[((size_t)c * 2 + cls) * nc + n] = acc;
            continue;
        }
        T qp[TG_PMAX + 1];
        qp[0] = T(1);
        for (int e = 1; e <= p; ++e) qp[e] = qp[e - 1] * (T)q;
        const int ncn = ncoef_dev(nx + ny + nz);
        T acc = 0;
        for (int ch_i = 0; ch_i < nch; ++ch_i) {
            const int ch = t.child_first[c] + ch_i;
            const bool neg_x = !(t.cx[ch] & 1u), neg_y = !(t.cy[ch] & 1u), neg_z = !(t.cz[ch] & 1u);
            const double *Mc = M + ((size_t)ch * 2 + cls) * nc;
            for (int k = 0; k < ncn; ++k) {
                const int kx = c_mi_x[k], ky = c_mi_y[k], kz = c_mi_z[k];
                if (kx > nx || ky > ny || kz > nz) continue;
                const int dx = nx - kx, dy = ny - ky, dz = nz - kz;
                const bool neg = ((neg_x && (dx & 1)) ^ (neg_y && (dy & 1)) ^ (neg_z && (dz & 1)));
                T v = (T)(c_binom_f[nx][kx] * c_binom_f[ny][ky] * c_binom_f[nz][kz]) * qp[dx + dy + dz] * (T)Mc[k];
                acc += neg ? -v : v;
            }
        }
        M[((size_t)c * 2 + cls) * nc + n] = (double)acc;
    }
}

// ------------------------------------------------------------------ dual tree walk
// Breadth-first Algorithm 4 over UNORDERED pairs: a frontier of (a, b), a == b for self pairs.
// Self pair: leaf -> P2P(a, a); else all child pairs (ci <= cj), both cells opened.
// Distinct pair: well separated -> M2L; both leaves -> P2P; one leaf -> open the other; else
// open both (all child pairs).  This is the directed walk from (root, root) with each
// unordered pair kept once.
struct WalkOut {
    uint2 *front_out;
    uint2 *m2l;
    uint2 *p2p;
    unsigned long long *counters;   // [0] frontier, [1] m2l, [2] p2p
    unsigned long long cap_front, cap_m2l, cap_p2p;
};

__device__ __forceinline__ void emit(uint2 *arr, unsigned long long cap, unsigned long long *ctr, uint2 v)
{
    unsigned long long i = atomicAdd(ctr, 1ull);
    if (i < cap) arr[i] = v;
}

__global__ void walk_step(TreeView t, MacParams mp, const uint2 *front_in, int n_in, WalkOut o)
{
    for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < n_in; w += gridDim.x * blockDim.x) {
        const uint2 pr = front_in[w];
        const int a = (int)pr.x, b = (int)pr.y;
        const int na = t.nchild[a], nb = t.nchild[b];
        if (a == b) {
            if (na == 0) {
                emit(o.p2p, o.cap_p2p, o.counters + 2, make_uint2(a, a));
            } else {
                const int f = t.child_first[a];
                const unsigned long long k = (unsigned long long)na * (na + 1) / 2;
                unsigned long long base = atomicAdd(o.counters + 0, k);
                for (int i = 0; i < na; ++i)
                    for (int j = i; j < na; ++j, ++base)
                        if (base < o.cap_front) o.front_out[base] = make_uint2(f + i, f + j);
            }
            continue;
        }
        if (well_separated(t, mp, a, b)) {
            emit(o.m2l, o.cap_m2l, o.counters + 1, make_uint2(a, b));
        } else if (na == 0 && nb == 0) {
            emit(o.p2p, o.cap_p2p, o.counters + 2, make_uint2(a, b));
        } else if (na == 0) {
            unsigned long long base = atomicAdd(o.counters + 0, (unsigned long long)nb);
            for (int j = 0; j < nb; ++j, ++base)
                if (base < o.cap_front) o.front_out[base] = make_uint2(a, t.child_first[b] + j);
        } else if (nb == 0) {
            unsigned long long base = atomicAdd(o.counters + 0, (unsigned long long)na);
            for (int i = 0; i < na; ++i, ++base)
                if (base < o.cap_front) o.front_out[base] = make_uint2(t.child_first[a] + i, b);
        } else {
            unsigned long long base = atomicAdd(o.counters + 0, (unsigned long long)na * nb);
            for (int i = 0; i < na; ++i)
                for (int j = 0; j < nb; ++j, ++base)
                    if (base < o.cap_front) o.front_out[base] = make_uint2(t.child_first[a] + i, t.child_first[b] + j);
        }
    }
}

// ------------------------------------------------------------------ L2L (one level)
// L_c^n += sum_{k >= n, |k| <= p} L_P^k d^(k-n) / (k-n)!, d = z_c - z_P.  Thread per (cell, class, n).
template <class T>
__global__ void l2l_level(TreeView t, const Geom *gp, int lb, int le, int p, int nc, int ncls, T *L)
{
    const Geom g = *gp;
    const int64_t total = (int64_t)(le - lb) * ncls * nc;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
        const int c = lb + (int)(w / (ncls * nc));
        const int cls = (int)((w / nc) % ncls);
        const int n = (int)(w % nc);
        const int par = t.parent[c];
        if (par < 0) continue;
        const T dx = (T)(cell_centre(g, t, c, 0) - cell_centre(g, t, par, 0));
        const T dy = (T)(cell_centre(g, t, c, 1) - cell_centre(g, t, par, 1));
        const T dz = (T)(cell_centre(g, t, c, 2) - cell_centre(g, t, par, 2));
        const int nx = c_mi_x[n], ny = c_mi_y[n], nz = c_mi_z[n];
        const T *Lp = L + ((size_t)par * 2 + cls) * nc;
        T acc = 0;
        for (int k = 0; k < nc; ++k) {
            const int kx = c_mi_x[k], ky = c_mi_y[k], kz = c_mi_z[k];
            if (kx < nx || ky < ny || kz < nz) continue;
            T v = Lp[k] * (T)(c_inv_fact[c_mi_lookup[((kx - nx) * 9 + (ky - ny)) * 9 + (kz - nz)]]);
            for (int e = nx; e < kx; ++e) v *= dx;
            for (int e = ny; e < ky; ++e) v *= dy;
            for (int e = nz; e < kz; ++e) v *= dz;
            acc += v;
        }
        L[((size_t)c * 2 + cls) * nc + n] += acc;
    }
}

// ------------------------------------------------------------------ L2P
// phi = sum_n L^n rho^n / n!, a = -grad phi.  Thread per particle; writes acc4 (= initialises it).
template <class T, class T4>
__global__ void l2p_particles(int n, const T4 *pf, const int32_t *leaf_of, const uint8_t *fs, int masked, int p,
                              int nc, const T *L, double *acc4)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const T4 r = pf[s];
        const int c = leaf_of[s];
        const int cls = (masked && fs[s]) ? 1 : 0;
        const T *Lc = L + ((size_t)c * 2 + cls) * nc;
        T px[TG_PMAX + 1], py[TG_PMAX + 1], pz[TG_PMAX + 1];
        px[0] = py[0] = pz[0] = (T)1;
        for (int e = 1; e <= p; ++e) {
            px[e] = px[e - 1] * r.x;
            py[e] = py[e - 1] * r.y;
            pz[e] = pz[e - 1] * r.z;
        }
        T phi = 0, gx = 0, gy = 0, gz = 0;
        for (int k = 0; k < nc; ++k) {
            const int kx = c_mi_x[k], ky = c_mi_y[k], kz = c_mi_z[k];
            const T mono = px[kx] * py[ky] * pz[kz] * (T)c_inv_fact[k];
            phi += Lc[k] * mono;
            if (kx + ky + kz < p) {
                gx += Lc[c_mi_lookup[((kx + 1) * 9 + ky) * 9 + kz]] * mono;
                gy += Lc[c_mi_lookup[(kx * 9 + ky + 1) * 9 + kz]] * mono;
                gz += Lc[c_mi_lookup[(kx * 9 + ky) * 9 + kz + 1]] * mono;
            }
        }
        acc4[s] = -(double)gx;
        acc4[(size_t)n + s] = -(double)gy;
        acc4[2 * (size_t)n + s] = -(double)gz;
        acc4[3 * (size_t)n + s] = (double)phi;
    }
}

// ------------------------------------------------------------------ scatter back to input order
__global__ void scatter_out(int n, const uint32_t *perm, const double *acc4, double *acc, int64_t stride, double *pot)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const uint32_t q = perm[s];
        acc[q] = acc4[s];
        acc[stride + q] = acc4[(size_t)n + s];
        acc[2 * stride + q] = acc4[2 * (size_t)n + s];
        if (pot) pot[q] = acc4[3 * (size_t)n + s];
    }
}

__global__ void convert_moments(const double *M, float *Mf, int64_t count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        Mf[i] = (float)M[i];
}

// ------------------------------------------------------------------ direct summation (float64)
__global__ void direct_sum(int64_t n, const double *pos, const double *mass, const uint8_t *fast, int64_t n_sink,
                           const int64_t *sink_idx, int kernel, double eps, double *acc, double *pot)
{
    __shared__ double sx[256], sy[256], sz[256], sm[256];
    __shared__ uint8_t sf[256];
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < n_sink;
    const int64_t i = active ? (sink_idx ? sink_idx[t] : t) : 0;
    const double xi = active ? pos[i] : 0.0, yi = active ? pos[n + i] : 0.0, zi = active ? pos[2 * n + i] : 0.0;
    const bool fi = active && fast && fast[i];
    double ax = 0, ay = 0, az = 0, ph = 0;
    const double eps2 = eps * eps;
    for (int64_t j0 = 0; j0 < n; j0 += 256) {
        const int64_t j = j0 + threadIdx.x;
        if (j < n) {
            sx[threadIdx.x] = pos[j];
            sy[threadIdx.x] = pos[n + j];
            sz[threadIdx.x] = pos[2 * n + j];
            sm[threadIdx.x] = mass[j];
            sf[threadIdx.x] = fast ? fast[j] : 0;
        }
        __syncthreads();
        const int cnt = (int)((n - j0) < 256 ? (n - j0) : 256);
        if (active) {
            for (int q = 0; q < cnt; ++q) {
                if (j0 + q == i) continue;
                if (fi && sf[q]) continue;
                const double dx = sx[q] - xi, dy = sy[q] - yi, dz = sz[q] - zi;
                const double r2 = dx * dx + dy * dy + dz * dz;
                double g, phi;
                if (kernel == TG_KERNEL_PLUMMER) {
                    const double s2 = r2 + eps2, inv = 1.0 / sqrt(s2);
                    phi = -inv;
                    g = inv * inv * inv;
                } else if (r2 < eps2) {
                    const double u = sqrt(r2) / eps, u2 = u * u, u3 = u2 * u, u4 = u2 * u2, u5 = u4 * u;
                    phi = (3.0 * u4 * u3 - 15.0 * u3 * u3 + 28.0 * u5 - 21.0 * u4 + 7.0 * u2 - 3.0) / eps;
                    g = (21.0 * u5 - 90.0 * u4 + 140.0 * u3 - 84.0 * u2 + 14.0) / (eps * eps2);
                } else {
                    const double inv = 1.0 / sqrt(r2);
                    phi = -inv;
                    g = inv * inv * inv;
                }
                ax += sm[q] * g * dx;
                ay += sm[q] * g * dy;
                az += sm[q] * g * dz;
                ph += sm[q] * phi;
            }
        }
        __syncthreads();
    }
    if (active) {
        acc[t] = ax;
        acc[n_sink + t] = ay;
        acc[2 * n_sink + t] = az;
        if (pot) pot[t] = ph;
    }
}

tg_status direct_eval(tg_ctx *c, int64_t n, const double *pos, const double *mass, const uint8_t *fast,
                      int64_t n_sink, const int64_t *sink_idx, double *acc, double *pot)
{
    if (n_sink <= 0) return TG_OK;
    {
        ProfScope ps_(c, TG_K_OTHER);
        direct_sum<<<(int)((n_sink + 255) / 256), 256, 0, c->stream>>>(n, pos, mass, fast, n_sink, sink_idx,
                                                                      c->prm.kernel, c->prm.eps, acc, pot);
    }
    return cuda_check(c, cudaGetLastError(), "direct summation");
}

// ------------------------------------------------------------------ orchestration
static tg_status run_walk(tg_ctx *c, const TreeView &t, const Geom *d_geom_host_unused, int64_t *n_m2l,
                          int64_t *n_p2p)
{
    (void)d_geom_host_unused;
    tg_status st;
    MacParams mp;
    mp.theta2 = c->prm.theta * c->prm.theta;
    mp.kappa2 = c->prm.kappa * c->prm.kappa;
    mp.eps = c->prm.eps;
    mp.wendland = c->prm.kernel == TG_KERNEL_WENDLAND_C2;
    // log2 of the root side, copied back with the other counters below
    mp.log2L = 0;
    {
        const Geom *dg = static_cast<const Geom *>(c->buf[B_GEOM].p);
        cudaMemcpyAsync(c->h_pinned + 32, &dg->log2L, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_check(c, e, "walk setup");
        mp.log2L = *reinterpret_cast<int *>(c->h_pinned + 32);
    }
    size_t cap_front = (size_t)t.ncell * 16 + 1024, cap_m2l = (size_t)t.ncell * 64 + 1024,
           cap_p2p = (size_t)t.ncell * 32 + 1024;
    for (int attempt = 0; attempt < 6; ++attempt) {
        uint2 *f0, *f1, *m2l, *p2p;
        unsigned long long *ctr;
        if ((st = ensure_t(c, B_FRONT0, cap_front, &f0)) || (st = ensure_t(c, B_FRONT1, cap_front, &f1)) ||
            (st = ensure_t(c, B_M2L, cap_m2l, &m2l)) || (st = ensure_t(c, B_P2P, cap_p2p, &p2p)) ||
            (st = ensure_t(c, B_WALK_CNT, 8, &ctr)))
            return st;
        const uint2 root = make_uint2(0, 0);
        cudaMemcpyAsync(f0, &root, sizeof(uint2), cudaMemcpyHostToDevice, c->stream);
        cudaMemsetAsync(ctr, 0, 8 * sizeof(unsigned long long), c->stream);
        unsigned long long n_in = 1, tot_m2l = 0, tot_p2p = 0;
        bool overflow = false;
        size_t need_front = 0;
        while (n_in > 0) {
            cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), c->stream);   // frontier counter only
            WalkOut o{f1, m2l, p2p, ctr, cap_front, cap_m2l, cap_p2p};
            {
                ProfScope ps_(c, TG_K_WALK);
                walk_step<<<grid_for((int64_t)n_in, 128), 128, 0, c->stream>>>(t, mp, f0, (int)n_in, o);
            }
            cudaMemcpyAsync(c->h_pinned, ctr, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
            cudaError_t e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return cuda_check(c, e, "walk step");
            const unsigned long long *h = reinterpret_cast<const unsigned long long *>(c->h_pinned);
            n_in = h[0];
            tot_m2l = h[1];
            tot_p2p = h[2];
            if (n_in > cap_front || tot_m2l > cap_m2l || tot_p2p > cap_p2p) {
                overflow = true;
                need_front = n_in > need_front ? n_in : need_front;
                break;
            }
            std::swap(f0, f1);
            std::swap(c->buf[B_FRONT0], c->buf[B_FRONT1]);
        }
        if (!overflow) {
            *n_m2l = (int64_t)tot_m2l;
            *n_p2p = (int64_t)tot_p2p;
            return TG_OK;
        }
        cap_front = std::max(cap_front * 2, need_front + need_front / 2);
        if (tot_m2l > cap_m2l) cap_m2l = tot_m2l * 2;
        else cap_m2l = cap_m2l * 3 / 2;
        if (tot_p2p > cap_p2p) cap_p2p = tot_p2p * 2;
        else cap_p2p = cap_p2p * 3 / 2;
    }
    return set_err(c, TG_ERR_CAPACITY, "interaction lists did not fit after regrowth");
}

template <class T, class T4>
static tg_status eval_typed(tg_ctx *c, int n, int ncell, const TreeView &t, const Geom *d_geom, bool masked,
                            int64_t n_m2l, int64_t n_p2p)
{
    tg_status st;
    const int p = c->prm.p, nc = ncoef(p);
    const double *xs = static_cast<const double *>(c->buf[B_XS].p), *ys = static_cast<const double *>(c->buf[B_YS].p),
                 *zs = static_cast<const double *>(c->buf[B_ZS].p), *ms = static_cast<const double *>(c->buf[B_MS].p);
    const uint8_t *fs = static_cast<const uint8_t *>(c->buf[B_FS].p);
    T4 *pf;
    int32_t *leaf_of;
    double *M, *acc4;
    T *L;
    if ((st = ensure_t(c, B_PF, n, &pf)) || (st = ensure_t(c, B_LEAF_OF, n, &leaf_of)) ||
        (st = ensure_t(c, B_MOM, (size_t)ncell * 2 * nc, &M)) || (st = ensure_t(c, B_LOC, (size_t)ncell * 2 * nc, &L)) ||
        (st = ensure_t(c, B_ACC, (size_t)4 * n, &acc4)))
        return st;
    const int ncls = masked ? 2 : 1;
    {
        ProfScope ps_(c, TG_K_UP);
        leaf_particles<T4><<<grid_for((int64_t)ncell * 32, 256), 256, 0, c->stream>>>(t, d_geom, xs, ys, zs, ms, pf, leaf_of);
    }
    // upward pass
    {
        ProfScope ps_(c, TG_K_UP);
        p2m_leaves<T><<<grid_for((int64_t)ncell * 32, 256), 256, 0, c->stream>>>(t, d_geom, xs, ys, zs, ms, fs, p, nc, M);
    }
    const int nlev = (int)c->level_begin.size() - 1;
    for (int l = nlev - 2; l >= 0; --l) {
        const int lb = c->level_begin[l], le = c->level_begin[l + 1];
        {
            ProfScope ps_(c, TG_K_UP);
            m2m_level<T><<<grid_for((int64_t)(le - lb) * 2 * nc, 128), 128, 0, c->stream>>>(t, d_geom, lb, le, p, nc, M);
        }
    }
    // M2L (mutual) into zeroed local expansions
    cudaMemsetAsync(L, 0, sizeof(T) * (size_t)ncell * 2 * nc, c->stream);
    const uint2 *m2l = static_cast<const uint2 *>(c->buf[B_M2L].p);
    const uint2 *p2p = static_cast<const uint2 *>(c->buf[B_P2P].p);
    const Mom<T> mom = make_moments<T>(c, M, (size_t)ncell * 2 * nc, &st);
    if (st) return st;
    if (n_m2l > 0) {
        if ((st = launch_m2l<T>(c, t, d_geom, m2l, n_m2l, mom, L, p, nc, masked))) return st;
    }
    // downward pass
    for (int l = 1; l < nlev; ++l) {
        const int lb = c->level_begin[l], le = c->level_begin[l + 1];
        {
            ProfScope ps_(c, TG_K_DOWN);
            l2l_level<T><<<grid_for((int64_t)(le - lb) * ncls * nc, 128), 128, 0, c->stream>>>(t, d_geom, lb, le, p, nc,
                                                                                           ncls, L);
        }
    }
    {
        ProfScope ps_(c, TG_K_DOWN);
        l2p_particles<T, T4><<<grid_for(n, 128), 128, 0, c->stream>>>(n, pf, leaf_of, fs, masked ? 1 : 0, p, nc, L, acc4);
    }
    // P2P (mutual) adds onto the L2P result
    if (n_p2p > 0) {
        if ((st = launch_p2p<T, T4>(c, t, d_geom, p2p, n_p2p, pf, fs, masked, acc4))) return st;
    }
    return cuda_check(c, cudaGetLastError(), "fmm evaluation");
}

tg_status fmm_eval(tg_ctx *c, int n, const double *pos, int64_t stride, const int64_t *sub, const double *mass,
                   const uint8_t *fast, double *acc, int64_t out_stride, double *pot, bool keep_tree)
{
    (void)keep_tree;
    tg_status st;
    if (n <= 0) return TG_OK;
    Geom *d_geom;
    if ((st = ensure_t(c, B_GEOM, 1, &d_geom))) return st;
    if ((st = root_cube(c, n, pos, stride, sub, d_geom))) return st;
    if ((st = keys_sort_gather(c, n, pos, stride, sub, mass, fast, d_geom))) return st;
    int ncell = 0;
    if ((st = build_octree(c, n, &ncell))) return st;
    TreeView t = tree_view(c, n, ncell);
    int64_t n_m2l = 0, n_p2p = 0;
    if ((st = run_walk(c, t, d_geom, &n_m2l, &n_p2p))) return st;
    c->last_n = n;
    c->last_ncell = ncell;
    c->last_nm2l = n_m2l;
    c->last_np2p = n_p2p;
    const bool masked = fast != nullptr;
    if (c->prm.precision == TG_PREC_FP32) st = eval_typed<float, float4>(c, n, ncell, t, d_geom, masked, n_m2l, n_p2p);
    else st = eval_typed<double, dbl4>(c, n, ncell, t, d_geom, masked, n_m2l, n_p2p);
    if (st) return st;
    const uint32_t *perm = static_cast<const uint32_t *>(c->buf[B_VALS0].p);
    const double *acc4 = static_cast<const double *>(c->buf[B_ACC].p);
    {
        ProfScope ps_(c, TG_K_DOWN);
        scatter_out<<<grid_for(n, 256), 256, 0, c->stream>>>(n, perm, acc4, acc, out_stride, pot);
    }
    c->stats.evaluations += 1;
    c->stats.sink_forces += n;
    c->stats.m2l_pairs += n_m2l;
    c->stats.p2p_cell_pairs += n_p2p;
    c->stats.cells += ncell;
    return cuda_check(c, cudaGetLastError(), "fmm scatter");
}

}  // namespace tg
