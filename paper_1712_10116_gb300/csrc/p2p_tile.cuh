// p2p_tile.cuh -- mutual particle-particle interaction of leaf pairs (P2P, Sec. 2.1, Eq. 2).
// Each unordered leaf pair (A, B) is visited once; for every particle pair the kernel value is
// computed once and applied with opposite signs to both particles (a_i += m_j g d, a_j -= m_i g d).
// Positions are relative to leaf centres (exact float offsets between centres).  F-F pairs are
// skipped when classes are given (kickS2F feels slow masses only).
#pragma once
#include "tg_common.cuh"

namespace tg {

constexpr int kP2PThreads = 64;

// PTX rsqrt.approx.ftz.f32: the hardware approximate reciprocal square root with a subnormal
// argument flushed to zero.  Only used where the argument is at least eps^2 (or a squared
// distance between distinct leaves, which is larger), so the flush never applies and the
// subnormal handling of the non-flushing form is saved.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <class T>
__device__ __forceinline__ T tg_rsqrt(T x);
// float: hardware reciprocal square root refined by one Newton step (relative error ~1e-7)
template <>
__device__ __forceinline__ float tg_rsqrt<float>(float x)
{
    const float y = rsqrtf(x);
    return y * fmaf(-0.5f * x, y * y, 1.5f);
}
template <>
__device__ __forceinline__ double tg_rsqrt<double>(double x) { return rsqrt(x); }

// pair kernel: g = phi'(r)/r and phi(r) of a unit mass, Wendland C2 (Eq. 8) or Plummer.
// For u = r/eps in [1/2, 1) the Wendland terms are evaluated in the equivalent forms
//   g = M(u)/r^3,  M(u) = 1 - (1-u)^5 (21u^3 + 15u^2 + 5u + 1)   (enclosed mass fraction),
//   phi = -(1 - (1-u)^6 (3u^2 + 3u + 1))/r,
// which avoid the cancellation of the expanded polynomial near u = 1 in float32; below u = 1/2
// the expanded (Horner) forms are well conditioned.
template <class T, int KERNEL>
__device__ __forceinline__ void pair_kernel(T r2, T eps, T eps2, T inv_eps, T inv_eps3, T &g, T &phi)
{
    if (KERNEL == TG_KERNEL_PLUMMER) {
        const T si = tg_rsqrt<T>(r2 + eps2);
        phi = -si;
        g = si * si * si;
    } else if (r2 >= eps2) {
        const T ri = tg_rsqrt<T>(r2);
        phi = -ri;
        g = ri * ri * ri;
    } else if (r2 >= T(0.25) * eps2) {
        const T ri = tg_rsqrt<T>(r2);
        const T u = r2 * ri * inv_eps, w = T(1) - u, w2 = w * w, w5 = w2 * w2 * w;
        const T mfrac = T(1) - w5 * (((T(21) * u + T(15)) * u + T(5)) * u + T(1));
        g = mfrac * ri * ri * ri;
        phi = -(T(1) - w5 * w * ((T(3) * u + T(3)) * u + T(1))) * ri;
    } else {
        const T u = sqrt(r2) * inv_eps, u2 = u * u;
        // phi = (1/eps)(3u^7 - 15u^6 + 28u^5 - 21u^4 + 7u^2 - 3); g = (1/eps^3)(21u^5 - 90u^4 + 140u^3 - 84u^2 + 14)
        phi = ((((((T(3) * u - T(15)) * u + T(28)) * u - T(21)) * u2 + T(7)) * u2) - T(3)) * inv_eps;
        g = ((((T(21) * u - T(90)) * u + T(140)) * u - T(84)) * u2 + T(14)) * inv_eps3;
    }
}

// Batched path (walk_ctr non-null): the distinct leaf pairs [0, walk_ctr[2]) and the walk_ctr[4] self
// pairs at the end of the buffer (capacity cap_p2p) in one launch.
template <class T, class T4, bool MASKED, int KERNEL>
__global__ void __launch_bounds__(kP2PThreads) p2p_mutual(TreeView t, const Geom *gp, const uint2 *pairs,
                                                          int64_t npairs, const T4 *pf, const uint8_t *fs, T eps,
                                                          double *acc4, int n, unsigned long long *pair_counter,
                                                          const unsigned long long *walk_ctr = nullptr,
                                                          unsigned long long cap_p2p = 0)
{
    int64_t ndist = npairs, self0 = 0;
    if (walk_ctr) {
        ndist = (int64_t)walk_ctr[2];
        self0 = (int64_t)(cap_p2p - walk_ctr[4]);
        npairs = ndist + (int64_t)walk_ctr[4];
    }
    __shared__ T4 sb[kMaxNcrit];
    __shared__ uint8_t sfb[kMaxNcrit];
    __shared__ T colacc[kMaxNcrit][4];
    const Geom g = *gp;
    const int lane = threadIdx.x & 31;
    const T eps2 = eps * eps, inv_eps = T(1) / eps, inv_eps3 = inv_eps * inv_eps * inv_eps;
    unsigned long long my_pairs = 0;
    for (int64_t w = blockIdx.x; w < npairs; w += gridDim.x) {
        const uint2 pr = pairs[w < ndist ? w : self0 + (w - ndist)];
        const int a = (int)pr.x, b = (int)pr.y;
        const int fa = t.first[a], na = t.count[a], fb = t.first[b], nb = t.count[b];
        const double sb_side = ldexp(g.L, -(int)t.level[b]), sa_side = ldexp(g.L, -(int)t.level[a]);
        const T ox = (T)(((double)t.cx[b] + 0.5) * sb_side - ((double)t.cx[a] + 0.5) * sa_side);
        const T oy = (T)(((double)t.cy[b] + 0.5) * sb_side - ((double)t.cy[a] + 0.5) * sa_side);
        const T oz = (T)(((double)t.cz[b] + 0.5) * sb_side - ((double)t.cz[a] + 0.5) * sa_side);
        const bool self = a == b;
        // B is staged in chunks of kMaxNcrit (leaves at the deepest level may exceed n_crit)
        for (int j0 = 0; j0 < nb; j0 += kMaxNcrit) {
            const int nbc = min(kMaxNcrit, nb - j0);
            __syncthreads();
            for (int j = threadIdx.x; j < nbc; j += blockDim.x) {
                T4 v = pf[fb + j0 + j];
                v.x += ox;
                v.y += oy;
                v.z += oz;
                sb[j] = v;
                sfb[j] = MASKED ? fs[fb + j0 + j] : 0;
                colacc[j][0] = colacc[j][1] = colacc[j][2] = colacc[j][3] = T(0);
            }
            __syncthreads();
            for (int i0 = 0; i0 < na; i0 += blockDim.x) {
                const int i = i0 + threadIdx.x;
                const bool row = i < na;
                T4 pi;
                if (row) pi = pf[fa + i];
                else pi.x = pi.y = pi.z = pi.w = T(0);
                const uint8_t fi = (MASKED && row) ? fs[fa + i] : 0;
                T rax = 0, ray = 0, raz = 0, rph = 0;
                for (int j = 0; j < nbc; ++j) {
                    const T4 pj = sb[j];
                    const bool use = row && (!self || j0 + j > i) && !(MASKED && fi && sfb[j]);
                    const T dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    T gk, ph;
                    pair_kernel<T, KERNEL>(use ? r2 : T(1), eps, eps2, inv_eps, inv_eps3, gk, ph);
                    if (!use) {
                        gk = T(0);
                        ph = T(0);
                    }
                    my_pairs += use ? 1 : 0;
                    rax += pj.w * gk * dx;
                    ray += pj.w * gk * dy;
                    raz += pj.w * gk * dz;
                    rph += pj.w * ph;
                    T cx = -pi.w * gk * dx, cy = -pi.w * gk * dy, cz = -pi.w * gk * dz, cp = pi.w * ph;
                    cx = warp_sum(cx);
                    cy = warp_sum(cy);
                    cz = warp_sum(cz);
                    cp = warp_sum(cp);
                    if (lane == 0) {
                        atomicAdd(&colacc[j][0], cx);
                        atomicAdd(&colacc[j][1], cy);
                        atomicAdd(&colacc[j][2], cz);
                        atomicAdd(&colacc[j][3], cp);
                    }
                }
                if (row) {
                    atomicAdd(&acc4[fa + i], (double)rax);
                    atomicAdd(&acc4[(size_t)n + fa + i], (double)ray);
                    atomicAdd(&acc4[2 * (size_t)n + fa + i], (double)raz);
                    atomicAdd(&acc4[3 * (size_t)n + fa + i], (double)rph);
                }
            }
            __syncthreads();
            for (int j = threadIdx.x; j < nbc; j += blockDim.x) {
                atomicAdd(&acc4[fb + j0 + j], (double)colacc[j][0]);
                atomicAdd(&acc4[(size_t)n + fb + j0 + j], (double)colacc[j][1]);
                atomicAdd(&acc4[2 * (size_t)n + fb + j0 + j], (double)colacc[j][2]);
                atomicAdd(&acc4[3 * (size_t)n + fb + j0 + j], (double)colacc[j][3]);
            }
        }
    }
    my_pairs = warp_sum(my_pairs);
    if (lane == 0 && my_pairs) atomicAdd(pair_counter, my_pairs);
}

// ------------------------------------------------------------------ float32 warp tiles
// Building blocks of the float32 P2P launch (p2p_owner.cuh): the pair value and the tile of one
// leaf pair, used there for the self pairs (A, A).

// float32 pair value: Newton by default, Wendland correction inside eps (rare, predicated).
// NEAR = false: the caller knows r >= eps for every pair (leaf cubes at least eps apart).
template <int KERNEL, bool NEAR = true>
__device__ __forceinline__ void pair_kernel_f32(float r2, float eps, float eps2, float inv_eps, float inv_eps3, float &g,
                                                float &phi)
{
    if (KERNEL == TG_KERNEL_PLUMMER) {
        const float si = tg_rsqrt<float>(r2 + eps2);
        phi = -si;
        g = si * si * si;
        return;
    }
    const float ri = NEAR ? rsqrtf(r2) : rsqrt_ftz(r2);   // far pairs: r2 >= eps^2
    phi = -ri;
    g = ri * ri * ri;
    if (NEAR && r2 < eps2) pair_kernel<float, TG_KERNEL_WENDLAND_C2>(r2, eps, eps2, inv_eps, inv_eps3, g, phi);
}

// One leaf pair.  Rows = particles of A, ROWS per lane (row i0 + lane + 32 r), chunks of 32*ROWS;
// columns = particles of B, staged once in the warp's shared-memory slice (positions shifted into
// A's frame) and read in batches of 8.  A lane keeps its rows' sums in registers and its 8 x 4
// column partials.  Lane l visits the 8 columns of a batch in the order c ^ ((l >> 2) & 7), so its
// partial for logical entry e sits in register e ^ (l & 28); the first three stages of the warp
// reduce-scatter (partners l ^ 16, l ^ 8, l ^ 4) then need no selects, and lane l ends with column
// l/4, component l%4, which it adds to global memory.  SELF (A == B) keeps column index > row index.
template <int KERNEL, bool SELF, int ROWS, bool NEAR>
__device__ __noinline__ void p2p_pair_f32(const float4 *__restrict__ pf, int fa, int na, int fb, int nb, float ox, float oy,
                                          float oz, float eps, double *acc4, int n, int lane, float4 *sq)
{
    const float eps2 = eps * eps, inv_eps = 1.0f / eps, inv_eps3 = inv_eps * inv_eps * inv_eps;
    const int cperm = (lane >> 2) & 7;
    for (int jc = 0; jc < nb; jc += kMaxNcrit) {
        const int nbc = min(kMaxNcrit, nb - jc);
        __syncwarp();
        for (int j = lane; j < nbc; j += 32) {
            float4 q = pf[fb + jc + j];
            q.x += ox;
            q.y += oy;
            q.z += oz;
            sq[j] = q;
        }
        __syncwarp();
        for (int i0 = 0; i0 < na; i0 += 32 * ROWS) {
            float4 p[ROWS];
            int ir[ROWS];
            float ra[ROWS][4];
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                ir[r] = i0 + lane + 32 * r;
                p[r] = ir[r] < na ? pf[fa + ir[r]] : make_float4(1e8f, 1e8f, 1e8f, 0.f);   // far away, massless
                ra[r][0] = ra[r][1] = ra[r][2] = ra[r][3] = 0.f;
            }
            for (int j0 = 0; j0 < nbc; j0 += 8) {
                float col[32];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int j = j0 + (c ^ cperm);
                    float cx = 0.f, cy = 0.f, cz = 0.f, cp = 0.f;
                    if (j < nbc) {
                        const float4 q = sq[j];
#pragma unroll
                        for (int r = 0; r < ROWS; ++r) {
                            const float dx = q.x - p[r].x, dy = q.y - p[r].y, dz = q.z - p[r].z;
                            float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                            bool use = true;
                            if (SELF) {
                                use = jc + j > ir[r];
                                r2 = use ? r2 : 1.0f;
                            }
                            float gk, ph;
                            pair_kernel_f32<KERNEL, NEAR>(r2, eps, eps2, inv_eps, inv_eps3, gk, ph);
                            if (SELF) {
                                gk = use ? gk : 0.f;
                                ph = use ? ph : 0.f;
                            }
                            const float mq = q.w * gk, mp = p[r].w * gk;
                            ra[r][0] = fmaf(mq, dx, ra[r][0]);
                            ra[r][1] = fmaf(mq, dy, ra[r][1]);
                            ra[r][2] = fmaf(mq, dz, ra[r][2]);
                            ra[r][3] = fmaf(q.w, ph, ra[r][3]);
                            cx = fmaf(-mp, dx, cx);
                            cy = fmaf(-mp, dy, cy);
                            cz = fmaf(-mp, dz, cz);
                            cp = fmaf(p[r].w, ph, cp);
                        }
                    }
                    col[4 * c + 0] = cx;
                    col[4 * c + 1] = cy;
                    col[4 * c + 2] = cz;
                    col[4 * c + 3] = cp;
                }
                // reduce-scatter: column bits (partners l^16, l^8, l^4) without selects ...
#pragma unroll
                for (int h = 16; h >= 4; h >>= 1)
#pragma unroll
                    for (int q = 0; q < h; ++q) col[q] += __shfl_xor_sync(0xffffffffu, col[q + h], h);
                // ... component bits (l^2, l^1) with selects
#pragma unroll
                for (int h = 2; h >= 1; h >>= 1) {
                    const bool hi = (lane & h) != 0;
#pragma unroll
                    for (int q = 0; q < h; ++q) {
                        const float send = hi ? col[q] : col[q + h];
                        const float keep = hi ? col[q + h] : col[q];
                        col[q] = keep + __shfl_xor_sync(0xffffffffu, send, h);
                    }
                }
                const int cj = lane >> 2, comp = lane & 3;
                if (j0 + cj < nbc) atomicAdd(&acc4[(size_t)comp * n + fb + jc + j0 + cj], f2d_exact(col[0]));
            }
#pragma unroll
            for (int r = 0; r < ROWS; ++r)
                if (ir[r] < na)
#pragma unroll
                    for (int comp = 0; comp < 4; ++comp)
                        atomicAdd(&acc4[(size_t)comp * n + fa + ir[r]], f2d_exact(ra[r][comp]));
        }
    }
}

template <class T, class T4>
static tg_status launch_p2p_generic(tg_ctx *c, const TreeView &t, const Geom *d_geom, const uint2 *pairs, int64_t npairs,
                            const T4 *pf, const uint8_t *fs, bool masked, double *acc4)
{
    const int grid = (int)std::min<int64_t>(npairs, (int64_t)c->num_sms * 16);
    const T eps = (T)c->prm.eps;
    unsigned long long *ctr = c->d_counters;
    const int kern = c->prm.kernel;
    ProfScope ps_(c, TG_K_P2P);
#define TG_P2P_LAUNCH(M, K) \
    p2p_mutual<T, T4, M, K><<<grid, kP2PThreads, 0, c->stream>>>(t, d_geom, pairs, npairs, pf, fs, eps, acc4, t.n, ctr)
    if (masked) {
        if (kern == TG_KERNEL_PLUMMER) TG_P2P_LAUNCH(true, TG_KERNEL_PLUMMER);
        else TG_P2P_LAUNCH(true, TG_KERNEL_WENDLAND_C2);
    } else {
        if (kern == TG_KERNEL_PLUMMER) TG_P2P_LAUNCH(false, TG_KERNEL_PLUMMER);
        else TG_P2P_LAUNCH(false, TG_KERNEL_WENDLAND_C2);
    }
#undef TG_P2P_LAUNCH
    return cuda_check(c, cudaGetLastError(), "p2p launch");
}

// float64 P2P with every count on the device (batched path): one launch over the distinct and self pairs
tg_status launch_p2p_f64_dev(tg_ctx *c, const TreeView &t, const Geom *d_geom, const unsigned long long *walk_ctr,
                             const uint2 *p2p, size_t cap_p2p, const dbl4 *pf, const uint8_t *fs, double *acc4, int stride)
{
    const int grid = c->num_sms * 16;
    const double eps = c->prm.eps;
    ProfScope ps_(c, TG_K_P2P);
    if (c->prm.kernel == TG_KERNEL_PLUMMER)
        p2p_mutual<double, dbl4, true, TG_KERNEL_PLUMMER><<<grid, kP2PThreads, 0, c->stream>>>(
            t, d_geom, p2p, 0, pf, fs, eps, acc4, stride, c->d_counters, walk_ctr, (unsigned long long)cap_p2p);
    else
        p2p_mutual<double, dbl4, true, TG_KERNEL_WENDLAND_C2><<<grid, kP2PThreads, 0, c->stream>>>(
            t, d_geom, p2p, 0, pf, fs, eps, acc4, stride, c->d_counters, walk_ctr, (unsigned long long)cap_p2p);
    return cuda_check(c, cudaGetLastError(), "p2p launch (device sizes, float64)");
}

// float64 P2P: one block per leaf pair, the distinct pairs then the self pairs (the tile tells them
// apart at run time and masks fast-fast pairs one by one); float32 goes through p2p_owner.cuh.
tg_status launch_p2p_f64(tg_ctx *c, const TreeView &t, const Geom *d_geom, const uint2 *pairs, int64_t npairs,
                         const uint2 *self_pairs, int64_t nself, const dbl4 *pf, const uint8_t *fs, bool masked,
                         double *acc4)
{
    tg_status st;
    if (npairs > 0 && (st = launch_p2p_generic<double, dbl4>(c, t, d_geom, pairs, npairs, pf, fs, masked, acc4)))
        return st;
    if (nself > 0 && (st = launch_p2p_generic<double, dbl4>(c, t, d_geom, self_pairs, nself, pf, fs, masked, acc4)))
        return st;
    return TG_OK;
}

}  // namespace tg
