// fmm.cu -- one FMM evaluation (the Poisson-solver call of Algorithm 3, Zhu 2017):
// upward pass (P2M, M2M), dual tree walk (Algorithm 4) emitting blocks of unordered cell pairs,
// mutual M2L and P2P (Sec. 2.1: F_AB = -F_BA), downward pass (L2L, L2P) and the
// float64 direct summation (tg_direct_forces) that the force errors are measured against.
//
// Expansions are Cartesian Taylor series truncated at total degree p, stored normalised by the
// cell side s:
//   M~_A^j = sum_{i in A} m_i ((x_i - z_A)/s_A)^j,   phi(x) = (1/s) sum_n L~^n ((x - z)/s)^n / n!.
// With this scaling the translation operators have constant coefficients (a child's centre is at
// +-s_P/4 from its parent's), and every stored number is O(1) in any precision.
//
// Each cell carries two moment classes (slow S and fast F particles) and two local expansions:
// L_all (slow sinks, sources S + F) and L_S (fast sinks, sources S only).  One walk and one
// evaluation thus serve a kickFS2S + kickS2F pair of Algorithm 2.
#include "tg_common.cuh"
#include "tg_tables.cuh"

namespace tg {

// Eq. (1) with R = kappa * side, and the rule that cell pairs closer than eps (cube gap) never use
// M2L for the Wendland kernel.  In integer units of half the finer cell's side the tests read
//   (double)d2 * theta^2 > kappa^2 * (2 (h_a + h_b))^2   and   (double)g2 > (eps / u)^2,
// where one of h_a, h_b is 1 and the other 2^dl (dl = level difference), u = L / 2^(lf+1).  Both
// sides are monotone in the integers d2, g2, so the host turns each comparison into an integer
// threshold per dl (MAC) and per finer level lf (gap), reproducing the float64 decisions exactly.
struct MacParams {
    long long mac_min_d2[kMaxLevel + 1];   // well separated iff d2 >= mac_min_d2[dl]
    long long gap_min_g2[kMaxLevel + 1];   // gap rule passes iff g2 >= gap_min_g2[lf]
    int wendland;
    int sphere;                            // TG_MAC_SPHERE: R_a + R_b < theta d with the cell radii
    int log2L;
    double theta;
};

// smallest integer v >= 0 with pred(v) (pred monotone), searched over [0, 2^62)
template <class Pred>
static long long min_true(Pred pred)
{
    long long lo = 0, hi = 1ll << 62;   // pred(hi) assumed true
    if (pred(0)) return 0;
    while (hi - lo > 1) {
        const long long mid = lo + (hi - lo) / 2;
        if (pred(mid)) hi = mid;
        else lo = mid;
    }
    return hi;
}

static MacParams make_mac_params(const tg_params &prm, int log2L)
{
    MacParams mp;
    const double theta2 = prm.theta * prm.theta, kappa2 = prm.kappa * prm.kappa;
    for (int dl = 0; dl <= kMaxLevel; ++dl) {
        const double rsum = (double)(2 * (1ll + (1ll << dl)));
        const double K = kappa2 * (rsum * rsum);
        mp.mac_min_d2[dl] = min_true([&](long long d2) { return (double)d2 * theta2 > K; });
    }
    for (int lf = 0; lf <= kMaxLevel; ++lf) {
        const double eu = ldexp(prm.eps, lf + 1 - log2L);
        const double E = eu * eu;
        mp.gap_min_g2[lf] = min_true([&](long long g2) { return (double)g2 > E; });
    }
    mp.wendland = prm.kernel == TG_KERNEL_WENDLAND_C2;
    mp.sphere = prm.mac == TG_MAC_SPHERE;
    mp.log2L = log2L;
    mp.theta = prm.theta;
    return mp;
}

// The test from the cells' levels and integer coordinates (the dual walk loads the eight column cells
// of a pair once, side by side); a and b are only read by the sphere criterion.
struct CellGeo {
    uint32_t x, y, z;
    int level;
};
__device__ __forceinline__ bool well_separated_geo(const TreeView &t, const MacParams &mp, int a, const CellGeo &ga,
                                                   int b, const CellGeo &gb)
{
    const int la = ga.level, lb = gb.level;
    const int lf = la > lb ? la : lb;
    const long long ha = 1ll << (lf - la), hb = 1ll << (lf - lb);
    const long long dxs[3] = {centre_delta(ga.x, la, gb.x, lb, lf), centre_delta(ga.y, la, gb.y, lb, lf),
                              centre_delta(ga.z, la, gb.z, lb, lf)};
    long long d2 = 0, g2 = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const long long dk = dxs[k] < 0 ? -dxs[k] : dxs[k];
        d2 += dk * dk;
        const long long gk = dk - (ha + hb);
        if (gk > 0) g2 += gk * gk;
    }
    if (mp.sphere) {
        // R_a + R_b < theta d: a float test settles everything but a 1e-5 band about the threshold,
        // where the decision is taken in float64 with explicitly rounded operations
        const float df = sqrtf((float)d2) * pow2f(mp.log2L - lf - 1);
        const float lhs = t.radf[a] + t.radf[b], rhs = (float)mp.theta * df;
        bool ok;
        if (lhs < rhs * (1.0f - 1e-5f)) ok = true;
        else if (lhs > rhs * (1.0f + 1e-5f)) ok = false;
        else {
            const double d = sqrt((double)d2) * ldexp(1.0, mp.log2L - lf - 1);
            ok = __dadd_rn(t.rad[a], t.rad[b]) < __dmul_rn(mp.theta, d);
        }
        if (!ok) return false;
    } else if (d2 < mp.mac_min_d2[la > lb ? la - lb : lb - la]) {
        return false;
    }
    if (mp.wendland && g2 < mp.gap_min_g2[lf]) return false;
    return true;
}

__device__ __forceinline__ bool well_separated(const TreeView &t, const MacParams &mp, int a, int b)
{
    return well_separated_geo(t, mp, a, CellGeo{t.cx[a], t.cy[a], t.cz[a], (int)t.level[a]}, b,
                              CellGeo{t.cx[b], t.cy[b], t.cz[b], (int)t.level[b]});
}

// ------------------------------------------------------------------ enclosing radii (TG_MAC_SPHERE)
// Cell centre and distances with explicitly rounded float64 operations (no contraction into FMA), so
// that the radii are reproducible bit for bit: the acceptance decisions depend on them.
__device__ __forceinline__ double exact_centre(const Geom &g, const TreeView &t, int c, int axis)
{
    const uint32_t ci = axis == 0 ? t.cx[c] : (axis == 1 ? t.cy[c] : t.cz[c]);
    return __dadd_rn(g.lo[axis], __dmul_rn((double)ci + 0.5, ldexp(g.L, -(int)t.level[c])));
}

// leaves: the farthest particle from the cell centre (warp per leaf, lanes over particles)
__global__ void cell_radii_leaves(TreeView t, const Geom *gp, const double *xs, const double *ys, const double *zs,
                                  double *rad, float *radf)
{
    const Geom g = *gp;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = warp; c < t.ncell; c += nwarps) {
        if (t.nchild[c] != 0) continue;
        const double zx = exact_centre(g, t, c, 0), zy = exact_centre(g, t, c, 1), zz = exact_centre(g, t, c, 2);
        double r = 0.0;
        for (int s = t.first[c] + lane; s < t.first[c] + t.count[c]; s += 32) {
            const double dx = __dsub_rn(xs[s], zx), dy = __dsub_rn(ys[s], zy), dz = __dsub_rn(zs[s], zz);
            const double d = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
            r = d > r ? d : r;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double v = __shfl_xor_sync(0xffffffffu, r, o);
            r = v > r ? v : r;
        }
        if (lane == 0) {
            rad[c] = r;
            radf[c] = (float)r;
        }
    }
}

// parents of one level: max over children of |z_c - z_p| + R_c, with |z_c - z_p| = sqrt(3) side / 4
__global__ void cell_radii_level(TreeView t, int lb, int le, const Geom *gp, double *rad, float *radf)
{
    const double L = gp->L;
    for (int c = lb + blockIdx.x * blockDim.x + threadIdx.x; c < le; c += gridDim.x * blockDim.x) {
        const int nch = t.nchild[c];
        if (nch == 0) continue;
        const double dcp = __dmul_rn(sqrt(3.0), ldexp(L, -((int)t.level[c] + 2)));
        double r = 0.0;
        for (int q = 0; q < nch; ++q) {
            const double v = __dadd_rn(dcp, rad[t.child_first[c] + q]);
            r = v > r ? v : r;
        }
        rad[c] = r;
        radf[c] = (float)r;
    }
}

static tg_status cell_radii(tg_ctx *c, TreeView &t, const Geom *d_geom)
{
    tg_status st;
    double *rad;
    float *radf;
    if ((st = ensure_t(c, B_C_RAD, t.ncell, &rad)) || (st = ensure_t(c, B_C_RADF, t.ncell, &radf))) return st;
    const double *xs = static_cast<const double *>(c->buf[B_XS].p), *ys = static_cast<const double *>(c->buf[B_YS].p),
                 *zs = static_cast<const double *>(c->buf[B_ZS].p);
    {
        ProfScope ps_(c, TG_K_TREE);
        cell_radii_leaves<<<grid_for((int64_t)t.ncell * 32, 256), 256, 0, c->stream>>>(t, d_geom, xs, ys, zs, rad, radf);
    }
    const int nlev = (int)c->level_begin.size() - 1;
    for (int l = nlev - 2; l >= 0; --l) {
        const int lb = c->level_begin[l], le = c->level_begin[l + 1];
        ProfScope ps_(c, TG_K_TREE);
        cell_radii_level<<<grid_for(le - lb, 128), 128, 0, c->stream>>>(t, lb, le, d_geom, rad, radf);
    }
    t.rad = rad;
    t.radf = radf;
    return cuda_check(c, cudaGetLastError(), "cell radii");
}

__device__ __forceinline__ double to_double(float v) { return f2d_exact(v); }
__device__ __forceinline__ double to_double(double v) { return v; }

template <class T>
__device__ __forceinline__ T inv_fact_t(int k);
template <>
__device__ __forceinline__ float inv_fact_t<float>(int k) { return c_inv_fact_f[k]; }
template <>
__device__ __forceinline__ double inv_fact_t<double>(int k) { return c_inv_fact[k]; }

// ------------------------------------------------------------------ per-particle local data
// pf[s] = (x - z_leaf, y - z_leaf, z - z_leaf, m) in precision T; leaf_of[s] = leaf cell id.
template <class T4>
__global__ void leaf_particles(TreeView t, const Geom *gp, const double *xs, const double *ys, const double *zs,
                               const double *ms, T4 *pf, int32_t *leaf_of)
{
    const Geom g = *gp;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int ncell = t.cells();
    for (int c = warp; c < ncell; c += nwarps) {
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

// ------------------------------------------------------------------ slow-before-fast leaves
// With classes, every leaf's particles are stably reordered so the slow ones come first
// (nslow[leaf] of them).  Leaf ranges and the tree are unchanged; a mutual P2P tile can then skip
// the fast-fast block (kickS2F feels slow masses only) instead of masking it pair by pair.
__global__ void leaf_class_partition(TreeView t, const double *xs, const double *ys, const double *zs, const double *ms,
                                     const uint8_t *fs, const uint32_t *perm, double *xs2, double *ys2, double *zs2,
                                     double *ms2, uint8_t *fs2, uint32_t *perm2, int32_t *nslow)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int ncell = t.cells();
    for (int c = warp; c < ncell; c += nwarps) {
        if (t.nchild[c] != 0) continue;
        const int first = t.first[c], count = t.count[c];
        int ns = 0;
        for (int q0 = 0; q0 < count; q0 += 32) ns += __popc(__ballot_sync(0xffffffffu, q0 + lane < count && !fs[first + q0 + lane]));
        int slow_seen = 0, fast_seen = 0;
        for (int q0 = 0; q0 < count; q0 += 32) {
            const int q = q0 + lane;
            const bool valid = q < count;
            const bool slow = valid && !fs[first + q];
            const unsigned bs = __ballot_sync(0xffffffffu, slow), bf = __ballot_sync(0xffffffffu, valid && !slow);
            if (valid) {
                const int dst = first + (slow ? slow_seen + __popc(bs & lt) : ns + fast_seen + __popc(bf & lt));
                const int src = first + q;
                xs2[dst] = xs[src];
                ys2[dst] = ys[src];
                zs2[dst] = zs[src];
                ms2[dst] = ms[src];
                fs2[dst] = fs[src];
                perm2[dst] = perm[src];
            }
            slow_seen += __popc(bs);
            fast_seen += __popc(bf);
        }
        if (lane == 0) nslow[c] = ns;
    }
}

// ------------------------------------------------------------------ P2M
// Moments live in two arrays: M[cell][class][ncp] in precision T (every order) and
// M01[cell][class][4] in float64 (monopole and dipole, the "centre of mass" part, accumulated in
// float64 from float64 positions).  Offsets are in units of the cell side s.
template <class T, class T4>
__global__ void __launch_bounds__(128) p2m_leaves(TreeView t, const Geom *gp, const double *xs, const double *ys,
                                                  const double *zs, const double *ms, const uint8_t *fs, const T4 *pf,
                                                  int p, int nc, int ncp, T *M, double *M01)
{
    // per warp: powers r_a^e (axis a, 0 <= e <= p) of 32 particles, rows padded to 33 against bank
    // conflicts, and the particles' masses split by class
    __shared__ T s_pw[4][3][TG_PMAX + 1][33];
    __shared__ T s_w[4][2][32];
    __shared__ uint8_t s_e[3][168];
    for (int k = threadIdx.x; k < 168; k += blockDim.x) {
        s_e[0][k] = k < nc ? c_mi_x[k] : 0;
        s_e[1][k] = k < nc ? c_mi_y[k] : 0;
        s_e[2][k] = k < nc ? c_mi_z[k] : 0;
    }
    __syncthreads();
    const Geom g = *gp;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const int ncell = t.cells();
    for (int c = warp; c < ncell; c += nwarps) {
        if (t.nchild[c] != 0) continue;
        const int first = t.first[c], count = t.count[c];
        const double zx = cell_centre(g, t, c, 0), zy = cell_centre(g, t, c, 1), zz = cell_centre(g, t, c, 2);
        const double inv_s = ldexp(1.0, (int)t.level[c] - g.log2L);
        // float64 monopole and dipole: lanes over particles, then a warp reduction
        double lo[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
        for (int s = first + lane; s < first + count; s += 32) {
            const double m = ms[s];
            const bool fast = fs[s] != 0;
            const double r[4] = {1.0, (xs[s] - zx) * inv_s, (ys[s] - zy) * inv_s, (zs[s] - zz) * inv_s};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const double v = k ? m * r[k] : m;
                lo[0][k] += fast ? 0.0 : v;
                lo[1][k] += fast ? v : 0.0;
            }
        }
        // reduce-scatter of the 8 sums over the warp: after the stages over lane bits 4, 3, 2 lane l
        // holds entry (l >> 2) & 7 summed over its group of four lanes, then bits 1, 0 finish the sum
        double v8[8] = {lo[0][0], lo[0][1], lo[0][2], lo[0][3], lo[1][0], lo[1][1], lo[1][2], lo[1][3]};
#pragma unroll
        for (int h = 4, d = 16; h >= 1; h >>= 1, d >>= 1) {
            const bool hi = (lane & d) != 0;
#pragma unroll
            for (int q = 0; q < h; ++q) {
                const double send = hi ? v8[q] : v8[q + h];
                const double keep = hi ? v8[q + h] : v8[q];
                v8[q] = keep + __shfl_xor_sync(0xffffffffu, send, d);
            }
        }
        double mine = v8[0];
        mine += __shfl_xor_sync(0xffffffffu, mine, 2);
        mine += __shfl_xor_sync(0xffffffffu, mine, 1);
        // entry e = cls * 4 + k sits in lanes 4e .. 4e + 3; move it to lane e
        mine = __shfl_sync(0xffffffffu, mine, 4 * (lane & 7));
        if (lane < 8) {
            const int cls = lane >> 2, k = lane & 3;
            M01[((size_t)c * 2 + cls) * 4 + k] = mine;
            M[((size_t)c * 2 + cls) * ncp + k] = (T)mine;
        }
        // orders >= 2 in T from the per-particle offsets: lanes over coefficients k = 4 + lane + 32 q
        const T inv_st = (T)ldexpf(1.0f, (int)t.level[c] - g.log2L);
        T accS[(168 - 4 + 31) / 32], accF[(168 - 4 + 31) / 32];
#pragma unroll
        for (int q = 0; q < (168 - 4 + 31) / 32; ++q) accS[q] = accF[q] = T(0);
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
#pragma unroll
            for (int q = 0; q < (168 - 4 + 31) / 32; ++q) {
                const int k = 4 + lane + 32 * q;
                if (4 + 32 * q < nc && k < nc) {
                    const int ex = s_e[0][k], ey = s_e[1][k], ez = s_e[2][k];
                    T aS = 0, aF = 0;
                    for (int i = 0; i < m; ++i) {
                        const T v = s_pw[wib][0][ex][i] * s_pw[wib][1][ey][i] * s_pw[wib][2][ez][i];
                        aS += s_w[wib][0][i] * v;
                        aF += s_w[wib][1][i] * v;
                    }
                    accS[q] += aS;
                    accF[q] += aF;
                }
            }
        }
#pragma unroll
        for (int q = 0; q < (168 - 4 + 31) / 32; ++q) {
            const int k = 4 + lane + 32 * q;
            if (k < ncp) {
                M[((size_t)c * 2 + 0) * ncp + k] = k < nc ? accS[q] : T(0);
                M[((size_t)c * 2 + 1) * ncp + k] = k < nc ? accF[q] : T(0);
            }
        }
    }
}

// coefficient i of a generated translation list in the precision of the expansions
template <class T>
__device__ __forceinline__ T trans_coef(const float *cf, const double *cd, int i);
template <>
__device__ __forceinline__ float trans_coef<float>(const float *cf, const double *, int i)
{
    return cf[i];
}
template <>
__device__ __forceinline__ double trans_coef<double>(const float *, const double *cd, int i)
{
    return cd[i];
}

// M2M for the parents of one level, normalised: with d = z_child - z_parent = (+-s/4)^3 and
// s_child = s/2,  M~_P^n = sum_children sum_{k <= n} C(n,k) 2^-(2|n-k| + |k|) (+-1)^(n-k) M~_c^k.
// Block per parent cell.  |n| <= 1 in float64 (M01, threads 0..7), every order also in T (M).
// Orders >= 2: lane (n, q) with q = lane % 8 sums the terms k <= n (componentwise) of child q,
// then the eight children are added with three shuffles.  The children's moments are staged in
// shared memory; the terms of each n (coefficient index, parity of n - k, coefficient) come from the
// generated lists g_m2m_* in the order of the sum, k_x outermost.
constexpr int kM2MThreads = 256;

template <class T>
__global__ void __launch_bounds__(kM2MThreads) m2m_level(TreeView t, int lb, int le, int p, int nc, int ncp, T *M,
                                                         double *M01, const DevEval *de, int lvl)
{
    if (de) {   // level range on the device (batched path); levels past the tree are empty
        if (lvl + 1 >= de->nlev) return;
        lb = de->level_begin[lvl];
        le = de->level_begin[lvl + 1];
    }
    extern __shared__ __align__(16) unsigned char m2m_smem[];
    T *s_mc = reinterpret_cast<T *>(m2m_smem);   // [8 children][2 classes][ncp]
    const int lane = threadIdx.x & 31, q = lane & 7;
    const int sub = threadIdx.x >> 3;   // 0 .. blockDim/8 - 1: which n of the pass
    const int per_pass = blockDim.x >> 3;
    for (int c = lb + blockIdx.x; c < le; c += gridDim.x) {
        const int nch = t.nchild[c];   // uniform over the block
        if (nch == 0) continue;
        const int cf = t.child_first[c];
        __syncthreads();   // tables ready / previous parent done with s_mc
        {
            const int tot = nch * 2 * ncp;
            const T *src = M + (size_t)cf * 2 * ncp;
            for (int k = threadIdx.x; k < tot; k += blockDim.x) s_mc[k] = src[k];
        }
        __syncthreads();
        if (threadIdx.x < 8) {
            const int cls = threadIdx.x >> 2, n = threadIdx.x & 3;
            double acc = 0.0;
            for (int qq = 0; qq < nch; ++qq) {
                const double *Mc = M01 + ((size_t)(cf + qq) * 2 + cls) * 4;
                double v = Mc[n];
                if (n > 0) {
                    const uint32_t cc = n == 1 ? t.cx[cf + qq] : (n == 2 ? t.cy[cf + qq] : t.cz[cf + qq]);
                    v = 0.5 * v + ((cc & 1u) ? 0.25 : -0.25) * Mc[0];
                }
                acc += v;
            }
            M01[((size_t)c * 2 + cls) * 4 + n] = acc;
            M[((size_t)c * 2 + cls) * ncp + n] = (T)acc;
        }
        // this lane's child: offsets toward the negative side flip the sign of odd powers (bit a of negm)
        unsigned negm = 0u;
        if (q < nch)
            negm = (t.cx[cf + q] & 1u ? 0u : 1u) | (t.cy[cf + q] & 1u ? 0u : 2u) | (t.cz[cf + q] & 1u ? 0u : 4u);
        const T *MS = s_mc + q * 2 * ncp, *MF = MS + ncp;
        for (int n0 = 4; n0 < ncp; n0 += per_pass) {
            const int n = n0 + sub;
            T sS = 0, sF = 0;
            if (n < nc && q < nch) {
                // the terms k <= n from the generated list: coefficient index, parity of n - k, coefficient
                const int i1 = g_m2m_off[n + 1];
                for (int i = g_m2m_off[n]; i < i1; ++i) {
                    const unsigned kp = g_m2m_kp[i];
                    const int k = (int)(kp & 0xffu);
                    T coef = trans_coef<T>(g_m2m_cf, g_m2m_cd, i);
                    coef = (__popc((kp >> 8) & negm) & 1) ? -coef : coef;
                    sS += coef * MS[k];
                    sF += coef * MF[k];
                }
            }
            // sum over the eight children (lanes q = 0..7 of this n)
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                sS += __shfl_xor_sync(0xffffffffu, sS, o);
                sF += __shfl_xor_sync(0xffffffffu, sF, o);
            }
            if (q == 0 && n < ncp) {
                M[((size_t)c * 2 + 0) * ncp + n] = n < nc ? sS : T(0);
                M[((size_t)c * 2 + 1) * ncp + n] = n < nc ? sF : T(0);
            }
        }
    }
}

// M2L operands: Ms[c][0] = (M~_S + M~_F)/j!, Ms[c][1] = M~_S/j! in precision T (padding zero);
// the monopole and dipole come from the float64 sums.
// 1/(kx! ky! kz!) for a multi-index past the tables (orders above TG_PMAX)
__device__ double inv_fact_beyond_tables(int k)
{
    int o = 0;
    while ((o + 1) * (o + 2) * (o + 3) / 6 <= k) ++o;
    int r = k - o * (o + 1) * (o + 2) / 6, a = 0;
    while ((a + 1) * (a + 2) / 2 <= r) ++a;
    const int kz = r - a * (a + 1) / 2, kx = o - a, ky = a - kz;
    double f = 1.0;
    for (int i = 2; i <= kx; ++i) f *= i;
    for (int i = 2; i <= ky; ++i) f *= i;
    for (int i = 2; i <= kz; ++i) f *= i;
    return 1.0 / f;
}

template <class T>
__global__ void scale_moments(int ncell, int nc, int ncp, const T *M, const double *M01, T *Ms, const int *dncell)
{
    ncell = dev_or(dncell, ncell);
    const int64_t total = (int64_t)ncell * ncp;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = w / ncp;
        const int k = (int)(w % ncp);
        if (k < 4) {
            const double mS = M01[(c * 2 + 0) * 4 + k], mF = M01[(c * 2 + 1) * 4 + k];
            const double f = c_inv_fact[k];
            Ms[(c * 2 + 0) * ncp + k] = (T)((mS + mF) * f);
            Ms[(c * 2 + 1) * ncp + k] = (T)(mS * f);
        } else {
            const T mS = M[(c * 2 + 0) * ncp + k], mF = M[(c * 2 + 1) * ncp + k];
            const T f = k < nc ? (k < TG_NCOEF_MAX ? inv_fact_t<T>(k) : (T)inv_fact_beyond_tables(k)) : T(0);
            Ms[(c * 2 + 0) * ncp + k] = (mS + mF) * f;
            Ms[(c * 2 + 1) * ncp + k] = mS * f;
        }
    }
}

// ------------------------------------------------------------------ dual tree walk
// Breadth-first Algorithm 4 over UNORDERED pairs.  The frontier holds pairs (A, B) that are not
// well separated and not both leaves, i.e. pairs to open: both cells when both have children
// (the paper's "open both" rule), otherwise the non-leaf one; a self pair (A, A) opens A and
// yields the child pairs ci <= cj.  Each child pair (x, y) is classified at once:
//   x == y           -> P2P(x, x) if x is a leaf, else frontier
//   well separated   -> bit (i, j) of this pair's M2L block
//   both leaves      -> P2P(x, y)
//   otherwise        -> frontier
struct WalkOut {
    uint2 *front_out;
    M2LBlock *blocks;
    uint2 *p2p;
    unsigned long long *counters;   // [1] M2L blocks, [2] P2P pairs A != B, [3] M2L pairs,
                                    // [4] self P2P pairs (A, A), stored from the end of the P2P buffer
    unsigned long long *front_ctr;  // length of front_out
    unsigned long long cap_front, cap_blocks, cap_p2p;
};

// Warp-aggregated slot reservation on a shared counter: one atomic per warp, each lane gets its
// own base.  Every lane of the warp must call it (lanes with nothing to add pass 0).
__device__ __forceinline__ unsigned long long warp_reserve(unsigned long long *ctr, unsigned cnt)
{
    const int lane = threadIdx.x & 31;
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(ctr, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + (incl - cnt);
}

// One step of the dual walk.  The input length is read on the device (it is the previous step's
// output counter), so that all steps can be queued without waiting for the host.
__device__ __forceinline__ void walk_step_body(const TreeView &t, const MacParams &mp, const uint2 *front_in,
                                               const unsigned long long *n_in_ctr, const WalkOut &o)
{
    const unsigned long long n_in_raw = *n_in_ctr;
    const int64_t n_in = (int64_t)(n_in_raw < o.cap_front ? n_in_raw : o.cap_front);
    // whole warps iterate together so that the counters can be reserved per warp
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x; w0 < n_in; w0 += stride) {
        const int64_t w = w0 + threadIdx.x;
        const bool active = w < n_in;
        int A = 0, B = 0, ni = 0, nj = 0, baseA = 0, baseB = 0;
        bool self = false;
        // classes of the child pairs, bit 8i + j: well separated (M2L), P2P, self P2P, frontier
        unsigned long long mask = 0, mp2p = 0, mself = 0, mfront = 0;
        if (active) {
            const uint2 pr = front_in[w];
            A = (int)pr.x;
            B = (int)pr.y;
            self = A == B;
            const bool openA = t.nchild[A] != 0, openB = t.nchild[B] != 0;
            ni = openA ? t.nchild[A] : 1;
            nj = openB ? t.nchild[B] : 1;
            baseA = openA ? t.child_first[A] : A;
            baseB = openB ? t.child_first[B] : B;
            // the column cells' geometry, loaded once (independent loads, issued together)
            CellGeo gy[8];
            bool ly[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int y = baseB + (j < nj ? j : 0);
                gy[j] = CellGeo{t.cx[y], t.cy[y], t.cz[y], (int)t.level[y]};
                ly[j] = t.nchild[y] == 0;
            }
            // classify every child pair once
            for (int i = 0; i < ni; ++i) {
                const int x = baseA + i;
                const CellGeo gx{t.cx[x], t.cy[x], t.cz[x], (int)t.level[x]};
                const bool lx = t.nchild[x] == 0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (j >= nj || (self && j < i)) continue;
                    const int y = baseB + j;
                    const unsigned long long bit = 1ull << (8 * i + j);
                    if (x == y) {
                        if (lx) mself |= bit;
                        else mfront |= bit;
                    } else if (well_separated_geo(t, mp, x, gx, y, gy[j])) {
                        mask |= bit;
                    } else if (lx && ly[j]) {
                        mp2p |= bit;
                    } else {
                        mfront |= bit;
                    }
                }
            }
        }
        unsigned long long fb = warp_reserve(o.front_ctr, (unsigned)__popcll(mfront));
        unsigned long long pb = warp_reserve(o.counters + 2, (unsigned)__popcll(mp2p));
        unsigned long long sb = warp_reserve(o.counters + 4, (unsigned)__popcll(mself));
        const unsigned long long bb = warp_reserve(o.counters + 1, mask ? 1u : 0u);
        warp_reserve(o.counters + 3, (unsigned)__popcll(mask));
        if (!active) continue;
        if (mask && bb < o.cap_blocks) o.blocks[bb] = M2LBlock{(uint32_t)A, (uint32_t)B, mask};
        // write the entries of each class from its bits (lowest bit first, the order of the loops above)
        for (unsigned long long m = mself; m; m &= m - 1) {
            const int b = __ffsll((long long)m) - 1, x = baseA + (b >> 3);
            if (sb < o.cap_p2p) o.p2p[o.cap_p2p - 1 - sb] = make_uint2(x, x);
            ++sb;
        }
        for (unsigned long long m = mp2p; m; m &= m - 1) {
            const int b = __ffsll((long long)m) - 1;
            if (pb < o.cap_p2p) o.p2p[pb] = make_uint2(baseA + (b >> 3), baseB + (b & 7));
            ++pb;
        }
        for (unsigned long long m = mfront; m; m &= m - 1) {
            const int b = __ffsll((long long)m) - 1;
            if (fb < o.cap_front) o.front_out[fb] = make_uint2(baseA + (b >> 3), baseB + (b & 7));
            ++fb;
        }
    }
}

__global__ void walk_step(TreeView t, MacParams mp, const uint2 *front_in, const unsigned long long *n_in_ctr, WalkOut o)
{
    walk_step_body(t, mp, front_in, n_in_ctr, o);
}

// The same step with the criterion's thresholds in device memory (batched path), staged in shared memory.
__global__ void walk_step_dev(TreeView t, const MacParams *__restrict__ mpp, const uint2 *front_in,
                              const unsigned long long *n_in_ctr, WalkOut o)
{
    static_assert(sizeof(MacParams) % 4 == 0, "MacParams is copied as 32-bit words");
    __shared__ MacParams smp;
    for (int i = threadIdx.x; i < (int)(sizeof(MacParams) / 4); i += blockDim.x)
        reinterpret_cast<int *>(&smp)[i] = reinterpret_cast<const int *>(mpp)[i];
    __syncthreads();
    walk_step_body(t, smp, front_in, n_in_ctr, o);
}

// Gap thresholds of Eq. (1)'s eps rule for the root cube of this evaluation, on the device: the same
// integer searches in float64 as make_mac_params on the host, so the decisions are identical.
__global__ void mac_params_dev(const Geom *g, double eps, MacParams *mp)
{
    const int lf = threadIdx.x;
    const int log2L = g->log2L;
    if (lf <= kMaxLevel) {
        const double eu = ldexp(eps, lf + 1 - log2L);
        const double E = eu * eu;
        long long r = 0;
        if (!(0.0 > E)) {
            long long lo = 0, hi = 1ll << 62;
            while (hi - lo > 1) {
                const long long mid = lo + (hi - lo) / 2;
                if ((double)mid > E) hi = mid;
                else lo = mid;
            }
            r = hi;
        }
        mp->gap_min_g2[lf] = r;
    }
    if (lf == 0) mp->log2L = log2L;
}

// ------------------------------------------------------------------ L2L (one level), normalised
// L~_c^n += sum_{d} L~_P^(n+d) (+-1)^d 2^-(2|d| + |n| + 1) / d!  over |d| <= p - |n|.
// Warp per cell of the level, lanes over the coefficients n >= n_first (1 when only accelerations are
// wanted: L^0 feeds no force), both classes.  d runs through the
// multi-indices in their table order; the index of n + d, the parity of d and the coefficient come
// from the generated list g_l2l_* of n (built for order 8: order p takes its first terms).
constexpr int kM2MWarps = 2;   // warps per block of the L2L level kernel

template <class T>
__global__ void __launch_bounds__(32 * kM2MWarps) l2l_level(TreeView t, int lb, int le, int p, int nc, int ncp, int ncls,
                                                            int n_first, T *L, const DevEval *de, int lvl)
{
    if (de) {   // level range and classes on the device (batched path)
        if (lvl >= de->nlev) return;
        lb = de->level_begin[lvl];
        le = de->level_begin[lvl + 1];
        ncls = de->masked ? 2 : 1;
    }
    extern __shared__ __align__(16) unsigned char l2l_smem[];
    T *s_lp = reinterpret_cast<T *>(l2l_smem) + (size_t)(threadIdx.x >> 5) * 2 * ncp;   // parent's L, this warp
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int c = lb + warp; c < le; c += nwarps) {
        const int par = t.parent[c];
        if (par < 0) continue;
        // offsets toward the negative side flip the sign of odd powers (bit a of negm)
        const unsigned negm = (t.cx[c] & 1u ? 0u : 1u) | (t.cy[c] & 1u ? 0u : 2u) | (t.cz[c] & 1u ? 0u : 4u);
        __syncwarp();
#pragma unroll 4
        for (int k = lane; k < ncls * ncp; k += 32) s_lp[k] = L[(size_t)par * 2 * ncp + k];
        __syncwarp();
        const T *Lp = s_lp;
        for (int n = n_first + lane; n < nc; n += 32) {
            // the terms d with |d| <= p - |n|: the first ones of n's generated list (built for order 8)
            const int nd = ncoef_dev(p - (int)c_mi_order[n]);
            const int i0 = g_l2l_off[n];
            T acc0 = 0, acc1 = 0;
            for (int d = 0; d < nd; ++d) {
                const unsigned kp = g_l2l_kp[i0 + d];
                const int k = (int)(kp & 0xffu);
                const T coef = trans_coef<T>(g_l2l_cf, g_l2l_cd, i0 + d);
                const T cs = (__popc((kp >> 8) & negm) & 1) ? -coef : coef;
                acc0 += Lp[k] * cs;
                if (ncls > 1) acc1 += Lp[ncp + k] * cs;
            }
            L[((size_t)c * 2 + 0) * ncp + n] += acc0;
            if (ncls > 1) L[((size_t)c * 2 + 1) * ncp + n] += acc1;
        }
    }
}

// Multi-index k -> (kx, ky, kz) in the table order (total degree, then kx descending, then ky
// descending), as constexpr functions: inside fully unrolled loops every index folds to a constant.
struct MI3 {
    int x, y, z;
};
__host__ __device__ constexpr MI3 mi3(int k)
{
    int o = 0;
    while ((o + 1) * (o + 2) * (o + 3) / 6 <= k) ++o;
    int r = k - o * (o + 1) * (o + 2) / 6;
    for (int nx = o; nx >= 0; --nx) {
        const int len = o - nx + 1;   // ny = o - nx .. 0
        if (r < len) return MI3{nx, o - nx - r, r};
        r -= len;
    }
    return MI3{0, 0, 0};
}
__host__ __device__ constexpr int mi3_index(int x, int y, int z)
{
    const int o = x + y + z;
    int k = o * (o + 1) * (o + 2) / 6;
    for (int nx = o; nx > x; --nx) k += o - nx + 1;
    return k + (o - x - y);
}
__host__ __device__ constexpr int fact_i(int n)
{
    int f = 1;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// L2P at a fixed order P: monomials, coefficients and indices are compile-time after unrolling.
// POT = false: accelerations only (the potential slot is written as zero).
template <int P, class T, class T4, bool POT>
__global__ void l2p_fixed(int n, TreeView t, const Geom *__restrict__ gp, const T4 *__restrict__ pf,
                          const int32_t *__restrict__ leaf_of, const uint8_t *__restrict__ fs, int masked, int ncp,
                          const T *__restrict__ L, double *acc4, int stride, const DevEval *de)
{
    constexpr int NC = (P + 1) * (P + 2) * (P + 3) / 6;
    if (de) {
        n = de->n;
        masked = de->masked;
    }
    const int log2L = gp->log2L;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const T4 r = pf[s];
        const int c = leaf_of[s];
        const int cls = (masked && fs[s]) ? 1 : 0;
        const T *__restrict__ Lc = L + ((size_t)c * 2 + cls) * ncp;
        const T inv_s = (T)ldexpf(1.0f, (int)t.level[c] - log2L);
        const T rx = r.x * inv_s, ry = r.y * inv_s, rz = r.z * inv_s;
        T px[P + 1], py[P + 1], pz[P + 1];
        px[0] = py[0] = pz[0] = (T)1;
#pragma unroll
        for (int e = 1; e <= P; ++e) {
            px[e] = px[e - 1] * rx;
            py[e] = py[e - 1] * ry;
            pz[e] = pz[e - 1] * rz;
        }
        T Lk[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) Lk[k] = Lc[k];
        T phi = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const MI3 m = mi3(k);
            const T mono = px[m.x] * py[m.y] * pz[m.z] * (T(1) / (T)(fact_i(m.x) * fact_i(m.y) * fact_i(m.z)));
            if (POT) phi += Lk[k] * mono;
            if (m.x + m.y + m.z < P) {
                gx += Lk[mi3_index(m.x + 1, m.y, m.z)] * mono;
                gy += Lk[mi3_index(m.x, m.y + 1, m.z)] * mono;
                gz += Lk[mi3_index(m.x, m.y, m.z + 1)] * mono;
            }
        }
        const T is2 = inv_s * inv_s;
        acc4[s] = to_double(-gx * is2);
        acc4[(size_t)stride + s] = to_double(-gy * is2);
        acc4[2 * (size_t)stride + s] = to_double(-gz * is2);
        acc4[3 * (size_t)stride + s] = to_double(phi * inv_s);
    }
}

// ------------------------------------------------------------------ L2P, normalised
// With r = (x - z)/s:  phi = (1/s) sum_n L~^n r^n/n!,  a_e = -(1/s^2) sum_m L~^{m+e} r^m/m!.
// Thread per particle; writes acc4 (= initialises it).
template <class T, class T4>
__global__ void l2p_particles(int n, TreeView t, int log2L, const T4 *pf, const int32_t *leaf_of, const uint8_t *fs,
                              int masked, int p, int nc, int ncp, const T *L, double *acc4)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const T4 r = pf[s];
        const int c = leaf_of[s];
        const int cls = (masked && fs[s]) ? 1 : 0;
        const T *Lc = L + ((size_t)c * 2 + cls) * ncp;
        const T inv_s = (T)ldexpf(1.0f, (int)t.level[c] - log2L);
        const T rx = r.x * inv_s, ry = r.y * inv_s, rz = r.z * inv_s;
        T px[TG_PMAX + 1], py[TG_PMAX + 1], pz[TG_PMAX + 1];
        px[0] = py[0] = pz[0] = (T)1;
        for (int e = 1; e <= p; ++e) {
            px[e] = px[e - 1] * rx;
            py[e] = py[e - 1] * ry;
            pz[e] = pz[e - 1] * rz;
        }
        T phi = 0, gx = 0, gy = 0, gz = 0;
        for (int k = 0; k < nc; ++k) {
            const int kx = c_mi_x[k], ky = c_mi_y[k], kz = c_mi_z[k];
            const T mono = px[kx] * py[ky] * pz[kz] * inv_fact_t<T>(k);
            phi += Lc[k] * mono;
            if (kx + ky + kz < p) {
                gx += Lc[c_mi_lookup[((kx + 1) * 9 + ky) * 9 + kz]] * mono;
                gy += Lc[c_mi_lookup[(kx * 9 + ky + 1) * 9 + kz]] * mono;
                gz += Lc[c_mi_lookup[(kx * 9 + ky) * 9 + kz + 1]] * mono;
            }
        }
        const T is2 = inv_s * inv_s;
        acc4[s] = to_double(-gx * is2);
        acc4[(size_t)n + s] = to_double(-gy * is2);
        acc4[2 * (size_t)n + s] = to_double(-gz * is2);
        acc4[3 * (size_t)n + s] = to_double(phi * inv_s);
    }
}

// ------------------------------------------------------------------ scatter back to input order
// acc4 holds four arrays of length stride4 (the evaluation's n in the plain path)
__global__ void scatter_out(int n, const uint32_t *perm, const double *acc4, double *acc, int64_t stride, double *pot,
                            const int *dn, int64_t stride4, const double *acc4b = nullptr)
{
    n = dev_or(dn, n);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const uint32_t q = perm[s];
        // acc4b (nullable): the P2P sums kept apart when P2P ran beside the far field (accelerations only)
        acc[q] = acc4b ? acc4[s] + acc4b[s] : acc4[s];
        acc[stride + q] = acc4b ? acc4[(size_t)stride4 + s] + acc4b[(size_t)stride4 + s] : acc4[(size_t)stride4 + s];
        acc[2 * stride + q] =
            acc4b ? acc4[2 * (size_t)stride4 + s] + acc4b[2 * (size_t)stride4 + s] : acc4[2 * (size_t)stride4 + s];
        if (pot) pot[q] = acc4[3 * (size_t)stride4 + s];
    }
}

// zero the three acceleration rows of an acc4 array for the first dn[0] particles
__global__ void zero_acc3(double *acc4, int64_t stride4, const int *dn)
{
    const int n = dn[0];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        acc4[s] = 0.0;
        acc4[(size_t)stride4 + s] = 0.0;
        acc4[2 * (size_t)stride4 + s] = 0.0;
    }
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
__global__ void walk_init(uint2 *front, unsigned long long *front_ctr)
{
    front[0] = make_uint2(0, 0);
    front_ctr[0] = 1;
}

constexpr int kWalkMaxSteps = 24;   // a step descends one level; the octree has at most 22 levels

static tg_status run_walk(tg_ctx *c, const TreeView &t, int64_t *n_blocks, int64_t *n_m2l, int64_t *n_p2p,
                          int64_t *n_self)
{
    tg_status st;
    int log2L = 0;
    {
        const Geom *dg = static_cast<const Geom *>(c->buf[B_GEOM].p);
        cudaMemcpyAsync(c->h_pinned + 32, &dg->log2L, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        cudaError_t e = stream_sync(c);
        if (e != cudaSuccess) return cuda_check(c, e, "walk setup");
        log2L = *reinterpret_cast<int *>(c->h_pinned + 32);
    }
    const MacParams mp = make_mac_params(c->prm, log2L);
    c->walk_log2L = log2L;
    // capacities from the largest list sizes per cell seen so far (plus a margin), so that a walk is
    // normally run once
    size_t cap_front = (size_t)(t.ncell * c->walk_front_per_cell * 1.25) + 1024,
           cap_blocks = (size_t)(t.ncell * c->walk_blocks_per_cell * 1.25) + 1024,
           cap_p2p = (size_t)(t.ncell * c->walk_p2p_per_cell * 1.25) + 1024;
    for (int attempt = 0; attempt < 6; ++attempt) {
        uint2 *f0, *f1, *p2p;
        M2LBlock *blocks;
        unsigned long long *ctr;
        if ((st = ensure_t(c, B_FRONT0, cap_front, &f0)) || (st = ensure_t(c, B_FRONT1, cap_front, &f1)) ||
            (st = ensure_t(c, B_M2L, cap_blocks, &blocks)) || (st = ensure_t(c, B_P2P, cap_p2p, &p2p)) ||
            (st = ensure_t(c, B_WALK_CNT, 8 + kWalkMaxSteps + 1, &ctr)))
            return st;
        unsigned long long *front_ctr = ctr + 8;   // front_ctr[s]: input length of step s
        cudaMemsetAsync(ctr, 0, (8 + kWalkMaxSteps + 1) * sizeof(unsigned long long), c->stream);
        unsigned long long tot_blocks = 0, tot_p2p = 0, tot_pairs = 0, tot_self = 0;
        c->p2p_cap = (int64_t)cap_p2p;
        if (t.ncell == 1) {
            // the root is a leaf: one self P2P pair
            const uint2 root = make_uint2(0, 0);
            cudaMemcpyAsync(p2p + cap_p2p - 1, &root, sizeof(uint2), cudaMemcpyHostToDevice, c->stream);
            *n_blocks = 0;
            *n_m2l = 0;
            *n_p2p = 0;
            *n_self = 1;
            return cuda_check(c, stream_sync(c), "walk");
        }
        {
            ProfScope ps_(c, TG_K_WALK);
            walk_init<<<1, 1, 0, c->stream>>>(f0, front_ctr);
        }
        // every frontier pair holds a cell with children, at the level of the step: the walk ends
        // after at most (levels - 1) steps; all of them are queued, then the counters read once
        const int nsteps = std::min<int>(kWalkMaxSteps, std::max<int>(1, (int)c->level_begin.size() - 1));
        const int grid = c->num_sms * 4;
        for (int s = 0; s < nsteps; ++s) {
            WalkOut o{(s & 1) ? f0 : f1, blocks, p2p, ctr, front_ctr + s + 1, cap_front, cap_blocks, cap_p2p};
            ProfScope ps_(c, TG_K_WALK);
            walk_step<<<grid, 128, 0, c->stream>>>(t, mp, (s & 1) ? f1 : f0, front_ctr + s, o);
        }
        cudaMemcpyAsync(c->h_pinned, ctr, (8 + nsteps + 1) * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        c->stream);
        cudaError_t e = stream_sync(c);
        if (e != cudaSuccess) return cuda_check(c, e, "walk");
        const unsigned long long *h = reinterpret_cast<const unsigned long long *>(c->h_pinned);
        tot_blocks = h[1];
        tot_p2p = h[2];
        tot_pairs = h[3];
        tot_self = h[4];
        size_t need_front = 0;
        for (int s = 1; s <= nsteps; ++s) need_front = std::max<size_t>(need_front, h[8 + s]);
        if (h[8 + nsteps] != 0) return set_err(c, TG_ERR_CAPACITY, "walk frontier not empty after %d steps", nsteps);
        const bool overflow = need_front > cap_front || tot_blocks > cap_blocks || tot_p2p + tot_self > cap_p2p;
        const double nc = (double)t.ncell;
        c->walk_front_per_cell = std::max(c->walk_front_per_cell, need_front / nc);
        c->walk_blocks_per_cell = std::max(c->walk_blocks_per_cell, tot_blocks / nc);
        c->walk_p2p_per_cell = std::max(c->walk_p2p_per_cell, (tot_p2p + tot_self) / nc);
        if (!overflow) {
            *n_blocks = (int64_t)tot_blocks;
            *n_m2l = (int64_t)tot_pairs;
            *n_p2p = (int64_t)tot_p2p;
            *n_self = (int64_t)tot_self;
            return TG_OK;
        }
        c->stats.list_regrowths += 1;
        cap_front = std::max(cap_front * 2, need_front + need_front / 2);
        cap_blocks = tot_blocks > cap_blocks ? tot_blocks * 2 : cap_blocks * 3 / 2;
        cap_p2p = tot_p2p + tot_self > cap_p2p ? (tot_p2p + tot_self) * 2 : cap_p2p * 3 / 2;
    }
    return set_err(c, TG_ERR_CAPACITY, "interaction lists did not fit after regrowth");
}

static inline int pad4(int x) { return (x + 3) & ~3; }

// precision dispatch of the M2L and P2P launchers (m2l.cu, p2p.cu)
static tg_status launch_m2l_t(tg_ctx *c, const TreeView &t, const M2LBlock *blocks, int64_t nblocks, const float *Ms,
                              float *L, int p, int nc, int ncp, bool masked, bool pot, const uint32_t *fpre)
{
    return launch_m2l_f32(c, t, blocks, nblocks, Ms, L, p, nc, ncp, masked, pot, fpre);
}
static tg_status launch_m2l_t(tg_ctx *c, const TreeView &t, const M2LBlock *blocks, int64_t nblocks, const double *Ms,
                              double *L, int p, int nc, int ncp, bool masked, bool pot, const uint32_t *fpre)
{
    (void)fpre;   // the float64 contraction computes both classes for every pair
    (void)pot;   // the float64 contraction always includes the potential term
    return launch_m2l_f64(c, t, blocks, nblocks, Ms, L, p, nc, ncp, masked);
}
static tg_status launch_p2p_t(tg_ctx *c, const TreeView &t, const Geom *d_geom, const uint2 *pairs, int64_t npairs,
                              const uint2 *self_pairs, int64_t nself, const float4 *pf, const uint8_t *fs,
                              const int32_t *nslow, bool masked, bool pot, double *acc4)
{
    (void)d_geom;
    (void)fs;
    (void)masked;   // classes arrive as slow-first leaves (nslow)
    return launch_p2p_f32(c, t, pairs, npairs, self_pairs, nself, pf, nslow, pot, acc4);
}
static tg_status launch_p2p_t(tg_ctx *c, const TreeView &t, const Geom *d_geom, const uint2 *pairs, int64_t npairs,
                              const uint2 *self_pairs, int64_t nself, const dbl4 *pf, const uint8_t *fs,
                              const int32_t *nslow, bool masked, bool pot, double *acc4)
{
    (void)nslow;   // the float64 tiles mask fast-fast pairs one by one
    (void)pot;     // and always include the potential
    return launch_p2p_f64(c, t, d_geom, pairs, npairs, self_pairs, nself, pf, fs, masked, acc4);
}

template <class T, class T4>
static tg_status eval_typed(tg_ctx *c, int n, int ncell, const TreeView &t, const Geom *d_geom, bool masked, bool want_pot,
                            int64_t n_blocks, int64_t n_p2p, int64_t n_self)
{
    tg_status st;
    const int p = c->prm.p, nc = ncoef(p), ncp = pad4(nc);
    const double *xs = static_cast<const double *>(c->buf[B_XS].p), *ys = static_cast<const double *>(c->buf[B_YS].p),
                 *zs = static_cast<const double *>(c->buf[B_ZS].p), *ms = static_cast<const double *>(c->buf[B_MS].p);
    const uint8_t *fs = static_cast<const uint8_t *>(c->buf[B_FS].p);
    T4 *pf;
    int32_t *leaf_of;
    double *M01, *acc4;
    T *M, *L, *Ms;
    if ((st = ensure_t(c, B_PF, n, &pf)) || (st = ensure_t(c, B_LEAF_OF, n, &leaf_of)) ||
        (st = ensure_t(c, B_MOM, (size_t)ncell * 2 * ncp, &M)) || (st = ensure_t(c, B_MOMF, (size_t)ncell * 2 * ncp, &Ms)) ||
        (st = ensure_t(c, B_MOM01, (size_t)ncell * 2 * 4, &M01)) ||
        (st = ensure_t(c, B_LOC, (size_t)ncell * 2 * ncp, &L)) || (st = ensure_t(c, B_ACC, (size_t)4 * n, &acc4)))
        return st;
    const int ncls = masked ? 2 : 1;
    int32_t *nslow = nullptr;
    if (masked) {
        double *xs2, *ys2, *zs2, *ms2;
        uint8_t *fs2;
        uint32_t *perm2;
        if ((st = ensure_t(c, B_XS2, n, &xs2)) || (st = ensure_t(c, B_YS2, n, &ys2)) || (st = ensure_t(c, B_ZS2, n, &zs2)) ||
            (st = ensure_t(c, B_MS2, n, &ms2)) || (st = ensure_t(c, B_FS2, n, &fs2)) ||
            (st = ensure_t(c, B_PERM2, n, &perm2)) || (st = ensure_t(c, B_NSLOW, ncell, &nslow)))
            return st;
        {
            ProfScope ps_(c, TG_K_TREE);
            leaf_class_partition<<<grid_for((int64_t)ncell * 32, 256), 256, 0, c->stream>>>(
                t, xs, ys, zs, ms, fs, static_cast<const uint32_t *>(c->buf[B_VALS0].p), xs2, ys2, zs2, ms2, fs2, perm2, nslow);
        }
        std::swap(c->buf[B_XS], c->buf[B_XS2]);
        std::swap(c->buf[B_YS], c->buf[B_YS2]);
        std::swap(c->buf[B_ZS], c->buf[B_ZS2]);
        std::swap(c->buf[B_MS], c->buf[B_MS2]);
        std::swap(c->buf[B_FS], c->buf[B_FS2]);
        std::swap(c->buf[B_VALS0], c->buf[B_PERM2]);
        xs = xs2;
        ys = ys2;
        zs = zs2;
        ms = ms2;
        fs = fs2;
    }
    {
        ProfScope ps_(c, TG_K_UP);
        leaf_particles<T4><<<grid_for((int64_t)ncell * 32, 256), 256, 0, c->stream>>>(t, d_geom, xs, ys, zs, ms, pf, leaf_of);
    }
    const bool high = p > TG_PMAX;   // orders past the tables: high_order.cu
    if (high) {
        if ((st = launch_p2m_hi<T, T4>(c, t, d_geom, xs, ys, zs, ms, fs, pf, p, nc, ncp, M, M01))) return st;
    } else {
        ProfScope ps_(c, TG_K_UP);
        p2m_leaves<T, T4><<<grid_for((int64_t)ncell * 32, 128), 128, 0, c->stream>>>(t, d_geom, xs, ys, zs, ms, fs, pf, p, nc,
                                                                                     ncp, M, M01);
    }
    const int nlev = (int)c->level_begin.size() - 1;
    for (int l = nlev - 2; l >= 0; --l) {
        const int lb = c->level_begin[l], le = c->level_begin[l + 1];
        if (high) {
            if ((st = launch_m2m_hi<T>(c, t, lb, le, p, nc, ncp, M, M01))) return st;
            continue;
        }
        ProfScope ps_(c, TG_K_UP);
        m2m_level<T><<<std::min(le - lb, c->num_sms * 8), kM2MThreads, 8 * 2 * ncp * sizeof(T), c->stream>>>(
            t, lb, le, p, nc, ncp, M, M01, nullptr, 0);
    }
    {
        ProfScope ps_(c, TG_K_UP);
        scale_moments<T><<<grid_for((int64_t)ncell * ncp, 256), 256, 0, c->stream>>>(ncell, nc, ncp, M, M01, Ms, nullptr);
    }
    cudaMemsetAsync(L, 0, sizeof(T) * (size_t)ncell * 2 * ncp, c->stream);
    const M2LBlock *blocks = static_cast<const M2LBlock *>(c->buf[B_M2L].p);
    const uint2 *p2p = static_cast<const uint2 *>(c->buf[B_P2P].p);
    uint32_t *fpre = nullptr;
    if (masked && sizeof(T) == 4 && (st = fast_prefix(c, fs, n, &fpre, nullptr))) return st;
    if (n_blocks > 0 && (st = launch_m2l_t(c, t, blocks, n_blocks, Ms, L, p, nc, ncp, masked, want_pot, fpre))) return st;
    for (int l = 1; l < nlev; ++l) {
        const int lb = c->level_begin[l], le = c->level_begin[l + 1];
        if (high) {
            if ((st = launch_l2l_hi<T>(c, t, lb, le, p, nc, ncp, ncls, want_pot ? 0 : 1, L))) return st;
            continue;
        }
        ProfScope ps_(c, TG_K_DOWN);
        l2l_level<T><<<grid_for((int64_t)(le - lb) * 32, 32 * kM2MWarps), 32 * kM2MWarps,
                       kM2MWarps * 2 * ncp * sizeof(T), c->stream>>>(t, lb, le, p, nc, ncp, ncls,
                                                                     want_pot ? 0 : 1, L, nullptr, 0);
    }
    if (high) {
        if ((st = launch_l2p_hi<T, T4>(c, n, t, pf, leaf_of, fs, masked, p, ncp, L, acc4))) return st;
    } else {
        ProfScope ps_(c, TG_K_DOWN);
        const int g = grid_for(n, 128), mk = masked ? 1 : 0;
#define TG_L2P(PP)                                                                                                 \
    case PP:                                                                                                       \
        if (want_pot) l2p_fixed<PP, T, T4, true><<<g, 128, 0, c->stream>>>(n, t, d_geom, pf, leaf_of, fs, mk, ncp, L, acc4, n, nullptr); \
        else l2p_fixed<PP, T, T4, false><<<g, 128, 0, c->stream>>>(n, t, d_geom, pf, leaf_of, fs, mk, ncp, L, acc4, n, nullptr); \
        break;
        switch (p) {
            TG_L2P(4)
            TG_L2P(5)
            TG_L2P(6)
        default:
            l2p_particles<T, T4><<<grid_for(n, 128), 128, 0, c->stream>>>(n, t, c->walk_log2L, pf, leaf_of, fs, masked ? 1 : 0,
                                                                      p, nc, ncp, L, acc4);
        }
#undef TG_L2P
    }
    if ((st = launch_p2p_t(c, t, d_geom, p2p, n_p2p, p2p + (c->p2p_cap - n_self), n_self, pf, fs, nslow, masked,
                            want_pot, acc4)))
        return st;
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
    if (c->prm.mac == TG_MAC_SPHERE && (st = cell_radii(c, t, d_geom))) return st;
    int64_t n_blocks = 0, n_m2l = 0, n_p2p = 0, n_self = 0;
    if ((st = run_walk(c, t, &n_blocks, &n_m2l, &n_p2p, &n_self))) return st;
    c->last_n = n;
    c->last_ncell = ncell;
    c->last_nm2l = n_m2l;
    c->last_nblocks = n_blocks;
    c->last_np2p = n_p2p + n_self;
    c->last_np2p_self = n_self;
    const bool masked = fast != nullptr;
    if (c->prm.precision == TG_PREC_FP32) st = eval_typed<float, float4>(c, n, ncell, t, d_geom, masked, pot != nullptr, n_blocks, n_p2p, n_self);
    else st = eval_typed<double, dbl4>(c, n, ncell, t, d_geom, masked, pot != nullptr, n_blocks, n_p2p, n_self);
    if (st) return st;
    const uint32_t *perm = static_cast<const uint32_t *>(c->buf[B_VALS0].p);
    const double *acc4 = static_cast<const double *>(c->buf[B_ACC].p);
    {
        ProfScope ps_(c, TG_K_DOWN);
        scatter_out<<<grid_for(n, 256), 256, 0, c->stream>>>(n, perm, acc4, acc, out_stride, pot, nullptr, n);
    }
    c->stats.evaluations += 1;
    c->stats.sink_forces += n;
    c->stats.m2l_pairs += n_m2l;
    if (!m2l_classes_on_device(c)) c->stats.m2l_class_pairs += n_m2l * (masked ? 2 : 1);
    c->stats.p2p_cell_pairs += n_p2p + n_self;
    c->stats.cells += ncell;
    return cuda_check(c, cudaGetLastError(), "fmm scatter");
}

// fast flags of the sorted particles as words, with a zero at n (the prefix sum then ends in its total)
__global__ void fast_words(const uint8_t *fs, int n, uint32_t *w, const int *dn)
{
    n = dev_or(dn, n);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) w[i] = i < n ? fs[i] : 0u;
}

tg_status fast_prefix(tg_ctx *c, const uint8_t *fs, int n, uint32_t **fpre, const DevEval *de)
{
    tg_status st;
    uint32_t *w, *pre;
    if ((st = ensure_t(c, B_FWORDS, (size_t)n + 1, &w)) || (st = ensure_t(c, B_FPRE, (size_t)n + 1, &pre))) return st;
    {
        ProfScope ps_(c, TG_K_M2L);
        fast_words<<<grid_for((int64_t)n + 1, 256), 256, 0, c->stream>>>(fs, n, w, de ? &de->n : nullptr);
    }
    if ((st = exclusive_scan_u32(c, w, pre, n + 1, nullptr, de ? &de->np1 : nullptr))) return st;
    *fpre = pre;
    return TG_OK;
}

// zero rows[0] rows of `width` values (device row count)
template <class T>
__global__ void zero_rows_dev(T *p, const int *rows, int width)
{
    const int64_t n = (int64_t)*rows * width;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = T(0);
}

// ------------------------------------------------------------------ one evaluation, sizes on the device
// The batched HOLD step runs every evaluation inside one CUDA graph, so no size can be read on the host:
// the walk's counters, the tree's levels and cell count, and the particle count stay on the device, the
// launches are sized for the capacities in BatchCaps, and anything that would pass a capacity sets an
// overflow bit (the step is then restored and redone with larger buffers).  Float32, accelerations only,
// always with the two moment classes of a kick pair (the classes are read from de->masked).
__global__ void walk_init_dev(const DevEval *de, uint2 *front, unsigned long long *ctr, uint2 *p2p,
                              unsigned long long cap_p2p)
{
    for (int i = threadIdx.x; i < 8 + kWalkMaxSteps + 1; i += blockDim.x) ctr[i] = 0ull;
    __syncthreads();
    if (threadIdx.x == 0) {
        if (de->ncell == 1) {
            p2p[cap_p2p - 1] = make_uint2(0, 0);   // the root is a leaf: one self pair
            ctr[4] = 1ull;
        } else {
            front[0] = make_uint2(0, 0);
            ctr[8] = 1ull;
        }
    }
}

// lists over capacity (the walk stopped writing at the capacity): flag the step and clamp the counts,
// so that the launches after the walk stay inside their buffers
__global__ void walk_check_dev(DevEval *de, unsigned long long *ctr, int nsteps, unsigned long long cap_front,
                               unsigned long long cap_blocks, unsigned long long cap_p2p)
{
    bool over = ctr[8 + nsteps] != 0ull;
    for (int s = 1; s <= nsteps; ++s) over |= ctr[8 + s] > cap_front;
    over |= ctr[1] > cap_blocks || ctr[2] + ctr[4] > cap_p2p;
    if (over) {
        de->overflow |= 4u;
        ctr[1] = ctr[1] < cap_blocks ? ctr[1] : cap_blocks;
        ctr[2] = ctr[2] < cap_p2p ? ctr[2] : cap_p2p;
        ctr[4] = ctr[4] < cap_p2p - ctr[2] ? ctr[4] : cap_p2p - ctr[2];
    }
}

// counters of the evaluation into the step's totals: [0] evaluations, [1] particle-forces, [2] M2L pairs,
// [3] M2L pairs x classes (when the M2L kernels do not count them on the device), [4] P2P leaf pairs,
// [5] cells
__global__ void eval_finish_dev(const DevEval *de, const unsigned long long *ctr, unsigned long long *stats,
                                int count_classes)
{
    stats[0] += 1ull;
    stats[1] += (unsigned long long)de->n;
    stats[2] += ctr[3];
    if (count_classes) stats[3] += ctr[3] * (de->masked ? 2ull : 1ull);
    stats[4] += ctr[2] + ctr[4];
    stats[5] += (unsigned long long)de->ncell;
}

// The parts of the criterion's thresholds that do not depend on the root cube, uploaded once before a
// batched step is captured (mac_params_dev fills in the rest on every evaluation).  Synchronising.
tg_status mac_params_upload(tg_ctx *c)
{
    MacParams *mpd;
    tg_status st = ensure_t(c, B_MACP, 1, &mpd);
    if (st) return st;
    const MacParams mp = make_mac_params(c->prm, 0);
    return cuda_check(c, cudaMemcpy(mpd, &mp, sizeof(mp), cudaMemcpyHostToDevice), "criterion upload");
}

template <class T, class T4>
static tg_status fmm_eval_dev_t(tg_ctx *c, DevEval *de, const BatchCaps &cap, const double *xin, const double *min,
                                const uint8_t *fin, double *acc, unsigned long long *stats)
{
    tg_status st;
    const int p = c->prm.p, nc = ncoef(p), ncp = pad4(nc);
    if (p < 4 || p > 6) return set_err(c, TG_ERR_ARG, "batched evaluation needs 4 <= p <= 6");
    Geom *d_geom;
    MacParams *mpd;
    if ((st = ensure_t(c, B_GEOM, 1, &d_geom)) || (st = ensure_t(c, B_MACP, 1, &mpd))) return st;
    if ((st = root_cube(c, cap.n, xin, cap.n, nullptr, d_geom, &de->n))) return st;
    {
        ProfScope ps_(c, TG_K_WALK);
        mac_params_dev<<<1, 32, 0, c->stream>>>(d_geom, c->prm.eps, mpd);
    }
    if ((st = keys_sort_gather(c, cap.n, xin, cap.n, nullptr, min, fin, d_geom, de))) return st;
    if ((st = build_octree_dev(c, de, cap.cells, cap.levels))) return st;
    TreeView t = tree_view(c, cap.n, cap.cells);
    t.d_ncell = &de->ncell;

    // dual walk (Algorithm 4), every step queued, counters on the device
    uint2 *f0, *f1, *p2p;
    M2LBlock *blocks;
    unsigned long long *wctr;
    if ((st = ensure_t(c, B_FRONT0, cap.front, &f0)) || (st = ensure_t(c, B_FRONT1, cap.front, &f1)) ||
        (st = ensure_t(c, B_M2L, cap.blocks, &blocks)) || (st = ensure_t(c, B_P2P, cap.p2p, &p2p)) ||
        (st = ensure_t(c, B_WALK_CNT, 8 + kWalkMaxSteps + 1, &wctr)))
        return st;
    const int nsteps = std::min(kWalkMaxSteps, cap.levels);
    // the walk reads only the cells: it runs on the side stream beside the leaf passes and the moments
    // (ev_walk marks its end for M2L), and P2P follows it there
    cudaEventRecord(c->ev_fork, c->stream);
    cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    {
        cudaStream_t main_stream = c->stream;
        c->stream = c->side;
        {
            ProfScope ps_(c, TG_K_WALK);
            walk_init_dev<<<1, 64, 0, c->stream>>>(de, f0, wctr, p2p, cap.p2p);
        }
        for (int s = 0; s < nsteps; ++s) {
            WalkOut o{(s & 1) ? f0 : f1, blocks, p2p, wctr, wctr + 8 + s + 1, cap.front, cap.blocks, cap.p2p};
            ProfScope ps_(c, TG_K_WALK);
            walk_step_dev<<<c->num_sms * 4, 128, 0, c->stream>>>(t, mpd, (s & 1) ? f1 : f0, wctr + 8 + s, o);
        }
        {
            ProfScope ps_(c, TG_K_WALK);
            walk_check_dev<<<1, 1, 0, c->stream>>>(de, wctr, nsteps, cap.front, cap.blocks, cap.p2p);
        }
        c->stream = main_stream;
    }
    cudaEventRecord(c->ev_walk, c->side);

    // slow-first leaves, per-particle offsets, upward pass
    const double *xs = static_cast<const double *>(c->buf[B_XS].p), *ys = static_cast<const double *>(c->buf[B_YS].p),
                 *zs = static_cast<const double *>(c->buf[B_ZS].p), *ms = static_cast<const double *>(c->buf[B_MS].p);
    const uint8_t *fs = static_cast<const uint8_t *>(c->buf[B_FS].p);
    const uint32_t *perm = static_cast<const uint32_t *>(c->buf[B_VALS0].p);
    double *xs2, *ys2, *zs2, *ms2, *M01, *acc4;
    uint8_t *fs2;
    uint32_t *perm2;
    int32_t *nslow, *leaf_of;
    T4 *pf;
    T *M, *Ms, *L;
    const size_t rows = (size_t)cap.cells * 2;
    if ((st = ensure_t(c, B_XS2, cap.n, &xs2)) || (st = ensure_t(c, B_YS2, cap.n, &ys2)) ||
        (st = ensure_t(c, B_ZS2, cap.n, &zs2)) || (st = ensure_t(c, B_MS2, cap.n, &ms2)) ||
        (st = ensure_t(c, B_FS2, cap.n, &fs2)) || (st = ensure_t(c, B_PERM2, cap.n, &perm2)) ||
        (st = ensure_t(c, B_NSLOW, cap.cells, &nslow)) || (st = ensure_t(c, B_PF, cap.n, &pf)) ||
        (st = ensure_t(c, B_LEAF_OF, cap.n, &leaf_of)) || (st = ensure_t(c, B_MOM, rows * ncp, &M)) ||
        (st = ensure_t(c, B_MOMF, rows * ncp, &Ms)) || (st = ensure_t(c, B_MOM01, rows * 4, &M01)) ||
        (st = ensure_t(c, B_LOC, rows * ncp, &L)) || (st = ensure_t(c, B_ACC, (size_t)4 * cap.n, &acc4))) {
        cudaStreamWaitEvent(c->stream, c->ev_walk, 0);   // no unjoined work on the side stream
        return st;
    }
    const int gcell = grid_for((int64_t)cap.cells * 32, 256);
    {
        ProfScope ps_(c, TG_K_TREE);
        leaf_class_partition<<<gcell, 256, 0, c->stream>>>(t, xs, ys, zs, ms, fs, perm, xs2, ys2, zs2, ms2, fs2, perm2,
                                                           nslow);
    }
    {
        ProfScope ps_(c, TG_K_UP);
        leaf_particles<T4><<<gcell, 256, 0, c->stream>>>(t, d_geom, xs2, ys2, zs2, ms2, pf, leaf_of);
    }
    // float32: P2P needs only the walk's lists and the leaf offsets, so it runs on the side stream (after
    // the walk) beside the moments, M2L and the downward pass, into its own sums (acc4p, added by
    // scatter_out); its scan takes its own scratch slot.  The forks and joins are events, which a stream
    // capture turns into graph edges.
    double *acc4p = nullptr;
    const bool fork = sizeof(T) == 4;
    if (fork) {
        if ((st = ensure_t(c, B_ACC_P2P, (size_t)4 * cap.n, &acc4p))) {
            cudaStreamWaitEvent(c->stream, c->ev_walk, 0);
            return st;
        }
        cudaEventRecord(c->ev_fork, c->stream);   // the leaf offsets; the side stream is past the walk
        cudaStreamWaitEvent(c->side, c->ev_fork, 0);
        cudaStream_t main_stream = c->stream;
        c->stream = c->side;
        {
            ProfScope ps_(c, TG_K_OTHER);
            zero_acc3<<<c->num_sms * 4, 256, 0, c->stream>>>(acc4p, cap.n, &de->n);
        }
        st = launch_p2p_f32_dev(c, t, de, d_geom, wctr, p2p, cap.p2p, cap.cells, reinterpret_cast<const float4 *>(pf),
                                nslow, acc4p, cap.n, B_SCAN_TMP2);
        c->stream = main_stream;
        cudaEventRecord(c->ev_join, c->side);
        if (st) {
            cudaStreamWaitEvent(c->stream, c->ev_join, 0);
            return st;
        }
    } else {
        cudaEventRecord(c->ev_join, c->side);   // float64: P2P follows on the main stream
    }
    {
        ProfScope ps_(c, TG_K_UP);
        p2m_leaves<T, T4><<<grid_for((int64_t)cap.cells * 32, 128), 128, 0, c->stream>>>(
            t, d_geom, xs2, ys2, zs2, ms2, fs2, pf, p, nc, ncp, M, M01);
    }
    for (int l = cap.levels - 1; l >= 0; --l) {
        ProfScope ps_(c, TG_K_UP);
        m2m_level<T><<<c->num_sms * 8, kM2MThreads, 8 * 2 * ncp * sizeof(T), c->stream>>>(t, 0, 0, p, nc, ncp, M, M01,
                                                                                          de, l);
    }
    {
        ProfScope ps_(c, TG_K_UP);
        scale_moments<T><<<grid_for((int64_t)cap.cells * ncp, 256), 256, 0, c->stream>>>(cap.cells, nc, ncp, M, M01, Ms,
                                                                                        &de->ncell);
        zero_rows_dev<T><<<c->num_sms * 4, 256, 0, c->stream>>>(L, &de->rows, ncp);
    }
    cudaStreamWaitEvent(c->stream, c->ev_walk, 0);   // M2L reads the walk's blocks
    if (sizeof(T) == 4) {
        uint32_t *fpre = nullptr;
        st = fast_prefix(c, fs2, cap.n, &fpre, de);
        if (!st)
            st = launch_m2l_f32_dev(c, t, de, d_geom, blocks, wctr + 1, (int64_t)cap.blocks,
                                    reinterpret_cast<const float *>(Ms), reinterpret_cast<float *>(L), p, ncp, cap.cells,
                                    cap.m2l_src, fpre);
    } else {
        st = launch_m2l_f64_dev(c, t, de, d_geom, blocks, wctr + 1, (int64_t)cap.blocks,
                                reinterpret_cast<const double *>(Ms), reinterpret_cast<double *>(L), p, ncp);
    }
    if (st) {
        cudaStreamWaitEvent(c->stream, c->ev_join, 0);   // no unjoined work on the side stream
        return st;
    }
    for (int l = 1; l <= cap.levels; ++l) {
        ProfScope ps_(c, TG_K_DOWN);
        l2l_level<T><<<c->num_sms * 16, 32 * kM2MWarps, kM2MWarps * 2 * ncp * sizeof(T), c->stream>>>(
            t, 0, 0, p, nc, ncp, 2, 1, L, de, l);
    }
    {
        ProfScope ps_(c, TG_K_DOWN);
        const int g = grid_for(cap.n, 128);
        switch (p) {
        case 4:
            l2p_fixed<4, T, T4, false><<<g, 128, 0, c->stream>>>(cap.n, t, d_geom, pf, leaf_of, fs2, 1, ncp, L, acc4, cap.n, de);
            break;
        case 5:
            l2p_fixed<5, T, T4, false><<<g, 128, 0, c->stream>>>(cap.n, t, d_geom, pf, leaf_of, fs2, 1, ncp, L, acc4, cap.n, de);
            break;
        default:
            l2p_fixed<6, T, T4, false><<<g, 128, 0, c->stream>>>(cap.n, t, d_geom, pf, leaf_of, fs2, 1, ncp, L, acc4, cap.n, de);
        }
    }
    cudaStreamWaitEvent(c->stream, c->ev_join, 0);
    if (!fork && (st = launch_p2p_f64_dev(c, t, d_geom, wctr, p2p, cap.p2p, reinterpret_cast<const dbl4 *>(pf), fs2, acc4,
                                         cap.n)))
        return st;
    {
        ProfScope ps_(c, TG_K_DOWN);
        scatter_out<<<grid_for(cap.n, 256), 256, 0, c->stream>>>(cap.n, perm2, acc4, acc, cap.n, nullptr, &de->n, cap.n,
                                                                  acc4p);
    }
    {
        ProfScope ps_(c, TG_K_OTHER);
        eval_finish_dev<<<1, 1, 0, c->stream>>>(de, wctr, stats, m2l_classes_on_device(c) ? 0 : 1);
    }
    return cuda_check(c, cudaGetLastError(), "fmm evaluation (device sizes)");
}

tg_status fmm_eval_dev(tg_ctx *c, DevEval *de, const BatchCaps &cap, const double *xin, const double *min,
                       const uint8_t *fin, double *acc, unsigned long long *stats)
{
    if (c->prm.precision == TG_PREC_FP32) return fmm_eval_dev_t<float, float4>(c, de, cap, xin, min, fin, acc, stats);
    return fmm_eval_dev_t<double, dbl4>(c, de, cap, xin, min, fin, acc, stats);
}

}  // namespace tg
