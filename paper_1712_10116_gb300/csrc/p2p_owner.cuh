// p2p_owner.cuh -- mutual P2P of distinct leaf pairs with rows packed across partners (float32).
//
// Each unordered leaf pair {A, B} (A != B) gets one owner: the larger leaf (ties: the larger
// index).  A warp takes an owner B.  B's particles are the columns.  They are staged once in
// shared memory, together with B's reaction sums.  The particles of B's partners are packed
// densely into the rows, in chunks of 32*ROWS.  Each row is shifted into B's frame by the exact
// centre offset of its own leaf, so no row slot is wasted on the tail of a small leaf.  For every
// row/column pair the kernel value is computed once and applied to both particles, with opposite
// signs (Sec. 2.1, Eq. 2).  Rows keep their sums in registers and flush them once per chunk.
// Columns combine their partials with a warp reduce-scatter into shared memory, and flush them
// once per work unit (kOwnUnit partners of the owner; the units of all owners are handed out
// dynamically to the warps).
//
// With slow/fast classes the leaves hold their slow particles first.  Slow rows meet every
// column; fast rows meet only the owner's slow columns, so no fast-fast pair reaches a sum (a
// kickS2F feels the slow masses only).  The columns are staged in leaf order and padded to a
// multiple of 8 once; in the fast-row pass the fast columns of the batch that holds the slow/fast
// boundary carry zero mass and their reaction sums are dropped.  Within a batch the partners whose cube lies closer
// than eps to the owner's come first; chunks made only of the other partners' rows need no softening
// test, the others take the pair value at max(r, eps) and correct the rare pairs with r < eps.
#pragma once
#include "p2p_tile.cuh"

namespace tg {

constexpr int kOwnUnit = 32;   // partners per work unit of the owner kernel (one per lane)

// Owner and partner of each distinct leaf pair, and per-owner partner counts (own_cnt starts at zero).
// The walk writes the pairs of one row cell side by side, so lanes of a warp often share an owner:
// the lanes with equal owners add their count with one atomic (whole warps iterate together).
__global__ void p2p_owner_count(const uint2 *__restrict__ pairs, int64_t npairs, const int32_t *__restrict__ count,
                                uint32_t *own_cnt, uint2 *tagged, const unsigned long long *dnp)
{
    if (dnp) npairs = (int64_t)*dnp;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x; w0 < npairs; w0 += stride) {
        const int64_t w = w0 + threadIdx.x;
        uint32_t owner = 0xffffffffu;
        if (w < npairs) {
            const uint32_t x = pairs[w].x, y = pairs[w].y;
            const int cx = count[x], cy = count[y];
            owner = (cx > cy || (cx == cy && x > y)) ? x : y;
            tagged[w] = make_uint2(owner, owner == x ? y : x);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, owner);
        if (owner != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(&own_cnt[owner], (uint32_t)__popc(peers));
    }
}

// Partners grouped by owner: partners[own_off[B] .. own_off[B] + own_cnt[B]).  Every kOwnUnit-th
// partner of an owner also opens a work unit (owner, position); ctr[0] counts the units.
// own_fill and ctr start at zero.  Lanes with equal owners take consecutive slots with one atomic, and
// the units a warp opens are reserved with one atomic on ctr[0] (whole warps iterate together).
__global__ void p2p_owner_fill(const uint2 *__restrict__ tagged, int64_t npairs, const uint32_t *__restrict__ own_off,
                               uint32_t *own_fill, int32_t *partners, uint2 *units, uint32_t *ctr,
                               const unsigned long long *dnp)
{
    if (dnp) npairs = (int64_t)*dnp;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x; w0 < npairs; w0 += stride) {
        const int64_t w = w0 + threadIdx.x;
        const bool valid = w < npairs;
        uint2 op = make_uint2(0xffffffffu, 0u);
        if (valid) op = tagged[w];
        const unsigned peers = __match_any_sync(0xffffffffu, op.x);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0u;
        if (valid && lane == leader) base = atomicAdd(&own_fill[op.x], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        const uint32_t f = base + (uint32_t)__popc(peers & lt);
        if (valid) partners[own_off[op.x] + f] = (int32_t)op.y;
        const bool opens = valid && f % kOwnUnit == 0;
        const unsigned ob = __ballot_sync(0xffffffffu, opens);
        uint32_t ubase = 0u;
        if (lane == 0 && ob) ubase = atomicAdd(&ctr[0], (uint32_t)__popc(ob));
        ubase = __shfl_sync(0xffffffffu, ubase, 0);
        if (opens) units[ubase + __popc(ob & lt)] = make_uint2(op.x, f);
    }
}

// The partners of one work unit (at most 32), in slot order (near partners first).
struct OwnerBatch {
    float4 off[32];    // centre of the partner minus centre of the owner
    int first[32];     // first particle of the partner
    int nslow[32];     // slow particles of the partner (all of them without classes)
    int inc[2][32];    // inclusive row counts over slots: [0] slow rows, [1] fast rows
};

// Columns are staged in leaf order (slow first) and padded to a multiple of 8 with massless
// particles far away (on the other side of the origin from the padding rows), so every batch of 8
// columns is full.  Two neighbouring columns 2m, 2m+1 share two float4 slots, component-major:
// q[2m] = (x0, x1, y0, y1), q[2m+1] = (z0, z1, m0, m1), so one shared load gives each coordinate of
// both columns as a float2 and the pair arithmetic runs on packed float2 operations.
constexpr int kOwnCols = kMaxNcrit + 16;

struct OwnerShared {
    float4 q[8][kOwnCols];       // owner's particles (columns), per warp, in column pairs
    float acc[8][kOwnCols][4];   // owner's reaction sums (ax, ay, az, phi), per warp
    OwnerBatch b[8];
};

__device__ __forceinline__ void col_put(float4 *sq, int j, float4 v)
{
    float *f = reinterpret_cast<float *>(sq) + 8 * (j >> 1) + (j & 1);
    f[0] = v.x;
    f[2] = v.y;
    f[4] = v.z;
    f[6] = v.w;
}

__device__ __forceinline__ float4 col_get(const float4 *sq, int j)
{
    const float *f = reinterpret_cast<const float *>(sq) + 8 * (j >> 1) + (j & 1);
    return make_float4(f[0], f[2], f[4], f[6]);
}

__device__ __forceinline__ void col_zero_mass(float4 *sq, int j) { reinterpret_cast<float *>(sq)[8 * (j >> 1) + 6 + (j & 1)] = 0.f; }

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// Rows i0 .. i0 + 32*ROWS of one phase (0: slow rows, 1: fast rows) against the first ncol staged
// columns (a multiple of 8); the reaction sums of columns at or past nkeep are not kept.
// Each row meets two columns per packed operation: a row keeps two partial sums per component (one
// per column parity, added when the chunk is flushed); a column pair keeps its two columns' sums in
// one float2 across the rows.  Every product and sum is rounded as in the scalar form; only the order
// in which a row's sum is accumulated differs.
template <int KERNEL, int ROWS, bool NEAR, bool POT>
__device__ __noinline__ void owner_rows(const float4 *__restrict__ pf, const OwnerBatch *ob, int phase, int i0, int nrows,
                                        const float4 *sq, float (*sacc)[4], int ncol, int nkeep, float eps, double *acc4,
                                        int n, int lane)
{
    const float eps2 = eps * eps, inv_eps = 1.0f / eps, inv_eps3 = inv_eps * inv_eps * inv_eps;
    const int *inc = ob->inc[phase];
    float2 nx[ROWS], ny[ROWS], nz[ROWS], nm[ROWS];   // -x, -y, -z, -m of each row, in both halves
    int gi[ROWS];
    float2 ra[ROWS][4];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
        const int i = i0 + lane + 32 * r;
        gi[r] = -1;
        float4 q = make_float4(1e8f, 1e8f, 1e8f, 0.f);   // far away, massless
        if (i < nrows) {
            // slot s: the first with inc[s] > i (inc is non-decreasing and inc[31] = nrows > i)
            int s = 0;
#pragma unroll
            for (int b = 16; b >= 1; b >>= 1)
                if (inc[s + b - 1] <= i) s += b;
            const int loc = i - (s ? inc[s - 1] : 0);
            gi[r] = ob->first[s] + (phase ? ob->nslow[s] : 0) + loc;
            const float4 o = ob->off[s];
            q = pf[gi[r]];
            q.x += o.x;
            q.y += o.y;
            q.z += o.z;
        }
        nx[r] = f2(-q.x, -q.x);
        ny[r] = f2(-q.y, -q.y);
        nz[r] = f2(-q.z, -q.z);
        nm[r] = f2(-q.w, -q.w);
#pragma unroll
        for (int comp = 0; comp < 4; ++comp) ra[r][comp] = f2(0.f, 0.f);
    }
    // Wendland C2 and a partner closer than eps: the pair value is first taken at max(r, eps), where
    // it equals the Newtonian one, and pairs with r < eps are corrected after the batch (rare).
    constexpr bool CLAMP = NEAR && KERNEL == TG_KERNEL_WENDLAND_C2;
    // columns in batches of 8 (4 pairs); lane l visits pair m ^ ((l >> 3) & 3) at step m, so the first
    // two stages of the reduce-scatter below need no selects
    const int pperm = (lane >> 3) & 3;
    for (int j0 = 0; j0 < ncol; j0 += 8) {
        float2 col[4][4];   // [step][component]: (even column, odd column) of the pair visited at that step
        bool close = false;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int jp = (j0 >> 1) + (m ^ pperm);
            const float4 qa = sq[2 * jp], qb = sq[2 * jp + 1];
            const float2 qx = f2(qa.x, qa.y), qy = f2(qa.z, qa.w), qz = f2(qb.x, qb.y), qm = f2(qb.z, qb.w);
            float2 cx = f2(0.f, 0.f), cy = cx, cz = cx, cp = cx;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
                const float2 dx = __fadd2_rn(qx, nx[r]), dy = __fadd2_rn(qy, ny[r]), dz = __fadd2_rn(qz, nz[r]);
                const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
                float2 ri;
                if (KERNEL == TG_KERNEL_PLUMMER) {
                    ri = f2(tg_rsqrt<float>(r2.x + eps2), tg_rsqrt<float>(r2.y + eps2));
                } else if (CLAMP) {
                    close |= (r2.x < eps2) | (r2.y < eps2);
                    ri = f2(rsqrt_ftz(fmaxf(r2.x, eps2)), rsqrt_ftz(fmaxf(r2.y, eps2)));
                } else {
                    ri = f2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));   // far pairs: r2 >= eps^2
                }
                // g = ri^3, phi = -ri (a row keeps its potential sum negated and flips it at the flush; a column
                // pair's potential sum, -m_row * ri, has its own sign)
                const float2 g = __fmul2_rn(__fmul2_rn(ri, ri), ri);
                const float2 mq = __fmul2_rn(qm, g), nmp = __fmul2_rn(nm[r], g);
                ra[r][0] = __ffma2_rn(mq, dx, ra[r][0]);
                ra[r][1] = __ffma2_rn(mq, dy, ra[r][1]);
                ra[r][2] = __ffma2_rn(mq, dz, ra[r][2]);
                if (POT) ra[r][3] = __ffma2_rn(qm, ri, ra[r][3]);
                cx = __ffma2_rn(nmp, dx, cx);
                cy = __ffma2_rn(nmp, dy, cy);
                cz = __ffma2_rn(nmp, dz, cz);
                if (POT) cp = __ffma2_rn(nm[r], ri, cp);
            }
            col[m][0] = cx;
            col[m][1] = cy;
            col[m][2] = cz;
            col[m][3] = cp;
        }
        if (CLAMP && __any_sync(0xffffffffu, close)) {
            // exact softened value minus the clamped one, for the pairs with r < eps; rows in registers,
            // columns straight into the shared sums (before the batch's own column sums are added).  Lane l
            // takes column c ^ ((l >> 2) & 7) at step c, so at most 4 lanes add to one column's sums at once.
#pragma unroll 1
            for (int c = 0; c < 8; ++c) {
                const int j = j0 + (c ^ ((lane >> 2) & 7));
                const float4 q = col_get(sq, j);
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    const float dx = q.x + nx[r].x, dy = q.y + ny[r].x, dz = q.z + nz[r].x;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    if (r2 < eps2) {
                        const float ri = rsqrtf(eps2);
                        float g, ph;
                        pair_kernel<float, TG_KERNEL_WENDLAND_C2>(r2, eps, eps2, inv_eps, inv_eps3, g, ph);
                        const float dg = g - ri * ri * ri, dph = ph + ri;
                        const float mq = q.w * dg, mp = -nm[r].x * dg;
                        ra[r][0].x = fmaf(mq, dx, ra[r][0].x);
                        ra[r][1].x = fmaf(mq, dy, ra[r][1].x);
                        ra[r][2].x = fmaf(mq, dz, ra[r][2].x);
                        if (POT) ra[r][3].x = fmaf(q.w, -dph, ra[r][3].x);
                        if (j < nkeep) {
                            atomicAdd(&sacc[j][0], -mp * dx);
                            atomicAdd(&sacc[j][1], -mp * dy);
                            atomicAdd(&sacc[j][2], -mp * dz);
                            if (POT) atomicAdd(&sacc[j][3], -nm[r].x * dph);
                        }
                    }
                }
            }
            __syncwarp();
        }
        // reduce-scatter of the 8 columns x 4 components over the warp; lane l ends with column
        // j0 + l/4, component l%4.  Pair bits (partners l^16, l^8) without selects ...
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int comp = 0; comp < (POT ? 4 : 3); ++comp)
                col[m][comp] = __fadd2_rn(col[m][comp], f2(__shfl_xor_sync(0xffffffffu, col[m + 2][comp].x, 16),
                                                            __shfl_xor_sync(0xffffffffu, col[m + 2][comp].y, 16)));
#pragma unroll
        for (int comp = 0; comp < (POT ? 4 : 3); ++comp)
            col[0][comp] = __fadd2_rn(col[0][comp], f2(__shfl_xor_sync(0xffffffffu, col[1][comp].x, 8),
                                                        __shfl_xor_sync(0xffffffffu, col[1][comp].y, 8)));
        // ... column parity (l^4), then the component bits (l^2, l^1), with selects
        float v[4];
        {
            const bool hi = (lane & 4) != 0;
#pragma unroll
            for (int comp = 0; comp < 4; ++comp) {
                if (!POT && comp == 3) {
                    v[3] = 0.f;
                    continue;
                }
                const float send = hi ? col[0][comp].x : col[0][comp].y;
                const float keep = hi ? col[0][comp].y : col[0][comp].x;
                v[comp] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
            }
        }
#pragma unroll
        for (int h = 2; h >= 1; h >>= 1) {
            const bool hi = (lane & h) != 0;
#pragma unroll
            for (int q = 0; q < h; ++q) {
                const float send = hi ? v[q] : v[q + h];
                const float keep = hi ? v[q + h] : v[q];
                v[q] = keep + __shfl_xor_sync(0xffffffffu, send, h);
            }
        }
        if (j0 + (lane >> 2) < nkeep) sacc[j0 + (lane >> 2)][lane & 3] += v[0];
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r)
        if (gi[r] >= 0) {
            const float s[4] = {ra[r][0].x + ra[r][0].y, ra[r][1].x + ra[r][1].y, ra[r][2].x + ra[r][2].y,
                                -(ra[r][3].x + ra[r][3].y)};
#pragma unroll
            for (int comp = 0; comp < (POT ? 4 : 3); ++comp) atomicAdd(&acc4[(size_t)comp * n + gi[r]], f2d_exact(s[comp]));
        }
}

__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, d);
        if (lane >= d) v += u;
    }
    return v;
}

// One warp per work unit (kOwnUnit partners of one owner), units taken from a shared counter
// (ctr[1], starts at zero) so that the load stays balanced whatever the spread of leaf work.  After
// the units, the same counter hands out the self pairs (A, A): slow rows of A against every particle
// of A with a larger index, i.e. each slow-slow and slow-fast pair once (p2p_pair_f32, SELF).
// Batched path (walk_ctr non-null): the root cube comes from gp and the self pairs from the walk's
// counters on the device (they sit at the end of the P2P buffer of capacity cap_p2p).
template <int KERNEL, int ROWS, bool POT>
__global__ void __launch_bounds__(256, 2) p2p_owner_f32(TreeView t, int log2L, const uint2 *__restrict__ units,
                                                        uint32_t *ctr, const uint32_t *__restrict__ own_off,
                                                        const uint32_t *__restrict__ own_cnt,
                                                        const int32_t *__restrict__ partners,
                                                        const uint2 *__restrict__ self_pairs, uint32_t nself,
                                                        const float4 *__restrict__ pf, const int32_t *__restrict__ nslow,
                                                        float eps, double *acc4, int n, unsigned long long *pair_counter,
                                                        const Geom *gp, const unsigned long long *walk_ctr,
                                                        const uint2 *p2p_base, unsigned long long cap_p2p)
{
    if (walk_ctr) {
        log2L = gp->log2L;
        nself = (uint32_t)walk_ctr[4];
        self_pairs = p2p_base + (cap_p2p - nself);
    }
    static_assert(kOwnUnit <= 32, "one partner per lane");
    __shared__ OwnerShared sh;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    float4 *sq = sh.q[wib];
    float(*sacc)[4] = sh.acc[wib];
    OwnerBatch *ob = &sh.b[wib];
    const uint32_t nunits = ctr[0];
    unsigned long long my_pairs = 0;
    for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(&ctr[1], 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if (k >= nunits) {
            if (k - nunits >= nself) break;
            const int A = (int)self_pairs[k - nunits].x;
            const int fa = t.first[A], na = t.count[A], sa = nslow ? nslow[A] : na;
            if (sa == 0) continue;   // no slow row: every pair of the leaf is fast-fast
            __syncwarp();
            p2p_pair_f32<KERNEL, true, ROWS, true>(pf, fa, sa, fa, na, 0.f, 0.f, 0.f, eps, acc4, n, lane, sq);
            if (lane == 0) {
                const unsigned long long nf = na - sa;
                my_pairs += (unsigned long long)na * (na - 1) / 2 - nf * (nf - (nf > 0 ? 1 : 0)) / 2;
            }
            continue;
        }
        const uint2 u = units[k];
        const int B = (int)u.x, pb = (int)u.y;
        const int cnt = (int)own_cnt[B], base = (int)own_off[B];
        const int fb = t.first[B], nb = t.count[B], sB = nslow ? nslow[B] : nb, lB = t.level[B];
        {
            const int np = min(kOwnUnit, cnt - pb);
            int fa = 0, na = 0, sa = 0;
            float4 off = make_float4(0.f, 0.f, 0.f, 0.f);
            bool near = false;
            if (lane < np) {
                const int A = partners[base + pb + lane];
                fa = t.first[A];
                na = t.count[A];
                sa = nslow ? nslow[A] : na;
                // z_A - z_B = delta * L / 2^(lf+1), exact in float; |delta| < 2^23 fits int32
                const int lA = t.level[A], lf = lA > lB ? lA : lB;
                const long long dl[3] = {centre_delta(t.cx[A], lA, t.cx[B], lB, lf),
                                         centre_delta(t.cy[A], lA, t.cy[B], lB, lf),
                                         centre_delta(t.cz[A], lA, t.cz[B], lB, lf)};
                const float unit = pow2f(log2L - lf - 1);
                off = make_float4((float)(int)dl[0] * unit, (float)(int)dl[1] * unit, (float)(int)dl[2] * unit, 0.f);
                if (KERNEL == TG_KERNEL_WENDLAND_C2) {
                    // cube gap below eps: some pair may fall inside the softening length
                    const long long ha = 1ll << (lf - lA), hb = 1ll << (lf - lB);
                    long long g2 = 0;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const long long gd = (dl[d] < 0 ? -dl[d] : dl[d]) - (ha + hb);
                        if (gd > 0) g2 += gd * gd;
                    }
                    const float eu = eps * pow2f(lf + 1 - log2L);   // eps in half-units of the finer level
                    near = !((float)g2 >= eu * eu * 1.0001f);
                }
                // pairs evaluated: all minus fast-fast
                my_pairs += (unsigned long long)na * nb - (unsigned long long)(na - sa) * (nb - sB);
            }
            const unsigned bn = __ballot_sync(0xffffffffu, lane < np && near);
            const unsigned bf = __ballot_sync(0xffffffffu, lane < np && !near);
            const int n_near = __popc(bn);
            const int slot = near ? __popc(bn & lt) : n_near + __popc(bf & lt);
            __syncwarp();
            if (lane < np) {
                ob->off[slot] = off;
                ob->first[slot] = fa;
                ob->nslow[slot] = sa;
                ob->inc[1][slot] = na;   // partner size, replaced by the fast-row scan below
            }
            __syncwarp();
            const int cS = lane < np ? ob->nslow[lane] : 0;
            const int cF = lane < np ? ob->inc[1][lane] - cS : 0;
            const int incS = warp_incl_scan(cS, lane), incF = warp_incl_scan(cF, lane);
            __syncwarp();
            ob->inc[0][lane] = incS;
            ob->inc[1][lane] = incF;
            const int Ts = __shfl_sync(0xffffffffu, incS, 31), Tf = __shfl_sync(0xffffffffu, incF, 31);
            const int nearS = n_near ? __shfl_sync(0xffffffffu, incS, n_near - 1) : 0;
            const int nearF = n_near ? __shfl_sync(0xffffffffu, incF, n_near - 1) : 0;
            // nothing to evaluate: no slow rows, and no slow column for the fast rows (kick pairs of the
            // lowest rungs, whose slow set is a few particles of the whole system)
            if (Ts == 0 && (Tf == 0 || sB == 0)) continue;
            for (int jc = 0; jc < nb; jc += kMaxNcrit) {
                const int nbc = min(kMaxNcrit, nb - jc);
                // columns in leaf order (slow first), padded to a multiple of 8 once; without slow rows only
                // the slow columns (for the fast rows) are staged and flushed
                const int nsc = max(0, min(sB - jc, nbc));   // slow columns of this chunk (slow-first leaf)
                const int ns8 = (nsc + 7) & ~7, nt8 = (nbc + 7) & ~7;
                const int nstage = Ts > 0 ? nt8 : ns8, nflush = Ts > 0 ? nbc : nsc;
                if (nstage == 0) continue;
                __syncwarp();
                for (int j = lane; j < nstage; j += 32) {
                    col_put(sq, j, j < nbc ? pf[fb + jc + j] : make_float4(-1e8f, -1e8f, -1e8f, 0.f));
                    sacc[j][0] = sacc[j][1] = sacc[j][2] = sacc[j][3] = 0.f;
                }
                __syncwarp();
                for (int i0 = 0; i0 < Ts; i0 += 32 * ROWS) {
                    if (i0 < nearS) owner_rows<KERNEL, ROWS, true, POT>(pf, ob, 0, i0, Ts, sq, sacc, nt8, nt8, eps, acc4, n, lane);
                    else owner_rows<KERNEL, ROWS, false, POT>(pf, ob, 0, i0, Ts, sq, sacc, nt8, nt8, eps, acc4, n, lane);
                }
                if (nsc > 0 && Tf > 0) {
                    // fast rows meet the slow columns only: the batch that holds the first fast columns runs
                    // with their masses at zero (no force on the rows) and their reaction sums dropped
                    __syncwarp();
                    for (int j = nsc + lane; j < ns8; j += 32) col_zero_mass(sq, j);
                    __syncwarp();
                    for (int i0 = 0; i0 < Tf; i0 += 32 * ROWS) {
                        if (i0 < nearF) owner_rows<KERNEL, ROWS, true, POT>(pf, ob, 1, i0, Tf, sq, sacc, ns8, nsc, eps, acc4, n, lane);
                        else owner_rows<KERNEL, ROWS, false, POT>(pf, ob, 1, i0, Tf, sq, sacc, ns8, nsc, eps, acc4, n, lane);
                    }
                }
                __syncwarp();
                for (int j = lane; j < nflush; j += 32)
#pragma unroll
                    for (int comp = 0; comp < (POT ? 4 : 3); ++comp)
                        atomicAdd(&acc4[(size_t)comp * n + fb + jc + j], f2d_exact(sacc[j][comp]));
            }
        }
    }
    my_pairs = warp_sum(my_pairs);
    if (lane == 0 && my_pairs) atomicAdd(pair_counter, my_pairs);
}

}  // namespace tg

namespace tg {

// Resident blocks per SM of the owner kernel, queried once per rows-per-lane setting (tg_autotune: 1,
// 2 or 3; rows are packed densely, so the chunk is full whatever the leaf size).
static int owner_occupancy(int rows)
{
    static int occ[4] = {0, 0, 0, 0};
    if (occ[rows] == 0) {
        cudaError_t e = cudaErrorInvalidValue;
        if (rows == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], p2p_owner_f32<TG_KERNEL_WENDLAND_C2, 1, false>, 256, 0);
        if (rows == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[2], p2p_owner_f32<TG_KERNEL_WENDLAND_C2, 2, false>, 256, 0);
        if (rows == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[3], p2p_owner_f32<TG_KERNEL_WENDLAND_C2, 3, false>, 256, 0);
        if (e != cudaSuccess || occ[rows] < 1) {
            cudaGetLastError();
            occ[rows] = 1;
        }
    }
    return occ[rows];
}

// zero n32[0] + extra words at p (n32: a device count, nullable; the batched path cannot size a memset)
__global__ void zero_u32_dev(uint32_t *p, const int *n32, int extra)
{
    const int n = (n32 ? *n32 : 0) + extra;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0u;
}

// Every P2P pair in float32, one launch: the distinct leaf pairs grouped by owner, then the self pairs.
// pot = false: accelerations only (the potential slot of acc4 is left out).
tg_status launch_p2p_f32(tg_ctx *c, const TreeView &t, const uint2 *pairs, int64_t npairs, const uint2 *self_pairs,
                         int64_t nself, const float4 *pf, const int32_t *nslow, bool pot, double *acc4)
{
    tg_status st;
    const int ncell = t.ncell;
    uint32_t *own_cnt, *own_fill, *own_off;
    uint2 *tagged, *units;
    int32_t *partners;
    if (npairs + nself == 0) return TG_OK;
    if (nself > 0xffffffffll) return set_err(c, TG_ERR_CAPACITY, "too many self pairs for one P2P launch");
    const int64_t max_units = npairs / kOwnUnit + ncell + 1;
    if ((st = ensure_t(c, B_OWN_CNT, (size_t)ncell + 2, &own_cnt)) || (st = ensure_t(c, B_OWN_FILL, ncell, &own_fill)) ||
        (st = ensure_t(c, B_OWN_OFF, ncell, &own_off)) || (st = ensure_t(c, B_OWN_LIST, max_units, &units)) ||
        (st = ensure_t(c, B_OWN_TAG, npairs, &tagged)) || (st = ensure_t(c, B_OWN_PART, npairs, &partners)))
        return st;
    uint32_t *ctr = own_cnt + ncell;   // [0] work units, [1] next unit to take
    cudaMemsetAsync(own_cnt, 0, sizeof(uint32_t) * ((size_t)ncell + 2), c->stream);
    cudaMemsetAsync(own_fill, 0, sizeof(uint32_t) * (size_t)ncell, c->stream);
    if (npairs > 0) {
        {
            ProfScope ps_(c, TG_K_OTHER);
            p2p_owner_count<<<grid_for(npairs, 256), 256, 0, c->stream>>>(pairs, npairs, t.count, own_cnt, tagged, nullptr);
        }
        if ((st = exclusive_scan_u32(c, own_cnt, own_off, ncell, nullptr))) return st;
        {
            ProfScope ps_(c, TG_K_OTHER);
            p2p_owner_fill<<<grid_for(npairs, 256), 256, 0, c->stream>>>(tagged, npairs, own_off, own_fill, partners,
                                                                         units, ctr, nullptr);
        }
    }
    const float eps = (float)c->prm.eps;
    unsigned long long *pc = c->d_counters;
    const bool plummer = c->prm.kernel == TG_KERNEL_PLUMMER;
    ProfScope ps_(c, TG_K_P2P);
    const int rows = c->tune.p2p_rows;
    const int grid = c->num_sms * owner_occupancy(rows);
#define TG_OWNER(K, R, PT)                                                                                        \
    p2p_owner_f32<K, R, PT><<<grid, 256, 0, c->stream>>>(t, c->walk_log2L, units, ctr, own_off, own_cnt, partners,  \
                                                         self_pairs, (uint32_t)nself, pf, nslow, eps, acc4, t.n, pc,    \
                                                         nullptr, nullptr, nullptr, 0ull)
#define TG_OWNER_ROWS(K, PT)                                                                                      \
    switch (rows) {                                                                                               \
    case 1: TG_OWNER(K, 1, PT); break;                                                                            \
    case 3: TG_OWNER(K, 3, PT); break;                                                                            \
    default: TG_OWNER(K, 2, PT);                                                                                  \
    }
    if (plummer) {
        if (pot) TG_OWNER_ROWS(TG_KERNEL_PLUMMER, true)
        else TG_OWNER_ROWS(TG_KERNEL_PLUMMER, false)
    } else {
        if (pot) TG_OWNER_ROWS(TG_KERNEL_WENDLAND_C2, true)
        else TG_OWNER_ROWS(TG_KERNEL_WENDLAND_C2, false)
    }
#undef TG_OWNER_ROWS
#undef TG_OWNER
    return cuda_check(c, cudaGetLastError(), "p2p owner launch");
}

// The same launch with every size on the device (batched HOLD step): the leaf-pair and self-pair counts
// come from the walk's counters, the cell count from de; buffers are sized for the capacities.
tg_status launch_p2p_f32_dev(tg_ctx *c, const TreeView &t, const DevEval *de, const Geom *gp,
                             const unsigned long long *walk_ctr, const uint2 *p2p, size_t cap_p2p, int cap_cells,
                             const float4 *pf, const int32_t *nslow, double *acc4, int stride, int scan_scratch)
{
    tg_status st;
    uint32_t *own_cnt, *own_fill, *own_off, *ctr;
    uint2 *tagged, *units;
    int32_t *partners;
    const int64_t max_units = (int64_t)cap_p2p / kOwnUnit + cap_cells + 1;
    if ((st = ensure_t(c, B_OWN_CNT, (size_t)cap_cells + 2, &own_cnt)) ||
        (st = ensure_t(c, B_OWN_FILL, (size_t)cap_cells + 2, &own_fill)) ||
        (st = ensure_t(c, B_OWN_OFF, (size_t)cap_cells, &own_off)) || (st = ensure_t(c, B_OWN_LIST, max_units, &units)) ||
        (st = ensure_t(c, B_OWN_TAG, cap_p2p, &tagged)) || (st = ensure_t(c, B_OWN_PART, cap_p2p, &partners)))
        return st;
    ctr = own_fill + cap_cells;   // [0] work units, [1] next unit to take
    const int g = c->num_sms * 4;
    {
        ProfScope ps_(c, TG_K_OTHER);
        zero_u32_dev<<<g, 256, 0, c->stream>>>(own_cnt, &de->ncell, 0);
        zero_u32_dev<<<g, 256, 0, c->stream>>>(own_fill, &de->ncell, 0);
        zero_u32_dev<<<1, 32, 0, c->stream>>>(ctr, nullptr, 2);
        p2p_owner_count<<<g, 256, 0, c->stream>>>(p2p, (int64_t)cap_p2p, t.count, own_cnt, tagged, walk_ctr + 2);
    }
    if ((st = exclusive_scan_u32(c, own_cnt, own_off, cap_cells, nullptr, &de->ncell, scan_scratch))) return st;
    {
        ProfScope ps_(c, TG_K_OTHER);
        p2p_owner_fill<<<g, 256, 0, c->stream>>>(tagged, (int64_t)cap_p2p, own_off, own_fill, partners, units, ctr,
                                                  walk_ctr + 2);
    }
    const float eps = (float)c->prm.eps;
    unsigned long long *pc = c->d_counters;
    const bool plummer = c->prm.kernel == TG_KERNEL_PLUMMER;
    ProfScope ps_(c, TG_K_P2P);
    const int rows = c->tune.p2p_rows;
    const int grid = c->num_sms * owner_occupancy(rows);
#define TG_OWNER_DEV(K, R)                                                                                        \
    p2p_owner_f32<K, R, false><<<grid, 256, 0, c->stream>>>(t, 0, units, ctr, own_off, own_cnt, partners, nullptr, 0u, \
                                                            pf, nslow, eps, acc4, stride, pc, gp, walk_ctr, p2p,    \
                                                            (unsigned long long)cap_p2p)
#define TG_OWNER_DEV_ROWS(K)                                                                                      \
    switch (rows) {                                                                                               \
    case 1: TG_OWNER_DEV(K, 1); break;                                                                            \
    case 3: TG_OWNER_DEV(K, 3); break;                                                                            \
    default: TG_OWNER_DEV(K, 2);                                                                                  \
    }
    if (plummer) TG_OWNER_DEV_ROWS(TG_KERNEL_PLUMMER)
    else TG_OWNER_DEV_ROWS(TG_KERNEL_WENDLAND_C2)
#undef TG_OWNER_DEV_ROWS
#undef TG_OWNER_DEV
    return cuda_check(c, cudaGetLastError(), "p2p owner launch (device sizes)");
}

}  // namespace tg
