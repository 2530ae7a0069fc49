// m2l_sym.cuh -- mutual cell-cell interaction (M2L, Sec. 2.1 of Zhu 2017).
//
// The walk hands over M2L work in blocks: the well-separated child pairs (x_i, y_j) of one opened
// cell pair (A, B), as an 8x8 bit mask.  Each unordered pair is evaluated once: the derivative
// tensor D^k(d), |k| <= p, is built once and BOTH local expansions are updated,
//   L_x^n += sum_j (-1)^|j|/j! M_y^j D^{n+j},   L_y^n += (-1)^|n| sum_j M_x^j/j! D^{n+j}
// (D^k(-d) = (-1)^|k| D^k(d)), so the net forces of the two cells on each other cancel.
//
// Expansions are normalised by cell size s (M~^j = M^j / s^|j|, L~^n = L^n s^(|n|+1)) and the
// offset is measured in units of the x cell, d' = (z_x - z_y)/s_x; with rho = s_y/s_x,
//   L~_x^n += sum_j (-1)^|j| rho^|j| M~_y^j/j! D^{n+j}(d'),
//   L~_y^n += (-1)^|n| rho^(|n|+1) sum_j M~_x^j/j! D^{n+j}(d'),
// with the softening length scaled the same way (Plummer).  All terms are O(1): no overflow or
// underflow in float32 however deep the tree.  D comes from the McMurchie-Davidson auxiliary
// recurrence R^(m)_{k+e_a} = d_a R^(m+1)_k + k_a R^(m+1)_{k-e_a}.
//
// Lane layout of one warp over a block: lane l -> (row of the round l/8, column j = l%8); a round
// covers four rows.  The x-side sums of one row are reduced over its 8 lanes, the y-side sums of one
// column over its 4 lanes, each lane then adding its slice of the coefficients to global memory.
#pragma once
#include "tg_common.cuh"
#include "tg_tables.cuh"
#include "m2l_geom.cuh"
#include "m2l_gen.cuh"

namespace tg {

// ------------------------------------------------------------------ float32, fixed order P <= 6
// Rounds take the block's non-empty rows four at a time (a block whose rows fit in four needs one
// round).  The 8 lanes of a row and the 4 lanes of a column combine their partial expansions with a
// reduce-scatter (coefficients padded to RL per row lane, CL per column lane), after which every
// lane adds its own slice to global memory: no lane holds the whole sum.
template <int NC_>
struct M2LScatter {
    static constexpr int NC = NC_;
    static constexpr int RL = (NC + 31) / 32 * 4;   // coefficients per lane after the row reduction
    static constexpr int CL = (NC + 15) / 16 * 4;   // ... after the column reduction
    static constexpr int NP = 8 * RL > 4 * CL ? 8 * RL : 4 * CL;
};

// The two contraction sets of the block kernel.  Full: every coefficient |k| <= P, any G (the
// softened one included).  Harmonic (G = -1/|d| only): moments folded to j_z <= 1 per cell, locals
// formed for n_z <= 1 and completed per cell, D for k_z <= 2 (see gen_m2l.py); same result in exact
// arithmetic, (P+1)^2 instead of (P+1)(P+2)(P+3)/6 coefficients per side.
template <int P>
struct M2LFull : M2LGen<P> {
    static constexpr int ND = M2LGen<P>::NC;
    static constexpr bool HARMONIC = false;
    static __device__ __forceinline__ void dt(float dx, float dy, float dz, float soft2, float (&D)[ND])
    {
        M2LGen<P>::dtensor(dx, dy, dz, soft2, D);
    }
};
template <int P>
struct M2LHarm : M2LGenH<P> {
    static constexpr int ND = M2LGenH<P>::ND;
    static constexpr bool HARMONIC = true;
    static __device__ __forceinline__ void dt(float dx, float dy, float dz, float, float (&D)[ND])
    {
        M2LGenH<P>::dtensor(dx, dy, dz, D);
    }
};

// first index of total degree o in a coefficient list (both lists are ordered by total degree)
__host__ __device__ constexpr int first_of_order(bool harmonic, int o)
{
    return harmonic ? o * o : o * (o + 1) * (o + 2) / 6;
}
__host__ __device__ constexpr int order_in(bool harmonic, int k)
{
    int o = 0;
    while (first_of_order(harmonic, o + 1) <= k) ++o;
    return o;
}

// per cell and class: fold the moments onto j_z <= 1 (pads zeroed)
template <int P>
__global__ void m2l_reduce_moments_h(int64_t nrows, const float *__restrict__ Ms, int ncp, float *__restrict__ Mr, int ncpr,
                                     const int *drows)
{
    if (drows) nrows = *drows;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nrows; w += (int64_t)gridDim.x * blockDim.x) {
        M2LGenH<P>::reduce_moments(Ms + w * ncp, Mr + w * ncpr);
        for (int k = M2LGenH<P>::NC; k < ncpr; ++k) Mr[w * ncpr + k] = 0.f;
    }
}

// per cell and class: the full local expansion from its n_z <= 1 coefficients (pads zeroed)
template <int P>
__global__ void m2l_complete_locals_h(int64_t nrows, const float *__restrict__ Lr, int ncpr, float *__restrict__ L, int ncp,
                                      const int *drows)
{
    if (drows) nrows = *drows;
    constexpr int NC = M2LGen<P>::NC;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nrows; w += (int64_t)gridDim.x * blockDim.x) {
        M2LGenH<P>::complete_locals(Lr + w * ncpr, L + w * ncp);
        for (int k = NC; k < ncp; ++k) L[w * ncp + k] = 0.f;
    }
}

// halve the live coefficients once: lanes with bit d keep the upper half, the others the lower half
template <int NP, int H>
__device__ __forceinline__ void m2l_halve(float (&v)[NP], int lane, int d)
{
    const bool hi = (lane & d) != 0;
#pragma unroll
    for (int q = 0; q < H; ++q) {
        const float send = hi ? v[q] : v[q + H];
        const float keep = hi ? v[q + H] : v[q];
        v[q] = keep + __shfl_xor_sync(0xffffffffu, send, d);
    }
}

// Blocks whose well-separated pairs lie in one row (a leaf facing the children of an opened cell, about
// half of all blocks on clustered inputs) would fill 8 of the 32 lanes of a round.  m2l_partition puts
// them at the end of the block list (a block whose pairs lie in one column is transposed first), and the
// kernel takes them four at a time: row slot rr of a packed round holds its own block's row.  The row
// (x side) reduction stays within the 8 lanes of a row; the column (y side) sums of different blocks
// cannot be combined, so in a packed round every active lane adds its whole y-side expansion.
// part: the partitioned blocks, multi-row ones at [0, pcnt[0]) and one-row ones at [cap - pcnt[1], cap).
static __global__ void m2l_partition(const M2LBlock *__restrict__ in, int64_t nb, const unsigned long long *dnb,
                              M2LBlock *part, int64_t cap, unsigned long long *pcnt)
{
    if (dnb) nb = (int64_t)*dnb;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps iterate together: slots are reserved per warp
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x; w0 < nb; w0 += stride) {
        const int64_t w = w0 + threadIdx.x;
        M2LBlock blk{0u, 0u, 0ull};
        bool single = false;
        if (w < nb) {
            blk = in[w];
            unsigned rows = 0u, cols = 0u;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const unsigned r = (unsigned)((blk.mask >> (8 * i)) & 0xffull);
                if (r) rows |= 1u << i;
                cols |= r;
            }
            if (__popc(rows) == 1) {
                single = true;
            } else if (__popc(cols) == 1) {
                // all pairs in column j0: the transposed block (b, a) has them in row j0
                const int j0 = __ffs(cols) - 1;
                unsigned long long t = 0ull;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if ((blk.mask >> (8 * i + j0)) & 1ull) t |= 1ull << (8 * j0 + i);
                blk = M2LBlock{blk.b, blk.a, t};
                single = true;
            }
        }
        const bool valid = w < nb;
        const unsigned bm = __ballot_sync(0xffffffffu, valid && !single);
        const unsigned bs = __ballot_sync(0xffffffffu, valid && single);
        unsigned long long base_m = 0ull, base_s = 0ull;
        if (lane == 0) {
            if (bm) base_m = atomicAdd(&pcnt[0], (unsigned long long)__popc(bm));
            if (bs) base_s = atomicAdd(&pcnt[1], (unsigned long long)__popc(bs));
        }
        base_m = __shfl_sync(0xffffffffu, base_m, 0);
        base_s = __shfl_sync(0xffffffffu, base_s, 0);
        const unsigned lt = (1u << lane) - 1u;
        if (valid && !single) part[base_m + __popc(bm & lt)] = blk;
        if (valid && single) part[cap - 1 - (int64_t)(base_s + __popc(bs & lt))] = blk;
    }
}

// POT = false: accelerations only, L^0 is left at zero (see the generated *_forces contractions).
// G: M2LFull<P> or M2LHarm<P>; Ms and L hold that set's coefficients with row stride ncp.
// Work items: the pcnt[0] multi-row blocks of part (rounds of four rows), then the pcnt[1] one-row
// blocks at the end of part, four per packed round (see m2l_partition).
// Batched path (de non-null): the class count and the root cube come from the device; the launch for
// the other class count returns at once.
// Kick pairs (MASKED) with fpre (the prefix sum of the fast flags over the sorted particles): a target
// cell needs the all-sources local (class 0) only if it holds slow particles, and the slow-sources local
// (class 1) only if it holds fast particles, and a class-1 contraction adds something only if its source
// holds slow particles (class 1 carries the slow masses); a round skips a side's contraction of a class
// when no pair of the round needs it (a warp vote, so the warp stays converged).  The skipped locals are
// read by no particle (L2L hands them only to descendants, which hold no particle of that class either),
// and the skipped class-1 terms are zero.
template <class G, bool MASKED, bool POT>
__global__ void __launch_bounds__(128) m2l_blocks_f32(TreeView t, const M2LBlock *__restrict__ part, int64_t cap,
                                                      const unsigned long long *__restrict__ pcnt,
                                                      const float *__restrict__ Ms, float *L, int ncp, float eps_over_L,
                                                      int plummer, const DevEval *de, const Geom *gp, double eps,
                                                      const uint32_t *__restrict__ fpre, unsigned long long *class_ctr)
{
    unsigned long long my_sc = 0;   // side contractions the method needs: (pair side, class) with a target
    if (de) {
        if ((de->masked != 0) != MASKED) return;
        if (plummer) eps_over_L = (float)ldexp(eps, -gp->log2L);
    }
    using S = M2LScatter<G::NC>;
    constexpr int NC = S::NC, RL = S::RL, CL = S::CL, NP = S::NP, ND = G::ND;
    const int lane = threadIdx.x & 31;
    const int j = lane & 7, rr = (lane >> 3) & 3;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_multi = (int64_t)pcnt[0], n_single = (int64_t)pcnt[1];
    const int64_t n_items = n_multi + (n_single + 3) / 4;
    for (int64_t w = wid; w < n_items; w += nw) {
        const bool packed = w >= n_multi;   // warp-uniform
        M2LBlock blk{0u, 0u, 0ull};
        if (!packed) {
            blk = part[w];
        } else {
            const int64_t s = (w - n_multi) * 4 + rr;
            if (s < n_single) blk = part[cap - 1 - s];
        }
        const BlockGeom bg = block_geom(t, blk);
        const float rho = ldexpf(1.0f, bg.lx - bg.ly);
        const float soft = plummer ? ldexpf(eps_over_L, bg.lx) : 0.0f;   // eps / s_x
        const float soft2 = soft * soft;
        unsigned rowmask = 0;   // rows holding at least one well-separated pair
#pragma unroll
        for (int i = 0; i < 8; ++i)
            if (((blk.mask >> (8 * i)) & 0xffull) != 0ull) rowmask |= 1u << i;
        const int nrows = packed ? 1 : __popc(rowmask);
        for (int r0 = 0; r0 < nrows; r0 += 4) {
            // this lane's row: the (r0 + rr)-th non-empty row of the block (packed: its block's one row)
            int i = -1;
            {
                const int want = packed ? 0 : r0 + rr;
#pragma unroll
                for (int b = 0; b < 8; ++b)
                    if (((rowmask >> b) & 1u) && __popc(rowmask & ((1u << b) - 1u)) == want) i = b;
            }
            const bool active = i >= 0 && j < bg.nj && ((blk.mask >> (8 * i + j)) & 1ull);
            const unsigned amask = __ballot_sync(0xffffffffu, active);
            // x, y: this lane's row and column cells (every lane of a used row / column flushes a slice);
            // inactive lanes run the contractions on a zero tensor and an existing cell's moments
            const int x = bg.baseA + (i < 0 ? 0 : i), y = bg.baseB + j;
            const int xs = active ? x : bg.baseA, ys = active ? y : bg.baseB;
            float D[ND];
            if (active) {
                float dx, dy, dz;
                pair_offset<float>(t, x, y, bg.lx, bg.ly, dx, dy, dz);
                G::dt(dx, dy, dz, soft2, D);
            } else {
#pragma unroll
                for (int k = 0; k < ND; ++k) D[k] = 0.f;
            }
            const bool row_used = ((amask >> (lane & ~7)) & 0xffu) != 0u;   // this lane's row, this round
            // this lane's column, this round (packed: the lane's own pair, its block has one row)
            const bool col_used = packed ? active : (amask & (0x01010101u << j)) != 0u;
            // classes the round's targets need (side a: the row cells, side b: the column cells).  Class 1
            // holds the slow masses only: a source without slow particles has zero class-1 moments, so
            // its class-1 contraction adds nothing and is left out with the others of the round.
            unsigned need = 0xfu;   // bit cls: side a needs class cls; bit 2 + cls: side b does
            if (MASKED && fpre) {
                int fx = 0, sx = 0, fy = 0, sy = 0;
                if (active) {
                    const int ax = t.first[x], ay = t.first[y];
                    fx = (int)(fpre[ax + t.count[x]] - fpre[ax]);
                    sx = t.count[x] - fx;
                    fy = (int)(fpre[ay + t.count[y]] - fpre[ay]);
                    sy = t.count[y] - fy;
                }
                const bool a1 = fx > 0 && sy > 0, b1 = fy > 0 && sx > 0;
                need = (__any_sync(0xffffffffu, sx > 0) ? 1u : 0u) | (__any_sync(0xffffffffu, a1) ? 2u : 0u) |
                       (__any_sync(0xffffffffu, sy > 0) ? 4u : 0u) | (__any_sync(0xffffffffu, b1) ? 8u : 0u);
                my_sc += (unsigned)(sx > 0) + (unsigned)a1 + (unsigned)(sy > 0) + (unsigned)b1;
            } else if (active) {
                my_sc += MASKED ? 4u : 2u;
            }
            // One contraction in the code for both sides and both classes (the generated code is large; the
            // warps of an SM fetch one copy instead of four).  Side 0 is the row cell x with sources y:
            // L~_x^n = sum_j (-1)^|j| rho^|j| M~_y^j D^{n+j}.  Side 1 is the column cell y with sources x,
            // the same contraction with rho = -1: sum_j M~_x^j D^{n+j}, which is (-1)^|n| times L~_y^n
            // in the x normalisation; the flush applies (-1)^|n| rho^(|n|+1).
#pragma unroll 1
            for (int it = 0; it < (MASKED ? 4 : 2); ++it) {
                const int cls = it >> 1, side = it & 1;
                if (!(need & ((side ? 4u : 1u) << cls))) continue;
                float Lc[NP];
#pragma unroll
                for (int k = NC; k < NP; ++k) Lc[k] = 0.f;
                const float *src = Ms + ((size_t)(side ? xs : ys) * 2 + cls) * ncp;
                if (POT) G::side_a(D, src, side ? -1.0f : rho, reinterpret_cast<float(&)[NC]>(Lc));
                else G::side_a_forces(D, src, side ? -1.0f : rho, reinterpret_cast<float(&)[NC]>(Lc));
                if (side == 0) {
                    // reduce-scatter over the row's lanes (bits 2, 1, 0): lane j keeps RL*j .. RL*j + RL - 1
                    m2l_halve<NP, 4 * RL>(Lc, lane, 4);
                    m2l_halve<NP, 2 * RL>(Lc, lane, 2);
                    m2l_halve<NP, RL>(Lc, lane, 1);
                    if (row_used) {
                        float *dst = L + ((size_t)x * 2 + cls) * ncp;
#pragma unroll
                        for (int g = 0; g < RL; g += 4) {
                            const int k = RL * j + g;
                            if (k < NC) atomicAdd(reinterpret_cast<float4 *>(dst + k), make_float4(Lc[g], Lc[g + 1], Lc[g + 2], Lc[g + 3]));
                        }
                    }
                    continue;
                }
                float *dst = L + ((size_t)y * 2 + cls) * ncp;
                if (!packed) {
                    // block rounds: reduce-scatter over the column's lanes (bits 4, 3): lane (rr, j) keeps
                    // coefficients CL*rr .. CL*rr + CL - 1 of column j
                    m2l_halve<NP, 2 * CL>(Lc, lane, 16);
                    m2l_halve<NP, CL>(Lc, lane, 8);
                    if (col_used) {
                        const int k0 = CL * rr;
                        int o = order_in(G::HARMONIC, k0);
                        int next = first_of_order(G::HARMONIC, o + 1);
                        float sc = ldexpf((o & 1) ? -1.0f : 1.0f, (bg.lx - bg.ly) * (o + 1));
                        const float nrho = -rho;
#pragma unroll
                        for (int g = 0; g < CL; g += 4) {
                            float v[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int k = k0 + g + q;
                                if (k == next) {
                                    ++o;
                                    next = first_of_order(G::HARMONIC, o + 1);
                                    sc *= nrho;
                                }
                                v[q] = Lc[g + q] * sc;
                            }
                            if (k0 + g < NC) atomicAdd(reinterpret_cast<float4 *>(dst + k0 + g), make_float4(v[0], v[1], v[2], v[3]));
                        }
                    }
                } else if (col_used) {
                    // packed rounds: each lane's whole expansion (its column belongs to its own block)
                    float sc = rho;   // order 0: rho^1
                    const float nrho = -rho;
#pragma unroll
                    for (int g = 0; g < NC; g += 4) {
                        float v[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (g + q > 0 && order_in(G::HARMONIC, g + q) != order_in(G::HARMONIC, g + q - 1)) sc *= nrho;
                            v[q] = Lc[g + q] * sc;
                        }
                        atomicAdd(reinterpret_cast<float4 *>(dst + g), make_float4(v[0], v[1], v[2], v[3]));
                    }
                }
            }
        }
    }
    my_sc = warp_sum(my_sc);
    if (class_ctr && (threadIdx.x & 31) == 0 && my_sc) atomicAdd(class_ctr, my_sc);
}

// ------------------------------------------------------------------ directed, by target cell (harmonic set)
// The walk's blocks hold each well-separated cell pair once.  The directed form lists, for every cell,
// the cells it receives from (both members of each pair), and a warp takes one target: lanes stride
// over its sources, each adds its sources' contributions to the target's reduced locals in registers
// (m2l_acc_h), and one warp reduction per target writes them.  The derivative tensor is computed once
// per direction instead of once per pair, but no pair needs a reduction across lanes or an atomic.

// per block: sources gained by each row cell (its row's bits) and each column cell (its column's bits)
static __global__ void m2l_list_count(TreeView t, const M2LBlock *__restrict__ blocks, int64_t nblocks, uint32_t *cnt,
                               const unsigned long long *dnb)
{
    if (dnb) nblocks = (int64_t)*dnb;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nblocks; w += (int64_t)gridDim.x * blockDim.x) {
        const M2LBlock blk = blocks[w];
        const BlockGeom bg = block_geom(t, blk);
        unsigned long long colbits = 0ull;   // bit 8j + i: the transposed mask
        for (int i = 0; i < 8; ++i) {
            const unsigned row = (unsigned)((blk.mask >> (8 * i)) & 0xffull);
            if (row) atomicAdd(&cnt[bg.baseA + i], (uint32_t)__popc(row));
            for (unsigned r = row; r; r &= r - 1) colbits |= 1ull << (8 * (__ffs(r) - 1) + i);
        }
        for (int j = 0; j < 8; ++j) {
            const unsigned col = (unsigned)((colbits >> (8 * j)) & 0xffull);
            if (col) atomicAdd(&cnt[bg.baseB + j], (uint32_t)__popc(col));
        }
    }
}

// sources of each cell at off[cell] + fill[cell]; entries past `cap` are dropped (capacity overflow is
// detected by the caller from the total)
static __global__ void m2l_list_fill(TreeView t, const M2LBlock *__restrict__ blocks, int64_t nblocks,
                              const uint32_t *__restrict__ off, uint32_t *fill, uint32_t *src, uint64_t cap,
                              const unsigned long long *dnb)
{
    if (dnb) nblocks = (int64_t)*dnb;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nblocks; w += (int64_t)gridDim.x * blockDim.x) {
        const M2LBlock blk = blocks[w];
        const BlockGeom bg = block_geom(t, blk);
        unsigned long long colbits = 0ull;
        for (int i = 0; i < 8; ++i) {
            const unsigned row = (unsigned)((blk.mask >> (8 * i)) & 0xffull);
            if (!row) continue;
            const int x = bg.baseA + i;
            uint64_t at = (uint64_t)off[x] + atomicAdd(&fill[x], (uint32_t)__popc(row));
            for (unsigned r = row; r; r &= r - 1) {
                const int j = __ffs(r) - 1;
                if (at < cap) src[at] = (uint32_t)(bg.baseB + j);
                ++at;
                colbits |= 1ull << (8 * j + i);
            }
        }
        for (int j = 0; j < 8; ++j) {
            const unsigned col = (unsigned)((colbits >> (8 * j)) & 0xffull);
            if (!col) continue;
            const int y = bg.baseB + j;
            uint64_t at = (uint64_t)off[y] + atomicAdd(&fill[y], (uint32_t)__popc(col));
            for (unsigned r = col; r; r &= r - 1) {
                if (at < cap) src[at] = (uint32_t)(bg.baseA + __ffs(r) - 1);
                ++at;
            }
        }
    }
}

// sum of v over the warp, scattered: afterwards lane l holds coefficients 2l and 2l + 1 (NP = 64)
template <int NP>
__device__ __forceinline__ void warp_reduce_scatter64(float (&v)[NP], int lane)
{
    static_assert(NP == 64, "64 coefficients: two per lane");
    m2l_halve<NP, 32>(v, lane, 16);
    m2l_halve<NP, 16>(v, lane, 8);
    m2l_halve<NP, 8>(v, lane, 4);
    m2l_halve<NP, 4>(v, lane, 2);
    m2l_halve<NP, 2>(v, lane, 1);
}

template <int P, bool MASKED, bool POT>
__global__ void __launch_bounds__(128) m2l_directed_h(TreeView t, const uint32_t *__restrict__ off,
                                                      const uint32_t *__restrict__ cnt,
                                                      const uint32_t *__restrict__ src, uint64_t cap,
                                                      const float *__restrict__ Mr, float *__restrict__ Lr, int ncpr,
                                                      const DevEval *de, unsigned long long *class_ctr)
{
    using G = M2LGenH<P>;
    unsigned long long my_sc = 0;
    constexpr int NC = G::NC, ND = G::ND, NP = 64;
    static_assert(NC <= NP, "reduced set fits in two coefficients per lane");
    if (de && (de->masked != 0) != MASKED) return;
    const int ncell = t.cells();
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int x = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); x < ncell; x += nw) {
        const uint32_t b = off[x], e = (uint32_t)min((uint64_t)off[x] + cnt[x], cap);
        if (b >= e) continue;   // whole warp
        if (lane == 0) my_sc += (unsigned long long)(e - b) * (MASKED ? 2u : 1u);
        const int lx = t.level[x];
        float a0[NP], a1[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) a0[k] = a1[k] = 0.f;
        for (uint32_t q = b + lane; q < e; q += 32) {
            const int y = (int)src[q];
            const int ly = t.level[y];
            float dx, dy, dz;
            pair_offset<float>(t, x, y, lx, ly, dx, dy, dz);
            float D[ND];
            G::dtensor(dx, dy, dz, D);
            const float rho = ldexpf(1.0f, lx - ly);
            if (POT) G::acc(D, Mr + (size_t)y * 2 * ncpr, rho, reinterpret_cast<float(&)[NC]>(a0));
            else G::acc_forces(D, Mr + (size_t)y * 2 * ncpr, rho, reinterpret_cast<float(&)[NC]>(a0));
            if (MASKED) {
                if (POT) G::acc(D, Mr + ((size_t)y * 2 + 1) * ncpr, rho, reinterpret_cast<float(&)[NC]>(a1));
                else G::acc_forces(D, Mr + ((size_t)y * 2 + 1) * ncpr, rho, reinterpret_cast<float(&)[NC]>(a1));
            }
        }
        warp_reduce_scatter64<NP>(a0, lane);
        float *dst = Lr + (size_t)x * 2 * ncpr;
        if (2 * lane < NC) dst[2 * lane] = a0[0];
        if (2 * lane + 1 < NC) dst[2 * lane + 1] = a0[1];
        if (MASKED) {
            warp_reduce_scatter64<NP>(a1, lane);
            if (2 * lane < NC) dst[ncpr + 2 * lane] = a1[0];
            if (2 * lane + 1 < NC) dst[ncpr + 2 * lane + 1] = a1[1];
        }
    }
    if (class_ctr && lane == 0 && my_sc) atomicAdd(class_ctr, my_sc);
}

// ------------------------------------------------------------------ generic (p <= 8, float or double)
// Same block layout; each active lane evaluates its pair with run-time loops and adds both sides
// directly to global memory.  Used by the float64 path and by float32 for p > 6.
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
__global__ void m2l_blocks_generic(TreeView t, const M2LBlock *__restrict__ blocks, int64_t nblocks,
                                   const T *__restrict__ Ms, T *L, int p, int nc, int ncp, double eps_over_L,
                                   int plummer, const unsigned long long *dnb = nullptr, const DevEval *de = nullptr,
                                   const Geom *gp = nullptr, double eps = 0.0)
{
    if (dnb) {   // batched path: counts, classes and root cube on the device
        if ((de->masked != 0) != MASKED) return;
        nblocks = (int64_t)*dnb;
        if (plummer) eps_over_L = ldexp(eps, -gp->log2L);
    }
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = wid; w < nblocks; w += nw) {
        const M2LBlock blk = blocks[w];
        const BlockGeom bg = block_geom(t, blk);
        const T rho = (T)ldexp(1.0, bg.lx - bg.ly);
        const T soft = plummer ? (T)ldexp(eps_over_L, bg.lx) : T(0);
        for (int r = 0; r < 2; ++r) {
            const int i = 4 * r + (lane >> 3), j = lane & 7;
            const bool active = i < bg.ni && j < bg.nj && ((blk.mask >> (8 * i + j)) & 1ull);
            if (!active) continue;
            const int x = bg.baseA + i, y = bg.baseB + j;
            T dx, dy, dz;
            pair_offset<T>(t, x, y, bg.lx, bg.ly, dx, dy, dz);
            T D[TG_NCOEF_MAX];
            dtensor_generic<T>(p, dx, dy, dz, soft * soft, D);
            for (int cls = 0; cls < (MASKED ? 2 : 1); ++cls) {
                const T *My = Ms + ((size_t)y * 2 + cls) * ncp, *Mx = Ms + ((size_t)x * 2 + cls) * ncp;
                T *Lx = L + ((size_t)x * 2 + cls) * ncp, *Ly = L + ((size_t)y * 2 + cls) * ncp;
                for (int n = 0; n < nc; ++n) {
                    const int nx = c_mi_x[n], ny = c_mi_y[n], nz = c_mi_z[n], on = c_mi_order[n];
                    const int ncj = ncoef_dev(p - on);
                    T sa = 0, sb = 0, rpj = 1;
                    int oprev = 0;
                    for (int jj = 0; jj < ncj; ++jj) {
                        const int oj = c_mi_order[jj];
                        if (oj != oprev) {
                            rpj *= rho;
                            oprev = oj;
                        }
                        const T Dv = D[c_mi_lookup[((nx + c_mi_x[jj]) * 9 + ny + c_mi_y[jj]) * 9 + nz + c_mi_z[jj]]];
                        sa += ((oj & 1) ? -rpj : rpj) * My[jj] * Dv;
                        sb += Mx[jj] * Dv;
                    }
                    T rpn = rho;
                    for (int o = 0; o < on; ++o) rpn *= rho;
                    atomicAdd(&Lx[n], sa);
                    atomicAdd(&Ly[n], ((on & 1) ? -rpn : rpn) * sb);
                }
            }
        }
    }
}

}  // namespace tg
