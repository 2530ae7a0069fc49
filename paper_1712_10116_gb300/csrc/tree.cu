// tree.cu -- root cube, Morton keys, stable LSD radix sort, gather and level-synchronous
// octree build (Sec. 2.3 of Zhu 2017: octree with leaf size n_crit, built for every call).
//
// Keys: 21 bits per axis, x the most significant bit of each 3-bit group, so a cell at level l
// is the run of sorted keys sharing the top 3l bits.  The sort orders (key, input index), so ties
// keep input order.  Cells are emitted level by level in Morton order of their key prefix.
#include <cstdarg>
#include <cstring>

#include "tg_common.cuh"

namespace tg {

// ------------------------------------------------------------------ errors and buffers
tg_status set_err(tg_ctx *c, tg_status code, const char *fmt, ...)
{
    if (c->err.code == TG_OK) {
        char msg[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(msg, sizeof msg, fmt, ap);
        va_end(ap);
        c->err.code = code;
        c->err.msg = msg;
    }
    return code;
}

cudaError_t stream_sync(tg_ctx *c)
{
    c->stats.host_syncs += 1;
    return cudaStreamSynchronize(c->stream);
}

tg_status cuda_check(tg_ctx *c, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return TG_OK;
    return set_err(c, e == cudaErrorMemoryAllocation ? TG_ERR_OOM : TG_ERR_CUDA, "%s: %s", what,
                   cudaGetErrorString(e));
}

tg_status injected_alloc_failure(tg_ctx *c, size_t bytes, int slot)
{
    if (c->debug_fail_alloc_after < 0) return TG_OK;
    if (c->debug_fail_alloc_after == 0)
        return set_err(c, TG_ERR_OOM, "allocation of %zu bytes for scratch slot %d failed (injected)", bytes, slot);
    c->debug_fail_alloc_after -= 1;
    return TG_OK;
}

tg_status ensure(tg_ctx *c, int slot, size_t bytes, void **out)
{
    Buf &b = c->buf[slot];
    if (b.bytes < bytes) {
        size_t nb = bytes + bytes / 4 + 256;
        if (c->capturing)
            return set_err(c, TG_ERR_CAPACITY, "scratch slot %d would grow to %zu bytes inside a graph capture", slot, nb);
        if (tg_status inj = injected_alloc_failure(c, nb, slot)) return inj;
        c->alloc_epoch += 1;
        if (b.p) {
            cudaError_t e = stream_sync(c);
            if (e != cudaSuccess) return cuda_check(c, e, "sync before regrow");
            cudaFree(b.p);
            b.p = nullptr;
            b.bytes = 0;
        }
        cudaError_t e = cudaMalloc(&b.p, nb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_err(c, TG_ERR_OOM, "cudaMalloc(%zu) for scratch slot %d failed", nb, slot);
        }
        b.bytes = nb;
    }
    *out = b.p;
    return TG_OK;
}

// grow keeping the first `keep` bytes
static tg_status ensure_keep(tg_ctx *c, int slot, size_t bytes, size_t keep, void **out)
{
    Buf &b = c->buf[slot];
    if (b.bytes >= bytes) {
        *out = b.p;
        return TG_OK;
    }
    size_t nb = bytes + bytes / 2 + 256;
    if (c->capturing)
        return set_err(c, TG_ERR_CAPACITY, "scratch slot %d would grow to %zu bytes inside a graph capture", slot, nb);
    if (tg_status inj = injected_alloc_failure(c, nb, slot)) return inj;
    c->alloc_epoch += 1;
    void *np = nullptr;
    cudaError_t e = cudaMalloc(&np, nb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, TG_ERR_OOM, "cudaMalloc(%zu) for scratch slot %d failed", nb, slot);
    }
    if (b.p) {
        if (keep) cudaMemcpyAsync(np, b.p, keep, cudaMemcpyDeviceToDevice, c->stream);
        e = stream_sync(c);
        if (e != cudaSuccess) return cuda_check(c, e, "sync before regrow");
        cudaFree(b.p);
    }
    b.p = np;
    b.bytes = nb;
    *out = np;
    return TG_OK;
}

template <class T>
static tg_status ensure_keep_t(tg_ctx *c, int slot, size_t count, size_t keep_count, T **out)
{
    void *p = nullptr;
    tg_status s = ensure_keep(c, slot, count * sizeof(T) + 16, keep_count * sizeof(T), &p);
    *out = static_cast<T *>(p);
    return s;
}

// ------------------------------------------------------------------ live kernel timing
ProfScope::ProfScope(tg_ctx *ctx, int k) : c(ctx), cls(k), timed(false)
{
    c->prof_launches[k] += 1;
    if (c->prof_level >= 2 || (c->prof_level == 1 && (k == TG_K_M2L || k == TG_K_P2P))) {
        if (c->prof_used >= 2048) prof_collect(c);
        while (c->prof_events.size() < 2 * (c->prof_used + 1)) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                return;
            }
            c->prof_events.push_back(e);
        }
        if (c->prof_class.size() < c->prof_used + 1) c->prof_class.resize(c->prof_used + 1);
        c->prof_class[c->prof_used] = k;
        cudaEventRecord(c->prof_events[2 * c->prof_used], c->stream);
        timed = true;
    }
}

ProfScope::~ProfScope()
{
    if (!timed) return;
    cudaEventRecord(c->prof_events[2 * c->prof_used + 1], c->stream);
    c->prof_used += 1;
}

tg_status prof_collect(tg_ctx *c)
{
    if (c->prof_used == 0) return TG_OK;
    cudaError_t e = stream_sync(c);
    if (e != cudaSuccess) return cuda_check(c, e, "profile collect");
    for (size_t i = 0; i < c->prof_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->prof_events[2 * i], c->prof_events[2 * i + 1]) == cudaSuccess)
            c->prof_ms[c->prof_class[i]] += ms;
        else
            cudaGetLastError();
    }
    c->prof_used = 0;
    return TG_OK;
}

// ------------------------------------------------------------------ exclusive scan (uint32)
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
static_assert(kScanTile == kScanTileItems, "scan tile shared with the allocation-free sort");

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t warp_tot[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t t = lane < nw ? warp_tot[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;   // inclusive
    }
    __syncthreads();
    uint32_t base = warp > 0 ? warp_tot[warp - 1] : 0u;
    *total = warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void scan_tiles(const uint32_t *in, uint32_t *out, uint32_t *tile_sums, int n, const int *dn)
{
    n = dev_or(dn, n);
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0u;
        s += v[i];
    }
    uint32_t tot;
    uint32_t pre = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = pre;
        pre += v[i];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void scan_add(uint32_t *out, const uint32_t *tile_pre, int n, const int *dn)
{
    n = dev_or(dn, n);
    const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    const uint32_t add = tile_pre[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) out[base + i] += add;
}

size_t scan_scratch_words(int n)
{
    size_t need = 4;
    for (int m = n;;) {
        const int nt = (m + kScanTile - 1) / kScanTile;
        need += 2 * (size_t)nt + 2;
        if (nt == 1) break;
        m = nt;
    }
    return need;
}

// Exclusive scan of n uint32 values (out may alias in), with its scratch in slot `scratch` (a scan on
// another stream at the same time takes another slot).  The total is written to d_total (device word)
// when it is not null.  Recursive over tile sums.  With dn (a device count) the first
// level scans dn[0] <= n values; the launches are sized for n, and the tiles past dn[0] hand up
// zero sums, so the upper levels need no device count.
tg_status exclusive_scan_u32(tg_ctx *c, const uint32_t *in, uint32_t *out, int n, uint32_t *d_total, const int *dn,
                             int scratch)
{
    if (n <= 0) {
        if (d_total) cudaMemsetAsync(d_total, 0, sizeof(uint32_t), c->stream);
        return cuda_check(c, cudaGetLastError(), "exclusive scan");
    }
    uint32_t *tmp = nullptr;
    tg_status st = ensure_t(c, scratch, scan_scratch_words(n), &tmp);
    if (st) return st;
    struct Level { uint32_t *out; int n, ntiles; uint32_t *sums, *pre; };
    Level lv[8];
    int depth = 0;
    const uint32_t *cin = in;
    uint32_t *cout = out;
    int cn = n;
    uint32_t *cursor = tmp;
    while (true) {
        int nt = (cn + kScanTile - 1) / kScanTile;
        lv[depth] = {cout, cn, nt, cursor, cursor + nt};
        {
            ProfScope ps_(c, TG_K_OTHER);
            scan_tiles<<<nt, kScanThreads, 0, c->stream>>>(cin, cout, cursor, cn, depth == 0 ? dn : nullptr);
        }
        ++depth;
        if (nt == 1) break;
        cin = cursor;
        cout = cursor + nt;
        cn = nt;
        cursor += 2 * nt + 2;
    }
    for (int d = depth - 2; d >= 0; --d)
        {
            ProfScope ps_(c, TG_K_OTHER);
            scan_add<<<lv[d].ntiles, kScanThreads, 0, c->stream>>>(lv[d].out, lv[d].pre, lv[d].n, d == 0 ? dn : nullptr);
        }
    if (d_total)
        cudaMemcpyAsync(d_total, lv[depth - 1].sums, sizeof(uint32_t), cudaMemcpyDeviceToDevice, c->stream);
    return cuda_check(c, cudaGetLastError(), "exclusive scan");
}

// ------------------------------------------------------------------ root cube
constexpr int kRedThreads = 256;

__device__ __forceinline__ double pos_at(const double *pos, int64_t stride, const int64_t *sub, int64_t q, int axis)
{
    int64_t i = sub ? sub[q] : q;
    return pos[axis * stride + i];
}

__global__ void bbox_partial(const double *pos, int64_t stride, const int64_t *sub, int n, double *partial, const int *dn)
{
    n = dev_or(dn, n);
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double v = pos_at(pos, stride, sub, q, a);
            mn[a] = fmin(mn[a], v);
            mx[a] = fmax(mx[a], v);
        }
    }
    __shared__ double s[6][kRedThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double lo = mn[a], hi = mx[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            s[a][warp] = lo;
            s[3 + a][warp] = hi;
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double r = s[threadIdx.x][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            r = threadIdx.x < 3 ? fmin(r, s[threadIdx.x][w]) : fmax(r, s[threadIdx.x][w]);
        partial[blockIdx.x * 6 + threadIdx.x] = r;
    }
}

// Root cube from the bounding box: L = smallest power of two >= extent * (1 + 2^-20) (1 if the
// extent is 0), lo = floor(min / h) * h with h = L / 2^21.
__global__ void bbox_final(const double *partial, int nparts, int n, Geom *g, const int *dn)
{
    n = dev_or(dn, n);
    // one warp: lanes stride over the partial results, then a shuffle reduction
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nparts; b += 32)
        for (int a = 0; a < 3; ++a) {
            mn[a] = fmin(mn[a], partial[b * 6 + a]);
            mx[a] = fmax(mx[a], partial[b * 6 + 3 + a]);
        }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            mn[a] = fmin(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmax(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    if (threadIdx.x != 0) return;
    if (n <= 0) {
        for (int a = 0; a < 3; ++a) g->lo[a] = 0.0;
        g->L = 1.0;
        g->log2L = 0;
        g->inv_h = ldexp(1.0, kMaxLevel);
        return;
    }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = __dsub_rn(mx[a], mn[a]);
        if (e > ext) ext = e;
    }
    double L = 1.0;
    int log2L = 0;
    if (ext > 0.0) {
        double t = __dmul_rn(ext, 1.0 + ldexp(1.0, -20));
        int e;
        double f = frexp(t, &e);
        if (f == 0.5) {
            L = t;
            log2L = e - 1;
        } else {
            L = ldexp(1.0, e);
            log2L = e;
        }
    }
    double h = ldexp(L, -kMaxLevel);
    for (int a = 0; a < 3; ++a) g->lo[a] = __dmul_rn(floor(__ddiv_rn(mn[a], h)), h);
    g->L = L;
    g->log2L = log2L;
    g->inv_h = ldexp(1.0, kMaxLevel - log2L);
}

tg_status root_cube(tg_ctx *c, int n, const double *pos, int64_t stride, const int64_t *sub, Geom *d_geom,
                    const int *dn)
{
    double *partial = nullptr;
    int nb = grid_for(n, kRedThreads, 2 * 152);
    tg_status st = ensure_t(c, B_PARTIAL, (size_t)nb * 6, &partial);
    if (st) return st;
    {
        ProfScope ps_(c, TG_K_TREE);
        bbox_partial<<<nb, kRedThreads, 0, c->stream>>>(pos, stride, sub, n, partial, dn);
    }
    {
        ProfScope ps_(c, TG_K_TREE);
        bbox_final<<<1, 32, 0, c->stream>>>(partial, nb, n, d_geom, dn);
    }
    return cuda_check(c, cudaGetLastError(), "root cube");
}

// zero rows[0] rows of `width` floats (device row count)
__global__ void zero_rows_f32(float *p, const int *rows, int width)
{
    const int64_t n = (int64_t)*rows * width;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = 0.f;
}

// ------------------------------------------------------------------ input check
__global__ void count_nonfinite(const double *pos, int64_t stride, const int64_t *sub, int64_t n, const double *mass,
                                unsigned long long *bad)
{
    unsigned long long cnt = 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = sub ? sub[q] : q;
        const bool ok = isfinite(pos[i]) && isfinite(pos[stride + i]) && isfinite(pos[2 * stride + i]) &&
                        (mass == nullptr || isfinite(mass[i]));
        cnt += ok ? 0ull : 1ull;
    }
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(bad, cnt);
}

tg_status check_finite(tg_ctx *c, int64_t n, const double *pos, int64_t stride, const int64_t *sub, const double *mass)
{
    if (n <= 0) return TG_OK;
    unsigned long long *bad = c->d_counters + 10;
    cudaMemsetAsync(bad, 0, sizeof(unsigned long long), c->stream);
    {
        ProfScope ps_(c, TG_K_OTHER);
        count_nonfinite<<<grid_for(n, 256, 2 * c->num_sms), 256, 0, c->stream>>>(pos, stride, sub, n, mass, bad);
    }
    unsigned long long *h = reinterpret_cast<unsigned long long *>(c->h_pinned + 56);
    cudaMemcpyAsync(h, bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = stream_sync(c);
    if (e != cudaSuccess) return cuda_check(c, e, "finiteness check");
    if (*h) return set_err(c, TG_ERR_NONFINITE, "%llu particles have a non-finite position or mass", *h);
    return TG_OK;
}

// ------------------------------------------------------------------ keys
__device__ __forceinline__ uint64_t cell_coord(double x, double lo, double inv_h)
{
    double t = floor(__dmul_rn(__dsub_rn(x, lo), inv_h));
    if (t < 0.0) t = 0.0;
    const double top = (double)((1 << kMaxLevel) - 1);
    if (t > top) t = top;
    return (uint64_t)t;
}

__global__ void morton_keys(const double *pos, int64_t stride, const int64_t *sub, int n, const Geom *g,
                            uint64_t *keys, uint32_t *vals, const int *dn)
{
    n = dev_or(dn, n);
    const double lo0 = g->lo[0], lo1 = g->lo[1], lo2 = g->lo[2], inv_h = g->inv_h;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        uint64_t cx = cell_coord(pos_at(pos, stride, sub, q, 0), lo0, inv_h);
        uint64_t cy = cell_coord(pos_at(pos, stride, sub, q, 1), lo1, inv_h);
        uint64_t cz = cell_coord(pos_at(pos, stride, sub, q, 2), lo2, inv_h);
        keys[q] = (spread3_21(cx) << 2) | (spread3_21(cy) << 1) | spread3_21(cz);
        vals[q] = (uint32_t)q;
    }
}

// ------------------------------------------------------------------ radix sort
// Tiles of 2048 items: 8 warps x 8 rounds x 32 lanes, item index = warp*256 + round*32 + lane,
// so a warp's rounds run in input order and ranks are stable.
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
static_assert(kSortBins == 2 * kSortThreads, "the digit scan gives two digits to each thread");
static_assert(kSortTile == kSortTileItems, "tile size shared with the allocation-free sort");

__global__ void radix_hist(const uint64_t *keys, int n, int shift, uint32_t *hist, int nblocks, const DevEval *de)
{
    if (de) {
        n = de->n;
        nblocks = de->sort_blocks;
        if ((int)blockIdx.x >= nblocks) return;   // whole block
    }
    __shared__ uint32_t h[kSortBins];
    for (int d = threadIdx.x; d < kSortBins; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t base = (int64_t)blockIdx.x * kSortTile + warp * 256 + lane;
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t idx = base + r * 32;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & (kSortBins - 1u)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kSortBins; d += blockDim.x) hist[d * nblocks + blockIdx.x] = h[d];
}

// One pass of the stable LSD sort over a tile of kSortTile items.  Ranks: per warp in input order
// (match_any over the lanes, item r after item r - 1), warps in order.  The tile is then laid out in
// shared memory in digit order and written out by consecutive threads, so that each digit's run of
// the tile goes to global memory as one contiguous stretch.
__global__ void radix_scatter(const uint64_t *keys_in, const uint32_t *vals_in, uint64_t *keys_out,
                              uint32_t *vals_out, const uint32_t *offsets, int n, int shift, int nblocks,
                              const DevEval *de)
{
    if (de) {
        n = de->n;
        nblocks = de->sort_blocks;
        if ((int)blockIdx.x >= nblocks) return;   // whole block
    }
    __shared__ uint32_t wcount[8][kSortBins];
    __shared__ uint32_t dstart[kSortBins];
    __shared__ uint32_t wsum[8];
    __shared__ uint64_t sk[kSortTile];
    __shared__ uint32_t sv[kSortTile];
    for (int i = threadIdx.x; i < 8 * kSortBins; i += kSortThreads) (&wcount[0][0])[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kSortTile + warp * 256 + lane;
    uint64_t k[kSortItems];
    uint32_t v[kSortItems], rank[kSortItems], dig[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        int64_t idx = base + r * 32;
        bool valid = idx < n;
        k[r] = valid ? keys_in[idx] : ~0ull;   // past the end: the largest digit, after every valid item
        v[r] = valid ? vals_in[idx] : 0u;
        uint32_t d = (uint32_t)((k[r] >> shift) & (kSortBins - 1u));
        dig[r] = d;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t lower = peers & lt_mask;
        uint32_t pre = wcount[warp][d];
        rank[r] = pre + __popc(lower);
        __syncwarp();
        if (lower == 0) wcount[warp][d] = pre + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over the warps, and the tile total
    for (int d = threadIdx.x; d < kSortBins; d += kSortThreads) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            const uint32_t t = wcount[w][d];
            wcount[w][d] = run;
            run += t;
        }
        dstart[d] = run;
    }
    __syncthreads();
    // exclusive scan of the tile totals over the digits: thread t owns digits 2t, 2t + 1
    {
        const uint32_t a = dstart[2 * threadIdx.x], b = dstart[2 * threadIdx.x + 1];
        uint32_t incl = a + b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        const uint32_t excl = before + incl - (a + b);
        dstart[2 * threadIdx.x] = excl;
        dstart[2 * threadIdx.x + 1] = excl + a;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
        const uint32_t lp = dstart[dig[r]] + wcount[warp][dig[r]] + rank[r];
        sk[lp] = k[r];
        sv[lp] = v[r];
    }
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int cnt = (int)(n - tile0 < kSortTile ? n - tile0 : kSortTile);   // valid items: positions [0, cnt)
    for (int i = threadIdx.x; i < cnt; i += kSortThreads) {
        const uint64_t key = sk[i];
        const uint32_t d = (uint32_t)((key >> shift) & (kSortBins - 1u));
        const uint32_t pos = offsets[d * nblocks + blockIdx.x] + ((uint32_t)i - dstart[d]);
        keys_out[pos] = key;
        vals_out[pos] = sv[i];
    }
}

__global__ void gather_sorted(const uint32_t *perm, const double *pos, int64_t stride, const int64_t *sub,
                              const double *mass, const uint8_t *fast, int n, double *xs, double *ys, double *zs,
                              double *ms, uint8_t *fs, const int *dn)
{
    n = dev_or(dn, n);
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        uint32_t q = perm[s];
        int64_t i = sub ? sub[q] : (int64_t)q;
        xs[s] = pos[i];
        ys[s] = pos[stride + i];
        zs[s] = pos[2 * stride + i];
        ms[s] = mass[i];
        fs[s] = fast ? (fast[q] != 0) : 0;
    }
}

tg_status keys_sort_gather(tg_ctx *c, int n, const double *pos, int64_t stride, const int64_t *sub,
                           const double *mass, const uint8_t *fast, const Geom *d_geom, const DevEval *de)
{
    // with de the sizes live on the device; n is then the capacity the launches are sized for
    const int *dn = de ? &de->n : nullptr;
    uint64_t *k0, *k1;
    uint32_t *v0, *v1, *hist;
    const int nblocks = (n + kSortTile - 1) / kSortTile;
    tg_status st;
    if ((st = ensure_t(c, B_KEYS0, n, &k0)) || (st = ensure_t(c, B_KEYS1, n, &k1)) ||
        (st = ensure_t(c, B_VALS0, n, &v0)) || (st = ensure_t(c, B_VALS1, n, &v1)) ||
        (st = ensure_t(c, B_HIST, (size_t)kSortBins * nblocks + 1, &hist)))
        return st;
    {
        ProfScope ps_(c, TG_K_TREE);
        morton_keys<<<grid_for(n, 256), 256, 0, c->stream>>>(pos, stride, sub, n, d_geom, k0, v0, dn);
    }
    uint64_t *kin = k0, *kout = k1;
    uint32_t *vin = v0, *vout = v1;
    for (int pass = 0; pass < kSortPasses; ++pass) {
        const int shift = pass * kSortBits;
        {
            ProfScope ps_(c, TG_K_TREE);
            radix_hist<<<nblocks, kSortThreads, 0, c->stream>>>(kin, n, shift, hist, nblocks, de);
        }
        if ((st = exclusive_scan_u32(c, hist, hist, kSortBins * nblocks, nullptr, de ? &de->hist_items : nullptr)))
            return st;
        {
            ProfScope ps_(c, TG_K_TREE);
            radix_scatter<<<nblocks, kSortThreads, 0, c->stream>>>(kin, vin, kout, vout, hist, n, shift, nblocks, de);
        }
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    // the sorted keys and permutation live in the B_KEYS0 / B_VALS0 slots from here on
    if (kin != k0) {
        std::swap(c->buf[B_KEYS0], c->buf[B_KEYS1]);
        std::swap(c->buf[B_VALS0], c->buf[B_VALS1]);
        v0 = vin;
    }
    double *xs, *ys, *zs, *ms;
    uint8_t *fs;
    if ((st = ensure_t(c, B_XS, n, &xs)) || (st = ensure_t(c, B_YS, n, &ys)) || (st = ensure_t(c, B_ZS, n, &zs)) ||
        (st = ensure_t(c, B_MS, n, &ms)) || (st = ensure_t(c, B_FS, n, &fs)))
        return st;
    {
        ProfScope ps_(c, TG_K_TREE);
        gather_sorted<<<grid_for(n, 256), 256, 0, c->stream>>>(v0, pos, stride, sub, mass, fast, n, xs, ys, zs, ms, fs,
                                                               dn);
    }
    return cuda_check(c, cudaGetLastError(), "keys/sort/gather");
}

// ------------------------------------------------------------------ octree
__device__ __forceinline__ int key_digit(uint64_t key, int lvl) { return (int)((key >> (3 * (kMaxLevel - lvl))) & 7u); }

// first index in [s, e) whose digit at level lvl is >= d (digits are sorted within a cell)
__device__ __forceinline__ int digit_lower_bound(const uint64_t *keys, int s, int e, int lvl, int d)
{
    while (s < e) {
        int m = (s + e) >> 1;
        if (key_digit(keys[m], lvl) < d) s = m + 1;
        else e = m;
    }
    return s;
}

// Child boundaries of a cell that splits: warp per cell, lane d (1..7) finds the first particle whose
// digit at the child level is >= d; lane 0 holds the cell start and lanes 8..31 its end, so that child
// d (lane d < 8) spans [b_d, b_{d+1}).  The seven binary searches run side by side.
__device__ __forceinline__ int child_bound(const uint64_t *keys, int s, int e, int l, int lane)
{
    if (lane == 0) return s;
    if (lane >= 8) return e;
    return digit_lower_bound(keys, s, e, l, lane);
}

// Children of cell cidx (the t-th cell of its level): count (cnt[t]) and emission at le + off[t].
// The whole warp handles one cell.
__device__ __forceinline__ void oct_count_cell(const uint64_t *keys, int cidx, int t, const uint8_t *level,
                                               const int32_t *first, const int32_t *count, int n_crit, int max_level,
                                               uint32_t *cnt, int lane)
{
    if (count[cidx] <= n_crit || level[cidx] >= max_level) {
        if (lane == 0) cnt[t] = 0;
        return;
    }
    const int l = level[cidx] + 1, s = first[cidx], e = s + count[cidx];
    const int b = child_bound(keys, s, e, l, lane);
    const int bn = __shfl_down_sync(0xffffffffu, b, 1);
    const unsigned m = __ballot_sync(0xffffffffu, lane < 8 && bn > b);
    if (lane == 0) cnt[t] = __popc(m);
}

__device__ __forceinline__ void oct_emit_cell(const uint64_t *keys, int le, int cidx, int t, uint8_t *level,
                                              uint32_t *cx, uint32_t *cy, uint32_t *cz, int32_t *first, int32_t *count,
                                              int32_t *child_first, int32_t *parent, uint8_t *nchild,
                                              const uint32_t *off, const uint32_t *cnt, int lane)
{
    const int nch = cnt[t];
    if (nch == 0) {
        if (lane == 0) {
            nchild[cidx] = 0;
            child_first[cidx] = -1;
        }
        return;
    }
    const int base = le + (int)off[t];
    const int l = level[cidx] + 1, s = first[cidx], e = s + count[cidx];
    const uint32_t px = cx[cidx], py = cy[cidx], pz = cz[cidx];
    const int b = child_bound(keys, s, e, l, lane);
    const int bn = __shfl_down_sync(0xffffffffu, b, 1);
    const bool nonempty = lane < 8 && bn > b;
    const unsigned m = __ballot_sync(0xffffffffu, nonempty);
    if (nonempty) {
        const int digit = lane, ch = base + __popc(m & ((1u << lane) - 1u));
        level[ch] = (uint8_t)l;
        cx[ch] = 2u * px + ((digit >> 2) & 1);
        cy[ch] = 2u * py + ((digit >> 1) & 1);
        cz[ch] = 2u * pz + (digit & 1);
        first[ch] = b;
        count[ch] = bn - b;
        parent[ch] = cidx;
        nchild[ch] = 0;
        child_first[ch] = -1;
    }
    if (lane == 0) {
        nchild[cidx] = (uint8_t)nch;
        child_first[cidx] = base;
    }
}

__global__ void oct_count(const uint64_t *keys, int lb, int le, const uint8_t *level, const int32_t *first,
                          const int32_t *count, int n_crit, int max_level, uint32_t *cnt)
{
    const int t = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    const int cidx = lb + t;
    if (cidx >= le) return;   // whole warp
    oct_count_cell(keys, cidx, t, level, first, count, n_crit, max_level, cnt, lane);
}
__global__ void oct_emit(const uint64_t *keys, int lb, int le, uint8_t *level, uint32_t *cx, uint32_t *cy,
                         uint32_t *cz, int32_t *first, int32_t *count, int32_t *child_first, int32_t *parent,
                         uint8_t *nchild, const uint32_t *off, const uint32_t *cnt)
{
    const int t = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    const int cidx = lb + t;
    if (cidx >= le) return;   // whole warp
    oct_emit_cell(keys, le, cidx, t, level, cx, cy, cz, first, count, child_first, parent, nchild, off, cnt, lane);
}
__global__ void oct_root(int n, uint8_t *level, uint32_t *cx, uint32_t *cy, uint32_t *cz, int32_t *first,
                         int32_t *count, int32_t *child_first, int32_t *parent, uint8_t *nchild)
{
    level[0] = 0;
    cx[0] = cy[0] = cz[0] = 0;
    first[0] = 0;
    count[0] = n;
    child_first[0] = -1;
    parent[0] = -1;
    nchild[0] = 0;
}

tg_status build_octree(tg_ctx *c, int n, int *ncell_out)
{
    tg_status st;
    const uint64_t *keys = static_cast<const uint64_t *>(c->buf[B_KEYS0].p);
    int cap = 1024 + n / 4;
    uint8_t *level, *nchild;
    uint32_t *cx, *cy, *cz, *cnt, *off;
    int32_t *first, *count, *child_first, *parent;
    auto grow = [&](int need, int keep) -> tg_status {
        tg_status s;
        if ((s = ensure_keep_t(c, B_C_LEVEL, need, keep, &level)) || (s = ensure_keep_t(c, B_C_X, need, keep, &cx)) ||
            (s = ensure_keep_t(c, B_C_Y, need, keep, &cy)) || (s = ensure_keep_t(c, B_C_Z, need, keep, &cz)) ||
            (s = ensure_keep_t(c, B_C_FIRST, need, keep, &first)) ||
            (s = ensure_keep_t(c, B_C_COUNT, need, keep, &count)) ||
            (s = ensure_keep_t(c, B_C_CHILD, need, keep, &child_first)) ||
            (s = ensure_keep_t(c, B_C_PARENT, need, keep, &parent)) ||
            (s = ensure_keep_t(c, B_C_NCHILD, need, keep, &nchild)))
            return s;
        return TG_OK;
    };
    if ((st = grow(cap, 0))) return st;
    {
        ProfScope ps_(c, TG_K_TREE);
        oct_root<<<1, 1, 0, c->stream>>>(n, level, cx, cy, cz, first, count, child_first, parent, nchild);
    }
    c->level_begin.assign(1, 0);
    int lb = 0, le = 1;
    uint32_t *h_total = reinterpret_cast<uint32_t *>(c->h_pinned);
    uint32_t *d_total = reinterpret_cast<uint32_t *>(c->d_counters + 8);
    for (int lvl = 0; lvl < c->prm.max_level && le > lb; ++lvl) {
        const int m = le - lb;
        if ((st = ensure_t(c, B_C_TMP0, m, &cnt)) || (st = ensure_t(c, B_C_TMP1, m, &off))) return st;
        {
            ProfScope ps_(c, TG_K_TREE);
            oct_count<<<(int)(((int64_t)m * 32 + 255) / 256), 256, 0, c->stream>>>(keys, lb, le, level, first, count, c->prm.n_crit,
                                                             c->prm.max_level, cnt);
        }
        if ((st = exclusive_scan_u32(c, cnt, off, m, d_total, nullptr))) return st;
        cudaMemcpyAsync(h_total, d_total, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream);
        cudaError_t e = stream_sync(c);
        if (e != cudaSuccess) return cuda_check(c, e, "octree level");
        const int total = (int)*h_total;
        if (le + total > cap) {
            int ncap = le + total + (le + total) / 2 + 1024;
            if ((st = grow(ncap, le))) return st;
            cap = ncap;
        }
        {
            ProfScope ps_(c, TG_K_TREE);
            oct_emit<<<(int)(((int64_t)m * 32 + 255) / 256), 256, 0, c->stream>>>(keys, lb, le, level, cx, cy, cz, first, count, child_first,
                                                            parent, nchild, off, cnt);
        }
        c->level_begin.push_back(le);
        lb = le;
        le = le + total;
    }
    if (c->level_begin.back() != le) c->level_begin.push_back(le);
    *ncell_out = le;
    return cuda_check(c, cudaGetLastError(), "octree");
}

// ------------------------------------------------------------------ octree, sizes on the device
// The batched path builds the same tree level by level, but the level ranges, the cell count and
// the depth stay on the device (DevEval): launches are sized for the capacity, warps stride over the
// cells of their level, and levels past the tree's depth find no cells.  A level whose children
// would pass the cell capacity, or a tree deeper than the levels issued, sets an overflow bit; the
// step is then redone with larger buffers.
__global__ void oct_root_dev(DevEval *de, uint8_t *level, uint32_t *cx, uint32_t *cy, uint32_t *cz, int32_t *first,
                             int32_t *count, int32_t *child_first, int32_t *parent, uint8_t *nchild)
{
    level[0] = 0;
    cx[0] = cy[0] = cz[0] = 0;
    first[0] = 0;
    count[0] = de->n;
    child_first[0] = -1;
    parent[0] = -1;
    nchild[0] = 0;
    de->level_begin[0] = 0;
    de->level_begin[1] = 1;
    de->nlev = 1;
    de->ncell = 1;
    de->rows = 2;
    de->lvl_m = 1;
}

__global__ void oct_count_dev(const uint64_t *keys, const DevEval *de, int lvl, const uint8_t *level,
                              const int32_t *first, const int32_t *count, int n_crit, int max_level, uint32_t *cnt)
{
    if (lvl >= de->nlev) return;
    const int lb = de->level_begin[lvl], m = de->level_begin[lvl + 1] - lb;
    const int lane = threadIdx.x & 31, nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < m; t += nw)
        oct_count_cell(keys, lb + t, t, level, first, count, n_crit, max_level, cnt, lane);
}

__global__ void oct_emit_dev(const uint64_t *keys, const DevEval *de, int lvl, int cap, uint8_t *level, uint32_t *cx,
                             uint32_t *cy, uint32_t *cz, int32_t *first, int32_t *count, int32_t *child_first,
                             int32_t *parent, uint8_t *nchild, const uint32_t *off, const uint32_t *cnt)
{
    if (lvl >= de->nlev) return;
    const int lb = de->level_begin[lvl], le = de->level_begin[lvl + 1], m = le - lb;
    if ((int64_t)le + de->lvl_total > cap) return;   // over capacity: oct_finish_dev flags it
    const int lane = threadIdx.x & 31, nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); t < m; t += nw)
        oct_emit_cell(keys, le, lb + t, t, level, cx, cy, cz, first, count, child_first, parent, nchild, off, cnt, lane);
}

__global__ void oct_finish_dev(DevEval *de, int lvl, int cap, int last_issued, int max_level)
{
    if (lvl >= de->nlev) {
        de->lvl_m = 0;
        return;
    }
    const int le = de->level_begin[lvl + 1];
    int total = (int)de->lvl_total;
    if ((int64_t)le + total > cap) {
        de->overflow |= 1u;
        total = 0;
    }
    if (total > 0) {
        de->level_begin[lvl + 2] = le + total;
        de->nlev = lvl + 2;
        de->ncell = le + total;
        de->rows = 2 * (le + total);
        if (last_issued && lvl + 1 < max_level) de->overflow |= 2u;   // the tree goes deeper than issued
    }
    de->lvl_m = total;
}

tg_status build_octree_dev(tg_ctx *c, DevEval *de, int cap, int levels)
{
    tg_status st;
    const uint64_t *keys = static_cast<const uint64_t *>(c->buf[B_KEYS0].p);
    uint8_t *level, *nchild;
    uint32_t *cx, *cy, *cz, *cnt, *off;
    int32_t *first, *count, *child_first, *parent;
    if ((st = ensure_t(c, B_C_LEVEL, cap, &level)) || (st = ensure_t(c, B_C_X, cap, &cx)) ||
        (st = ensure_t(c, B_C_Y, cap, &cy)) || (st = ensure_t(c, B_C_Z, cap, &cz)) ||
        (st = ensure_t(c, B_C_FIRST, cap, &first)) || (st = ensure_t(c, B_C_COUNT, cap, &count)) ||
        (st = ensure_t(c, B_C_CHILD, cap, &child_first)) || (st = ensure_t(c, B_C_PARENT, cap, &parent)) ||
        (st = ensure_t(c, B_C_NCHILD, cap, &nchild)) || (st = ensure_t(c, B_C_TMP0, cap, &cnt)) ||
        (st = ensure_t(c, B_C_TMP1, cap, &off)))
        return st;
    {
        ProfScope ps_(c, TG_K_TREE);
        oct_root_dev<<<1, 1, 0, c->stream>>>(de, level, cx, cy, cz, first, count, child_first, parent, nchild);
    }
    const int grid = c->num_sms * 8;
    for (int lvl = 0; lvl < levels; ++lvl) {
        {
            ProfScope ps_(c, TG_K_TREE);
            oct_count_dev<<<grid, 256, 0, c->stream>>>(keys, de, lvl, level, first, count, c->prm.n_crit,
                                                       c->prm.max_level, cnt);
        }
        if ((st = exclusive_scan_u32(c, cnt, off, cap, &de->lvl_total, &de->lvl_m))) return st;
        {
            ProfScope ps_(c, TG_K_TREE);
            oct_emit_dev<<<grid, 256, 0, c->stream>>>(keys, de, lvl, cap, level, cx, cy, cz, first, count, child_first,
                                                      parent, nchild, off, cnt);
            oct_finish_dev<<<1, 1, 0, c->stream>>>(de, lvl, cap, lvl == levels - 1, c->prm.max_level);
        }
    }
    return cuda_check(c, cudaGetLastError(), "octree (device sizes)");
}

TreeView tree_view(tg_ctx *c, int n, int ncell)
{
    TreeView t;
    t.n = n;
    t.ncell = ncell;
    t.level = static_cast<const uint8_t *>(c->buf[B_C_LEVEL].p);
    t.cx = static_cast<const uint32_t *>(c->buf[B_C_X].p);
    t.cy = static_cast<const uint32_t *>(c->buf[B_C_Y].p);
    t.cz = static_cast<const uint32_t *>(c->buf[B_C_Z].p);
    t.first = static_cast<const int32_t *>(c->buf[B_C_FIRST].p);
    t.count = static_cast<const int32_t *>(c->buf[B_C_COUNT].p);
    t.child_first = static_cast<const int32_t *>(c->buf[B_C_CHILD].p);
    t.parent = static_cast<const int32_t *>(c->buf[B_C_PARENT].p);
    t.nchild = static_cast<const uint8_t *>(c->buf[B_C_NCHILD].p);
    return t;
}

}  // namespace tg
