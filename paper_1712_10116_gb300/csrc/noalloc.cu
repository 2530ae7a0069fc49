// noalloc.cu -- tg_morton_sort_noalloc: root cube, Morton keys and the stable radix sort for
// callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: applications whose device memory is owned by another
// allocator (a framework's pool, a fixed memory budget that raw allocations would break) and
// loops that cannot afford the device-wide synchronisation an allocation can cause.  This entry
// point takes the caller's input and output buffers and keeps all of its scratch in one
// file-scope device array of fixed size, so it never allocates.
//
// The array lives in every GPU that loads the library until the process exits.  Host code must
// not use the array's name as a pointer: on the host it is only a stand-in for the device
// symbol.  Every call looks the device address up with cudaGetSymbolAddress, with the caller's
// device current (a cheap query that allocates nothing), so no address outlives a device reset.
#include "tg_common.cuh"

namespace {

using namespace tg;

constexpr int64_t kMaxN = TG_NOALLOC_MAX_N;
constexpr int kMaxSortBlocks = (int)((kMaxN + kSortTileItems - 1) / kSortTileItems);
constexpr int kMaxBboxBlocks = 2 * 152;
constexpr int64_t kHistItems = (int64_t)kSortBins * kMaxSortBlocks;
constexpr int64_t kScanTmpItems = 2 * ((kHistItems + kScanTileItems - 1) / kScanTileItems) + 64;

// levels of the tile-sum recursion of the histogram scan: scan_with_scratch keeps at most 8
constexpr int scan_levels(int64_t m) { return m <= kScanTileItems ? 1 : 1 + scan_levels((m + kScanTileItems - 1) / kScanTileItems); }
static_assert(scan_levels(kHistItems) <= 8, "the histogram scan of the largest input needs more than 8 levels");

// byte layout of the scratch array (every part 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kOffGeom = 0;
constexpr size_t kOffPartial = align256(kOffGeom + sizeof(Geom));
constexpr size_t kOffKeys0 = align256(kOffPartial + sizeof(double) * 6 * kMaxBboxBlocks);
constexpr size_t kOffKeys1 = align256(kOffKeys0 + sizeof(uint64_t) * kMaxN);
constexpr size_t kOffVals0 = align256(kOffKeys1 + sizeof(uint64_t) * kMaxN);
constexpr size_t kOffVals1 = align256(kOffVals0 + sizeof(uint32_t) * kMaxN);
constexpr size_t kOffHist = align256(kOffVals1 + sizeof(uint32_t) * kMaxN);
constexpr size_t kOffScan = align256(kOffHist + sizeof(uint32_t) * kHistItems);
constexpr size_t kScratchBytes = align256(kOffScan + sizeof(uint32_t) * kScanTmpItems);
static_assert(kScratchBytes < (8u << 20), "the allocation-free scratch must stay modest (< 8 MB)");

// The scratch.  Device code could name it directly; host code uses the looked-up address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Address of the scratch on the current device.  Looked up on every call: the query is cheap,
// allocates nothing, and stays right after a device reset reloads the module.
tg_status scratch_for_current_device(unsigned char **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
        cudaGetLastError();
        return TG_ERR_CUDA;
    }
    *out = static_cast<unsigned char *>(p);
    return TG_OK;
}

__global__ void noalloc_export(int n, const uint64_t *keys, const uint32_t *vals, uint64_t *keys_out, int64_t *perm_out)
{
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        keys_out[s] = keys[s];
        perm_out[s] = (int64_t)vals[s];
    }
}

// exclusive scan with caller-provided scratch (same kernels as the context path)
cudaError_t scan_with_scratch(cudaStream_t st, const uint32_t *in, uint32_t *out, int n, uint32_t *tmp)
{
    struct Level { uint32_t *out; int n, ntiles; uint32_t *sums, *pre; };
    Level lv[8];
    int depth = 0;
    const uint32_t *cin = in;
    uint32_t *cout = out;
    int cn = n;
    uint32_t *cursor = tmp;
    bool complete = false;
    while (depth < 8) {
        const int nt = (cn + kScanTileItems - 1) / kScanTileItems;
        lv[depth] = {cout, cn, nt, cursor, cursor + nt};
        scan_tiles<<<nt, kScanThreads, 0, st>>>(cin, cout, cursor, cn, nullptr);
        ++depth;
        if (nt == 1) {
            complete = true;
            break;
        }
        cin = cursor;
        cout = cursor + nt;
        cn = nt;
        cursor += 2 * nt + 2;
    }
    if (!complete) return cudaErrorInvalidValue;   // excluded by the static_assert on scan_levels
    for (int d = depth - 2; d >= 0; --d) scan_add<<<lv[d].ntiles, kScanThreads, 0, st>>>(lv[d].out, lv[d].pre, lv[d].n, nullptr);
    return cudaGetLastError();
}

// device memory of the current device (managed memory is reachable from any device)
int check_dev(const void *p)
{
    cudaPointerAttributes a;
    int dev = -1;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeManaged) return 1;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" tg_status tg_morton_sort_noalloc(int64_t n, const double *pos, uint64_t *keys_out, int64_t *perm_out,
                                            void *cuda_stream)
{
    if (n < 0 || n > kMaxN) return TG_ERR_ARG;
    if (n == 0) return TG_OK;
    if (!check_dev(pos) || !check_dev(keys_out) || !check_dev(perm_out)) return TG_ERR_ARG;
    unsigned char *base = nullptr;
    tg_status st = scratch_for_current_device(&base);
    if (st) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    Geom *geom = reinterpret_cast<Geom *>(base + kOffGeom);
    double *partial = reinterpret_cast<double *>(base + kOffPartial);
    uint64_t *k0 = reinterpret_cast<uint64_t *>(base + kOffKeys0), *k1 = reinterpret_cast<uint64_t *>(base + kOffKeys1);
    uint32_t *v0 = reinterpret_cast<uint32_t *>(base + kOffVals0), *v1 = reinterpret_cast<uint32_t *>(base + kOffVals1);
    uint32_t *hist = reinterpret_cast<uint32_t *>(base + kOffHist), *scan = reinterpret_cast<uint32_t *>(base + kOffScan);
    const int ni = (int)n;
    // every scratch word used below is written before it is read, so nothing needs clearing
    const int nb = grid_for(n, 256, kMaxBboxBlocks);
    bbox_partial<<<nb, 256, 0, s>>>(pos, n, nullptr, ni, partial, nullptr);
    bbox_final<<<1, 32, 0, s>>>(partial, nb, ni, geom, nullptr);
    morton_keys<<<grid_for(n, 256), 256, 0, s>>>(pos, n, nullptr, ni, geom, k0, v0, nullptr);
    const int nblocks = (ni + kSortTileItems - 1) / kSortTileItems;
    uint64_t *kin = k0, *kout = k1;
    uint32_t *vin = v0, *vout = v1;
    for (int pass = 0; pass < kSortPasses; ++pass) {
        const int shift = pass * kSortBits;
        radix_hist<<<nblocks, 256, 0, s>>>(kin, ni, shift, hist, nblocks, nullptr);
        if (scan_with_scratch(s, hist, hist, kSortBins * nblocks, scan) != cudaSuccess) return TG_ERR_CUDA;
        radix_scatter<<<nblocks, 256, 0, s>>>(kin, vin, kout, vout, hist, ni, shift, nblocks, nullptr);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    noalloc_export<<<grid_for(n, 256), 256, 0, s>>>(ni, kin, vin, keys_out, perm_out);
    if (cudaGetLastError() != cudaSuccess) return TG_ERR_CUDA;
    return TG_OK;
}
