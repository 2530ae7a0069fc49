// tg_common.cuh -- shared declarations of the CUDA library (device helpers, context, launches).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/taichi_gb.h"

namespace tg {

constexpr int kMaxLevel = 21;         // Morton keys carry 21 bits per axis
constexpr int kMaxNcrit = 128;        // columns of a P2P tile: larger leaves (n_crit up to 256) take several

inline int ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// four doubles, 32-byte aligned (per-particle offset + mass in the float64 path)
struct __align__(32) dbl4 {
    double x, y, z, w;
};

// ---------------------------------------------------------------- grow-only device buffers
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Error state shared by the host-side pipeline.  Each host function returns tg_status; the
// first failure is recorded with a message.
struct Err {
    tg_status code = TG_OK;
    std::string msg;
};

// Geometry of the root cube of one evaluation, computed on the device.
struct Geom {
    double lo[3];     // lower corner, multiple of h = L / 2^21
    double L;         // side, a power of two
    double inv_h;     // 2^21 / L
    int log2L;        // L = 2^log2L
    int pad;
};

// Sizes of one evaluation kept in device memory, for launches whose sizes the host does not read
// (the batched HOLD step: every evaluation runs inside one CUDA graph).  The plain path passes
// nullptr to the kernels and host values instead.
struct DevEval {
    int n;                  // particles of the evaluation
    int masked;             // kick pair with a fast set (two moment classes)
    int sort_blocks;        // radix-sort tiles: ceil(n / kSortTileItems)
    int hist_items;         // digit histogram entries: kSortBins * sort_blocks
    int ncell;              // cells of the tree
    int nlev;               // levels of the tree
    int lvl_m;              // cells of the level being split (octree build)
    int rows;               // 2 * ncell (expansion rows, both classes)
    int np1;                // n + 1 (prefix sum of the fast flags, with its total)
    uint32_t lvl_total;     // children emitted by the level being split (scan total)
    uint32_t overflow;      // bit 0: cells, bit 1: levels, bit 2: walk lists; the step must be redone
    int level_begin[kMaxLevel + 3];   // first cell of each level; [nlev] = ncell
};

// Octree of one evaluation (structure of arrays, cells in BFS order).
struct TreeView {
    int32_t n;           // particles
    int32_t ncell;
    const uint8_t *level;
    const uint32_t *cx, *cy, *cz;   // integer coordinates at the cell's own level
    const int32_t *first, *count, *child_first, *parent;
    const uint8_t *nchild;
    const double *rad = nullptr;   // enclosing radii (TG_MAC_SPHERE), float64 and float32 copies
    const float *radf = nullptr;
    const int *d_ncell = nullptr;  // device cell count (batched path); ncell is then a capacity
    __device__ __forceinline__ int cells() const { return d_ncell ? *d_ncell : ncell; }
};

// device count if given, else the host value
__device__ __forceinline__ int dev_or(const int *p, int v) { return p ? *p : v; }

}  // namespace tg

// ---------------------------------------------------------------- context
constexpr int kMaxSlots = 96;   // capacity of tg_ctx::buf; the slot enum below is checked against it
struct tg_ctx {
    tg_params prm;
    cudaStream_t stream = nullptr;
    // the batched evaluation runs the walk and P2P on `side` beside the leaf passes, the moments, M2L and
    // the downward pass (fork, walk-done and join events)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_walk = nullptr, ev_join = nullptr;
    int device = 0;
    int num_sms = 0;
    tg::Err err;
    tg_stats stats{};

    // scratch buffers, grown on demand
    tg::Buf buf[kMaxSlots];

    // counters on the device (p2p pair count) and pinned host mirrors
    unsigned long long *d_counters = nullptr;   // 32 words: [0] p2p particle pairs
    int64_t *h_pinned = nullptr;                // small pinned staging area (64 int64)

    // last tree/walk (host copies of sizes)
    int64_t last_n = 0, last_ncell = 0, last_nm2l = 0, last_np2p = 0, last_nblocks = 0;
    int walk_log2L = 0;                         // log2 of the last root cube side
    int64_t last_np2p_self = 0, p2p_cap = 0;    // self P2P pairs sit at the end of the P2P buffer
    double walk_front_per_cell = 8, walk_blocks_per_cell = 8, walk_p2p_per_cell = 24;   // list sizes seen so far
    std::vector<int32_t> level_begin;           // cell index range of each level (BFS)

    // live kernel timing
    int prof_level = 0;
    std::vector<cudaEvent_t> prof_events;        // pool, reused after each tg_get_profile
    std::vector<int> prof_class;                 // class of each recorded (start, end) pair
    size_t prof_used = 0;
    int64_t prof_launches[TG_K_COUNT] = {0};
    double prof_ms[TG_K_COUNT] = {0};

    // HHS binding
    int64_t hhs_n = 0;
    double *hhs_pos = nullptr, *hhs_vel = nullptr;
    const double *hhs_mass = nullptr;
    double hhs_time = 0.0;
    int bound_integrator = 0;                   // 1: HHS (tg_hhs_init), 2: traditional (tg_trad_init)

    // failure injection (tg_debug_control): allocations allowed before they fail, < 0 = off
    int64_t debug_fail_alloc_after = -1;

    // launch shapes picked by tg_autotune (n_crit lives in prm)
    tg_tuning tune{0, 2, 16, 0, 0, 0.0, 0.0};

    // batched HOLD step: captured graph and its state (hhs.cu); scratch reallocations since tg_create
    // (a captured graph holds raw buffer addresses, so a reallocation makes it stale)
    struct HoldGraph *hold = nullptr;
    uint64_t alloc_epoch = 0;
    bool capturing = false;          // inside a stream capture: scratch must not grow
    unsigned debug_queue_limit = 0;  // tg_debug_control: iteration limit of the device loop (0: default)
    int debug_queue_hold = 0;        // tg_debug_control: the scheduler publishes no operation
    int64_t debug_batch_caps = 0;    // tg_debug_control: initial capacities of the batched step
};

namespace tg {

// buffer slots of tg_ctx::buf
enum Slot {
    B_GEOM = 0, B_PARTIAL, B_KEYS0, B_KEYS1, B_VALS0, B_VALS1, B_HIST, B_SCAN_TMP,
    B_XS, B_YS, B_ZS, B_MS, B_FS, B_PF, B_LEAF_OF,
    B_XS2, B_YS2, B_ZS2, B_MS2, B_FS2, B_PERM2, B_NSLOW,
    B_C_LEVEL, B_C_X, B_C_Y, B_C_Z, B_C_FIRST, B_C_COUNT, B_C_CHILD, B_C_PARENT, B_C_NCHILD,
    B_C_TMP0, B_C_TMP1, B_C_RAD, B_C_RADF,
    B_MOM, B_MOMF, B_MOM01, B_LOC, B_ACC, B_MOMH, B_LOCH,
    B_FRONT0, B_FRONT1, B_M2L, B_P2P, B_WALK_CNT,
    B_SUB_ACC, B_HHS_AOLD, B_HHS_ACUR, B_HHS_ATOT, B_TRAD_ACC, B_TRAD_END, B_HHS_DT, B_HHS_RUNG, B_HHS_IDX, B_HHS_FLAG,
    B_HHS_SCAN, B_HHS_TMP, B_RED, B_DIAG_POT, B_DIAG_ACC,
    B_OWN_CNT, B_OWN_FILL, B_OWN_OFF, B_OWN_LIST, B_OWN_TAG, B_OWN_PART, B_SNAP, B_TUNE_ACC,
    B_MACP, B_DEVEVAL, B_HOLD, B_FRAME_X, B_FRAME_M, B_FRAME_F, B_SPLIT_FLAG, B_SPLIT_PRE,
    B_M2L_CNT, B_M2L_OFF, B_M2L_FILL, B_M2L_SRC, B_FWORDS, B_FPRE, B_M2L_PART, B_M2L_PCNT, B_TUNE_SNAP, B_SCAN_TMP2, B_ACC_P2P,
    B_LAST_SLOT
};
static_assert(B_LAST_SLOT <= kMaxSlots, "tg_ctx::buf holds fewer entries than there are slots");

tg_status set_err(tg_ctx *c, tg_status code, const char *fmt, ...);
// Host wait on the context's stream inside the pipeline (counted in tg_stats.host_syncs).
cudaError_t stream_sync(tg_ctx *c);
tg_status cuda_check(tg_ctx *c, cudaError_t e, const char *what);
// Make buffer `slot` at least `bytes` long (contents are not preserved when it grows).
tg_status ensure(tg_ctx *c, int slot, size_t bytes, void **out);
template <class T>
inline tg_status ensure_t(tg_ctx *c, int slot, size_t count, T **out)
{
    void *p = nullptr;
    tg_status s = ensure(c, slot, count * sizeof(T) + 16, &p);
    *out = static_cast<T *>(p);
    return s;
}

// M2L work unit handed over by the walk: the well-separated child pairs of one opened cell pair.
struct M2LBlock {
    uint32_t a, b;             // cell pair that was opened (a == b: self pair, only i < j bits set)
    unsigned long long mask;   // bit 8i + j: pair (child i of a, child j of b) is well separated
};

// The float32 kernels for p <= 6 count the M2L side contractions they need on the device
// (d_counters[11]); the other paths count class pairs on the host.
inline bool m2l_classes_on_device(const tg_ctx *c) { return c->prm.precision == TG_PREC_FP32 && c->prm.p <= 6; }

// ---- tree.cu
// Root cube of the n particles pos[q] (q < n, gathered through sub when non-null) -> geom.
tg_status root_cube(tg_ctx *c, int n, const double *pos, int64_t stride, const int64_t *sub, Geom *d_geom,
                    const int *dn = nullptr);
// Keys, stable radix sort and gather into sorted order.  Returns device pointers in the ctx
// slots: B_KEYS0 (sorted keys), B_VALS0 (perm: sorted -> input index q), B_XS.. B_FS.
tg_status keys_sort_gather(tg_ctx *c, int n, const double *pos, int64_t stride, const int64_t *sub,
                           const double *mass, const uint8_t *fast, const Geom *d_geom, const DevEval *de = nullptr);
// Octree from the sorted keys; fills the cell slots and c->level_begin.  Returns ncell.
tg_status build_octree(tg_ctx *c, int n, int *ncell_out);
TreeView tree_view(tg_ctx *c, int n, int ncell);
// The same octree with its sizes on the device (de): `cap` cells at most, `levels` levels issued.
tg_status build_octree_dev(tg_ctx *c, DevEval *de, int cap, int levels);

// Expansion kernels for orders above the fixed tables (TG_PMAX < p <= kPHigh), high_order.cu.
constexpr int kPHigh = 20;
template <class T, class T4>
tg_status launch_p2m_hi(tg_ctx *c, const TreeView &t, const Geom *d_geom, const double *xs, const double *ys,
                        const double *zs, const double *ms, const uint8_t *fs, const T4 *pf, int p, int nc, int ncp,
                        T *M, double *M01);
template <class T>
tg_status launch_m2m_hi(tg_ctx *c, const TreeView &t, int lb, int le, int p, int nc, int ncp, T *M, double *M01);
template <class T>
tg_status launch_m2l_hi(tg_ctx *c, const TreeView &t, const M2LBlock *blocks, int64_t nblocks, const T *Ms, T *L,
                        int p, int nc, int ncp, bool masked, bool pot);
template <class T>
tg_status launch_l2l_hi(tg_ctx *c, const TreeView &t, int lb, int le, int p, int nc, int ncp, int ncls, int n_first,
                        T *L);
template <class T, class T4>
tg_status launch_l2p_hi(tg_ctx *c, int n, const TreeView &t, const T4 *pf, const int32_t *leaf_of, const uint8_t *fs,
                        bool masked, int p, int ncp, const T *L, double *acc4);

// Count the non-finite positions (gathered through sub when non-null) and masses of n particles on the
// device; TG_ERR_NONFINITE (with a message) if there is one.  Synchronising.
tg_status check_finite(tg_ctx *c, int64_t n, const double *pos, int64_t stride, const int64_t *sub,
                       const double *mass);
// count of the non-finite positions and masses of n particles, added to *bad (tree.cu)
__global__ void count_nonfinite(const double *pos, int64_t stride, const int64_t *sub, int64_t n, const double *mass,
                                unsigned long long *bad);
// Consume one allocation of the failure injection; TG_ERR_OOM when it says this one fails.
tg_status injected_alloc_failure(tg_ctx *c, size_t bytes, int slot);

// Device-wide exclusive scan of uint32 (in place allowed); optional total to a device word.
tg_status exclusive_scan_u32(tg_ctx *c, const uint32_t *in, uint32_t *out, int n, uint32_t *d_total,
                             const int *dn = nullptr, int scratch = B_SCAN_TMP);

// ---- m2l.cu: mutual M2L of the walk's blocks into L (normalised expansions).  pot = false: the
// float32 kernels leave out the potential term L^0.  fpre (kick pairs, nullable): prefix sum of the fast
// flags of the sorted particles, so that contractions no target needs are skipped.
tg_status launch_m2l_f32(tg_ctx *c, const TreeView &t, const M2LBlock *blocks, int64_t nblocks, const float *Ms,
                         float *L, int p, int nc, int ncp, bool masked, bool pot, const uint32_t *fpre = nullptr);
// the prefix sum of the fast flags fs of n sorted particles (n + 1 entries) into fpre (dn: device n)
tg_status fast_prefix(tg_ctx *c, const uint8_t *fs, int n, uint32_t **fpre, const DevEval *de);
tg_status launch_m2l_f32_dev(tg_ctx *c, const TreeView &t, const DevEval *de, const Geom *gp, const M2LBlock *blocks,
                             const unsigned long long *dnb, int64_t cap_blocks, const float *Ms, float *L, int p,
                             int ncp, int cap_cells, size_t cap_src, const uint32_t *fpre);
tg_status launch_m2l_f64_dev(tg_ctx *c, const TreeView &t, const DevEval *de, const Geom *gp, const M2LBlock *blocks,
                             const unsigned long long *dnb, int64_t cap_blocks, const double *Ms, double *L, int p,
                             int ncp);
tg_status launch_p2p_f64_dev(tg_ctx *c, const TreeView &t, const Geom *d_geom, const unsigned long long *walk_ctr,
                             const uint2 *p2p, size_t cap_p2p, const dbl4 *pf, const uint8_t *fs, double *acc4, int stride);
tg_status launch_m2l_f64(tg_ctx *c, const TreeView &t, const M2LBlock *blocks, int64_t nblocks, const double *Ms,
                         double *L, int p, int nc, int ncp, bool masked);
// ---- p2p.cu: mutual P2P of all leaf pairs (distinct pairs and self pairs) into acc4.
tg_status launch_p2p_f32(tg_ctx *c, const TreeView &t, const uint2 *pairs, int64_t npairs, const uint2 *self_pairs,
                         int64_t nself, const float4 *pf, const int32_t *nslow, bool pot, double *acc4);
tg_status launch_p2p_f32_dev(tg_ctx *c, const TreeView &t, const DevEval *de, const Geom *gp,
                             const unsigned long long *walk_ctr, const uint2 *p2p, size_t cap_p2p, int cap_cells,
                             const float4 *pf, const int32_t *nslow, double *acc4, int stride,
                             int scan_scratch = B_SCAN_TMP);
tg_status launch_p2p_f64(tg_ctx *c, const TreeView &t, const Geom *d_geom, const uint2 *pairs, int64_t npairs,
                         const uint2 *self_pairs, int64_t nself, const dbl4 *pf, const uint8_t *fs, bool masked,
                         double *acc4);

// Kernels of tree.cu, also launched by the allocation-free sort in noalloc.cu.
constexpr int kSortTileItems = 2048;     // items per radix-sort block (256 threads x 8)
constexpr int kSortBits = 9;             // radix digit width: 7 passes cover the 63 key bits
constexpr int kSortBins = 1 << kSortBits;
constexpr int kSortPasses = (63 + kSortBits - 1) / kSortBits;
constexpr int kScanThreads = 512;        // threads per scan block
constexpr int kScanTileItems = 2048;     // items per scan block (kScanThreads x 4)
// (optional device sizes: dn / de, nullptr for host sizes)
__global__ void scan_tiles(const uint32_t *in, uint32_t *out, uint32_t *tile_sums, int n, const int *dn);
__global__ void scan_add(uint32_t *out, const uint32_t *tile_pre, int n, const int *dn);
__global__ void bbox_partial(const double *pos, int64_t stride, const int64_t *sub, int n, double *partial, const int *dn);
__global__ void bbox_final(const double *partial, int nparts, int n, Geom *g, const int *dn);
__global__ void morton_keys(const double *pos, int64_t stride, const int64_t *sub, int n, const Geom *g,
                            uint64_t *keys, uint32_t *vals, const int *dn);
__global__ void radix_hist(const uint64_t *keys, int n, int shift, uint32_t *hist, int nblocks, const DevEval *de);
__global__ void radix_scatter(const uint64_t *keys_in, const uint32_t *vals_in, uint64_t *keys_out,
                              uint32_t *vals_out, const uint32_t *offsets, int n, int shift, int nblocks,
                              const DevEval *de);

// ---- fmm.cu
// Full FMM evaluation on a (sub)set of particles.  Outputs are in input order q:
// acc (3 SoA arrays of length n with stride `out_stride`), pot (nullable).
tg_status fmm_eval(tg_ctx *c, int n, const double *pos, int64_t stride, const int64_t *sub,
                   const double *mass, const uint8_t *fast, double *acc, int64_t out_stride, double *pot,
                   bool keep_tree);
tg_status direct_eval(tg_ctx *c, int64_t n, const double *pos, const double *mass, const uint8_t *fast,
                      int64_t n_sink, const int64_t *sink_idx, double *acc, double *pot);

// Capacities of the device-sized evaluation (batched HOLD step): particles, cells, octree levels issued,
// and the walk's frontier, M2L-block and P2P-pair lists.
struct BatchCaps {
    int n = 0, cells = 0, levels = 0;
    size_t front = 0, blocks = 0, p2p = 0;
    size_t m2l_src = 0;   // entries of the directed M2L source lists (two per cell pair)
};
// One float32 evaluation of de->n particles (xin: 3 x cap.n SoA, min, fin: kick-pair classes when
// de->masked) into acc (3 x cap.n SoA, input order), every size on the device; stats accumulates the
// counters of eval_finish_dev.  No host synchronisation, so it can be captured in a CUDA graph.
tg_status fmm_eval_dev(tg_ctx *c, DevEval *de, const BatchCaps &cap, const double *xin, const double *min,
                       const uint8_t *fin, double *acc, unsigned long long *stats);
// zero rows[0] rows of `width` floats (device row count)
__global__ void zero_rows_f32(float *p, const int *rows, int width);
// constant part of the acceptance thresholds into device memory (before a capture; synchronising)
tg_status mac_params_upload(tg_ctx *c);

// ---- batched HOLD step (hhs.cu)
tg_status hhs_step_batched(tg_ctx *c);
tg_status ensemble_step(tg_ctx **cs, int count);
void hold_graph_destroy(tg_ctx *c);
void hold_graph_reset_sizes(tg_ctx *c);
// words of scan scratch exclusive_scan_u32 needs for n values
size_t scan_scratch_words(int n);

// ---- tune.cu
tg_status autotune(tg_ctx *c, int n, const double *pos, const double *mass, const uint8_t *fast, tg_tuning *out);

// ---- hhs.cu
tg_status hhs_init(tg_ctx *c);
tg_status hhs_step(tg_ctx *c);
tg_status hhs_save(tg_ctx *c, int slot);
tg_status hhs_load(tg_ctx *c, int slot);
tg_status trad_init(tg_ctx *c);
tg_status trad_step(tg_ctx *c);
tg_status hhs_diagnostics(tg_ctx *c, double out[8]);
tg_status timesteps(tg_ctx *c, int64_t n, const double *a_old, const double *a_cur, const double *a_tot, double *dt,
                    int32_t *rung);

// Wrap each kernel launch: counts launches per class and, when profiling is on for the class,
// records CUDA events around it on the context stream.
struct ProfScope {
    tg_ctx *c;
    int cls;
    bool timed;
    ProfScope(tg_ctx *ctx, int k);
    ~ProfScope();
};
tg_status prof_collect(tg_ctx *c);

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ uint64_t spread3_21(uint64_t v)
{
    // spread the low 21 bits of v so that bit b lands on bit 3b
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Exact float -> double conversion on the integer pipe (GB300's FP64 pipe is ~1/64 the FP32 rate).
__device__ __forceinline__ double f2d_exact(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    if (e == 0) return __longlong_as_double((long long)sign);   // zero (float32 subnormals flush to zero)
    const uint64_t ee = (e == 0xffu) ? 0x7ffull : (uint64_t)(e + 896u);   // inf / nan keep their class
    const uint64_t bits = sign | (ee << 52) | ((uint64_t)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// Offset between two cell centres along one axis in units of 2^-(lf+1) of the root side, where
// lf is the finer level: (2 c_a + 1) 2^(lf - la) - (2 c_b + 1) 2^(lf - lb).  Exact integer.
__device__ __forceinline__ long long centre_delta(uint32_t ca, int la, uint32_t cb, int lb, int lf)
{
    return ((2ll * ca + 1) << (lf - la)) - ((2ll * cb + 1) << (lf - lb));
}

// 2^e as a float, exact, for -126 <= e <= 127 (built from the exponent bits)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

__host__ __device__ __forceinline__ int ncoef_dev(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// centre of cell c along one axis: lo + (i + 1/2) L / 2^level (exact: dyadic)
__device__ __forceinline__ double cell_centre(const Geom &g, const TreeView &t, int c, int axis)
{
    const uint32_t ci = axis == 0 ? t.cx[c] : (axis == 1 ? t.cy[c] : t.cz[c]);
    return g.lo[axis] + ((double)ci + 0.5) * ldexp(g.L, -(int)t.level[c]);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

inline int grid_for(int64_t n, int block, int max_blocks = 152 * 32)
{
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (int)g;
}

}  // namespace tg
