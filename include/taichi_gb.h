/*
 * taichi_gb.h -- C ABI of the GB300 (sm_103a) momentum-conserving FMM + HHS library.
 *
 * The method is Zhu (2017), "A momentum conserving N-body scheme with individual
 * timesteps": a fast multipole gravity solver whose cell-cell (M2L) and particle-particle
 * (P2P) interactions are evaluated mutually (F_AB = -F_BA, Sec. 2.1, Eq. 2), driven by the
 * hierarchical Hamiltonian splitting (HOLD) integrator with individual timesteps
 * (Sec. 2.2, Algorithms 1-3).  Every step runs in CUDA kernels of this library.
 *
 * Conventions for every entry point
 *   - Particle arrays are CALLER-OWNED DEVICE memory (e.g. torch CUDA tensors), in the caller's
 *     particle order.  Positions, velocities and accelerations are SoA float64 arrays of
 *     3*n doubles: x[0..n), y[0..n), z[0..n).  Masses are n float64 values.
 *   - G = 1; potentials are negative (-m/r far from a mass).
 *   - The context owns all scratch memory (tree, lists, expansions) and grows it on demand.
 *   - All work is issued on the CUDA stream given to tg_create.  Calls return when the work is
 *     enqueued, except where a call is documented as synchronising.  Inside a batched HOLD step the
 *     dual walk and P2P of each evaluation run on a second stream that the context creates and owns;
 *     it forks from and joins the caller's stream with events, so to the caller all the work is
 *     ordered on its own stream.
 *   - Errors are returned as tg_status codes; no exception crosses the ABI.  On an argument
 *     error nothing is launched and outputs are untouched.  tg_last_error() gives a message.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef TAICHI_GB_H
#define TAICHI_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TG_OK = 0,
    TG_ERR_ARG = -1,        /* invalid argument (null pointer, n < 0, p out of range, ...)  */
    TG_ERR_OOM = -2,        /* device allocation failed                                     */
    TG_ERR_CUDA = -3,       /* a CUDA runtime call or kernel launch failed                  */
    TG_ERR_TIMEOUT = -4,    /* a bounded device-side wait gave up                           */
    TG_ERR_NONFINITE = -5,  /* non-finite positions or masses                               */
    TG_ERR_CAPACITY = -6,   /* an internal list exceeded its limit even after regrowth      */
    TG_ERR_STATE = -7,      /* call out of order (e.g. tg_hhs_step before tg_hhs_init)       */
    TG_ERR_IO = -8          /* checkpoint file cannot be written, read, or fails its check     */
} tg_status;

typedef enum {
    TG_KERNEL_WENDLAND_C2 = 0,  /* Eq. (8), Sec. 2.3; cell pairs closer than eps use P2P      */
    TG_KERNEL_PLUMMER = 1       /* phi = -1/sqrt(r^2 + eps^2); expansions of that kernel       */
} tg_kernel;

typedef enum {
    TG_PREC_FP64 = 0,  /* plain path: every stage in float64                               */
    TG_PREC_FP32 = 1   /* P2P, M2L, L2L, L2P in float32 relative to float32 cell centres;   */
                       /* moments, drift, reductions and outputs in float64                */
} tg_precision;

typedef enum {
    TG_MAC_SIDE = 0,    /* Eq. (1) with R = kappa * cell side (the paper's criterion)          */
    TG_MAC_SPHERE = 1   /* R = radius of a sphere about the cell centre enclosing its particles */
                        /* (leaves: farthest particle; parents: max over children of            */
                        /* |z_c - z_p| + R_c), accepted when R_a + R_b < theta |z_a - z_b|,     */
                        /* decided in float64 with explicit rounding; the eps gap rule stays.  */
                        /* Not the paper's criterion: the alternative it names (Sec. 2.3, 4)   */
} tg_mac;

typedef struct {
    int p;            /* expansion order: Taylor terms of total degree <= p, 1 <= p <= 20     */
                      /* (p <= 6: generated float32 contractions; p > 8: table-free kernels   */
                      /* for the order sweeps of Sec. 3.2, slower)                             */
    int n_crit;       /* a cell holding more than n_crit particles is split (Sec. 2.3), 1..256 */
    int kernel;       /* tg_kernel                                                          */
    int precision;    /* tg_precision                                                       */
    int max_level;    /* deepest octree level, 1..21 (21 = Morton-key resolution)           */
    int k_max;        /* deepest HHS rung (timestep dt_max / 2^k_max), 0..30                 */
    double theta;     /* opening angle of Eq. (1), > 0                                       */
    double kappa;     /* R in Eq. (1) = kappa * cell side; the paper's reading is kappa = 1  */
    double eps;       /* softening length, > 0                                               */
    double eta;       /* timestep parameter: dt_i = sqrt(eta * eps / |a|), Sec. 2.2          */
    double dt_max;    /* step of rung 0                                                      */
    double eta_tot;   /* eta_1 of the minimum-timestep constraint of Eq. (9), >= 0; 0 = off:  */
                      /* dt_i = min(dt_i, sqrt(eta_tot * eps / |a|_tot,i)), |a|_tot from all  */
                      /* masses, recorded at the second kickFS2S of rung 0 (the whole system) */
    int mac;          /* tg_mac: the multipole acceptance criterion of the walk             */
    int batched;      /* 0: plain HOLD step, driven from the host (one launch sequence per     */
                      /*    evaluation, the host reads each split's size);                     */
                      /* 1: batched HOLD step: the recursion of Algorithms 1-2 runs as a       */
                      /*    device-side work queue inside one CUDA graph per rung-0 step        */
                      /*    (a WHILE node driven by a scheduler kernel, evaluations sized on    */
                      /*    the device).  Needs precision FP32, 4 <= p <= 6 and TG_MAC_SIDE.    */
} tg_params;

typedef struct tg_ctx tg_ctx;

/* Counters of the work done since tg_create or the last tg_reset_stats (host copies). */
typedef struct {
    int64_t evaluations;     /* FMM evaluations (one per tg_fmm_forces / kick pair)            */
    int64_t sink_forces;     /* particle forces delivered (particle-forces, the throughput unit) */
    int64_t p2p_pairs;       /* unordered particle pairs evaluated by P2P (F-F pairs excluded)   */
    int64_t m2l_pairs;       /* unordered cell pairs evaluated by M2L                           */
    int64_t p2p_cell_pairs;  /* unordered leaf pairs (self pairs included)                      */
    int64_t cells;           /* octree cells built, summed over evaluations                    */
    int64_t kdk_frames;      /* KDK frames of the HHS schedule                                  */
    int64_t max_rung;        /* deepest rung that held a slow particle                          */
    int64_t m2l_class_pairs; /* M2L cell pairs x local-expansion classes the pair's targets need     */
                             /* (a kick pair's cell needs class 0 only if it holds slow particles, */
                             /* class 1 only if it holds fast ones and the source slow ones, since */
                             /* class 1 carries the slow masses; counted per side, halved)         */
    int64_t list_regrowths;  /* dual walks re-run because an interaction list outgrew its buffer  */
    int64_t host_syncs;      /* host waits on the stream inside evaluations and HHS steps         */
} tg_stats;

/* Create a context bound to `cuda_stream` (a cudaStream_t, NULL = legacy default stream) on the
 * current device.  Validates params (TG_ERR_ARG).  Allocates only small control blocks, plus the
 * context's own non-blocking side stream and three events (TG_ERR_CUDA if they cannot be created). */
tg_status tg_create(const tg_params *params, void *cuda_stream, tg_ctx **out);
tg_status tg_destroy(tg_ctx *ctx);
const char *tg_last_error(const tg_ctx *ctx);
tg_status tg_get_stats(const tg_ctx *ctx, tg_stats *out);
tg_status tg_reset_stats(tg_ctx *ctx);

/* Root cube, Morton keys, radix sort and octree of n particles (Sec. 2.3), kept in the context
 * for tg_get_tree / tg_get_lists.  pos: device, 3*n float64.  Synchronising. */
tg_status tg_build_tree(tg_ctx *ctx, int64_t n, const double *pos);

/* One FMM evaluation: the Poisson-solver call of Algorithm 3 (get_force_potential), with the
 * mutual M2L/P2P of Sec. 2.1 and the Algorithm 4 walk.
 *   pos     device, 3*n float64 (SoA)
 *   mass    device, n float64
 *   is_fast device, n uint8 or NULL.  NULL: every particle feels every mass.  Otherwise the
 *           particles with is_fast[i] != 0 form the fast set F: slow sinks feel all masses
 *           (kickFS2S) and fast sinks feel slow masses only (kickS2F) -- one kick pair of
 *           Algorithm 2 evaluated on a single tree and walk.
 *   acc     device, 3*n float64 output (SoA), overwritten
 *   pot     device, n float64 output or NULL
 * TG_ERR_NONFINITE if a position or mass is NaN or infinite (checked on the device first; acc
 * and pot are then untouched).  Not synchronising (host reads of sizes aside). */
tg_status tg_fmm_forces(tg_ctx *ctx, int64_t n, const double *pos, const double *mass,
                        const uint8_t *is_fast, double *acc, double *pot);

/* Direct O(N^2) float64 summation for n_sink sinks (sink_idx device int64[n_sink], NULL = the
 * first n_sink particles) from all n sources, with the same kernel and mask semantics as
 * tg_fmm_forces.  acc: device 3*n_sink float64 (SoA); pot: device n_sink float64 or NULL.
 * Used to measure FMM force errors on a sample of sinks. */
tg_status tg_direct_forces(tg_ctx *ctx, int64_t n, const double *pos, const double *mass,
                           const uint8_t *is_fast, int64_t n_sink, const int64_t *sink_idx,
                           double *acc, double *pot);

/* HOLD integrator (Sec. 2.2).  tg_hhs_init binds caller-owned device arrays pos (3*n), vel (3*n)
 * and mass (n) to the context; they are updated in place by every tg_hhs_step and must stay
 * allocated until tg_destroy or the next tg_hhs_init.  It performs the initial all-from-all
 * evaluation that sets |a_current|; |a_old| starts at 0.  TG_ERR_NONFINITE if a position or
 * mass is not finite. */
tg_status tg_hhs_init(tg_ctx *ctx, int64_t n, double *pos, double *vel, const double *mass);
/* One rung-0 step of EVOLVE_HOLD (Algorithm 1) of length params.dt_max: recursive
 * slow/fast split, KDK (Algorithm 2) with the kickS2F/kickFS2S pairs of Algorithm 3, drifts.
 * With params.batched the step is one CUDA graph launch: the first batched step sizes its buffers
 * with one plain evaluation of the bound system and captures the graph (again after any buffer or
 * parameter change); a list, cell or depth capacity exceeded inside the step restores the state
 * and redoes the step with larger buffers; the device loop is bounded and returns TG_ERR_TIMEOUT
 * (state restored) if it runs out.  The host reads the step's counters once at its end.
 * The step length is params.dt_max (the survey's hhs_step(dt) reads dt from the parameters, fixed
 * at tg_create, so that the rung ladder dt_max / 2^k stays the same for the whole run).
 * The step is transactional: the bound pos and vel and the integrator state are saved first, and
 * any error inside the step (TG_ERR_OOM, TG_ERR_CAPACITY, ...) restores them before returning.
 * TG_ERR_NONFINITE (nothing changed) if a bound position or mass is not finite at the start.
 * Synchronising (the recursion reads the set sizes of each split). */
tg_status tg_hhs_step(tg_ctx *ctx);
/* Ensemble of independent systems: one rung-0 HOLD step of every context in ctxs[0..count) as ONE
 * CUDA graph launch.  Each context must be bound by tg_hhs_init, created with params.batched = 1, on the
 * current device and with the same stream as ctxs[0]; no context may appear twice.  The graph holds
 * every system's own work-queue loop (Algorithms 1-2, its own rungs) side by side with no dependencies
 * between them, so the systems run side by side on the GPU; the host waits once for all of them.  Per
 * system the step is transactional: a system whose buffers overflow is restored and redone alone; one
 * whose loop runs out is restored and reported (TG_ERR_TIMEOUT); the other systems keep their step.
 * The graph is captured on the first call and again when the members or their buffers change.
 * Errors are reported on ctxs[0] (tg_last_error).  Synchronising. */
tg_status tg_ensemble_step(tg_ctx **ctxs, int count);

/* The traditional integrator with individual timesteps that the paper sets beside HHS (Sec. 2.3),
 * on the same FMM.  tg_trad_init binds pos/vel/mass like tg_hhs_init (caller-owned device float64
 * SoA), evaluates the forces and picks the first rungs from dt_i = sqrt(eta eps / |a_i|).
 * tg_trad_step advances every particle by params.dt_max: block steps dt_max / 2^rung with
 * kick-drift-kick per particle; at the end of a particle's step it drifts, gets its force from all
 * masses at their stored positions (inactive particles are not synchronised), closes with a half
 * kick, takes a new rung (deepened until the next step starts on a multiple of itself, at most
 * k_max) and opens the next step.  No reaction reaches the sources, so momentum is not conserved:
 * this is the paper's comparison scheme.  Each boundary is one evaluation of the whole system;
 * tg_stats.sink_forces counts the active particles.  Synchronising (one read per boundary).
 * TG_ERR_STATE for tg_trad_step without tg_trad_init (tg_hhs_step likewise needs tg_hhs_init). */
tg_status tg_trad_init(tg_ctx *ctx, int64_t n, double *pos, double *vel, const double *mass);
tg_status tg_trad_step(tg_ctx *ctx);
/* Per-particle HHS state (device outputs, each nullable): rung (int32 n), |a_old|, |a_current|
 * and |a|_tot of Eq. (9) (float64 n).  After tg_trad_init only the rungs are kept; the other
 * arrays are written as zero.  Synchronising. */
tg_status tg_hhs_state(tg_ctx *ctx, int32_t *rung, double *a_old, double *a_cur, double *a_tot);
/* Set the per-particle |a_old|, |a_current| and (nullable) |a|_tot (device float64 n each). */
tg_status tg_hhs_set_accel(tg_ctx *ctx, const double *a_old, const double *a_cur, const double *a_tot);

/* Conservation diagnostics of the bound HHS system (Sec. 3.2): out[0..2] = total momentum
 * sum m v, out[3..5] = angular momentum sum m x cross v, out[6] = total energy
 * sum m v^2/2 + sum m phi/2 (phi from a fresh all-from-all evaluation), out[7] = time.
 * float64 device reductions.  Synchronising; out is host memory. */
tg_status tg_diagnostics(tg_ctx *ctx, double out[8]);

/* Checkpoint and resume of the HHS run (the integrator state of Algorithms 1-3 between two
 * rung-0 steps; the paper has no file format, this one is the library's own).
 * tg_checkpoint writes, to the host file `path`, the bound system and its integrator state:
 * n, the tg_params of the context, the time, pos (3n), vel (3n), mass (n), |a_old| (n),
 * |a_current| (n), |a|_tot (n) (float64) and the rungs (n, int32), followed by a 64-bit FNV-1a checksum of
 * everything before it.  It goes through a temporary file renamed over `path`.  Synchronising;
 * the device arrays are left unchanged.  TG_ERR_STATE before tg_hhs_init, TG_ERR_IO if the file
 * cannot be written.
 * tg_restore reads such a file into a context created with equal tg_params on which
 * tg_hhs_init has bound a system of the same n: it overwrites pos and vel (the caller's arrays
 * bound by tg_hhs_init), the integrator state and the time.  The masses in the file must equal
 * the bound masses bit for bit.  TG_ERR_IO for a missing, short or corrupt file; TG_ERR_STATE
 * before tg_hhs_init or when n, the parameters or the masses differ (nothing is changed then).
 * Synchronising. */
tg_status tg_checkpoint(tg_ctx *ctx, const char *path);
tg_status tg_restore(tg_ctx *ctx, const char *path);

/* ---- test hooks (synchronising; outputs are HOST memory sized by the *_count calls) ---- */

/* Geometry of the last tree: lo[3], L (root cube side), n, number of cells. */
tg_status tg_tree_info(tg_ctx *ctx, double lo[3], double *L, int64_t *n, int64_t *n_cells);
/* Sorted keys (uint64 n), permutation (int64 n: sorted position -> particle index) and cells
 * (level int32, integer coords int64 3*nc SoA, first/count int64 nc, nchild int32 nc). */
tg_status tg_get_tree(tg_ctx *ctx, uint64_t *keys, int64_t *perm, int32_t *level, int64_t *coords,
                      int64_t *first, int64_t *count, int32_t *nchild);
/* Unordered interaction lists of the last walk (cell ids as in tg_get_tree): counts first,
 * then pairs (int64 a[], b[]). */
tg_status tg_list_counts(tg_ctx *ctx, int64_t *n_m2l, int64_t *n_p2p);
tg_status tg_get_lists(tg_ctx *ctx, int64_t *m2l_a, int64_t *m2l_b, int64_t *p2p_a, int64_t *p2p_b);

/* Failure injection and capacity control for tests of the error paths (host side only; nothing
 * here makes a kernel fault).  what:
 *   TG_DEBUG_FAIL_ALLOC      value >= 0: after `value` more successful scratch allocations of this
 *                            context, every further one fails as if cudaMalloc had (TG_ERR_OOM);
 *                            value < 0 switches the injection off.
 *   TG_DEBUG_LIST_CAPACITY   value > 0: the walk's per-cell estimates of the interaction-list sizes
 *                            are set to value / 1000 (tiny values force the regrowth path: the
 *                            lists are sized from the estimates, overflow, and the walk is re-run
 *                            with larger buffers; tg_stats.list_regrowths counts the re-runs).
 *   TG_DEBUG_QUEUE_LIMIT     value >= 0: iteration limit of the batched step's device loop
 *                            (0 restores the default, 8 * 2^min(k_max, 22) + 64).
 *   TG_DEBUG_QUEUE_HOLD      value != 0: the batched step's scheduler publishes no operation, so the
 *                            loop spins idle until its limit and the step returns TG_ERR_TIMEOUT
 *                            with the state restored (the bounded wait's own failure path).
 *   TG_DEBUG_BATCH_CAPS      value > 0: the next sizing of the batched step starts its list
 *                            capacities at `value` entries and its cell capacity at max(value, 64),
 *                            so that the step overflows, restores the state and regrows.
 * TG_ERR_ARG for an unknown `what`.  Not synchronising. */
typedef enum { TG_DEBUG_FAIL_ALLOC = 1, TG_DEBUG_LIST_CAPACITY = 2, TG_DEBUG_QUEUE_LIMIT = 3,
               TG_DEBUG_QUEUE_HOLD = 4, TG_DEBUG_BATCH_CAPS = 5 } tg_debug_what;
tg_status tg_debug_control(tg_ctx *ctx, int what, int64_t value);

/* ---- autotuner (the paper has no counterpart: it picks launch shapes and the leaf size of Sec. 2.3
 * for this GPU and this particle distribution) ----
 * tg_autotune times FMM evaluations of the given system (CUDA events on the context's stream, one
 * warm-up, best of two) for candidate settings and keeps the fastest in the context:
 *   n_crit            leaf size: 48, 64, 80, 96, 112, 128, 160, 192 (the tree, and so the results, change within
 *                     the FMM's own accuracy; params.n_crit of the context is replaced)
 *   p2p_rows          rows per lane of the float32 P2P tile: 1, 2, 3 (the same pairs and terms; the float32
 *                     sums are added in another order, so results change only by rounding)
 *   m2l_blocks_per_sm grid of the float32 M2L kernel in blocks per SM: 4, 8, 16, 32 (the same terms; only the
 *                     order of the float32 atomics changes)
 *   m2l_form          float32 M2L with the harmonic set (Wendland kernel): 0 mutual (the default), a
 *                     lane per cell pair of a block, both sides combined across lanes; 1 directed, a
 *                     warp per target cell over its sources (the same terms, summed in another order)
 * searched one after another in that order (each at the best of the ones before).  The objective is
 * the time of one all-from-all evaluation plus, when is_fast is given, one kick-pair evaluation with
 * that fast set (accelerations only, as the HHS kicks ask).  pos: device 3*n float64, mass: device n
 * float64, is_fast: device n uint8 or NULL.
 * With pos = mass = is_fast = NULL (n = 0 or the bound size) the objective is instead one rung-0 HOLD
 * step of the system bound by tg_hhs_init (Algorithm 1, batched or plain as params.batched says),
 * timed after one untimed step at the same setting: a step's evaluations run from the whole system down
 * to the deepest rung's, so its best leaf size can differ from the largest evaluation's.  The bound
 * pos, vel, |a| bookkeeping, rungs and time are saved first and put back after every step and at the
 * end; TG_ERR_STATE without a bound system.
 * out (host, nullable) receives the choice.  Synchronising; leaves every caller array as it found it.
 * The float64 path has no tunable launch shapes: only n_crit is searched.
 * tg_get_tuning reports the settings in use (the defaults before any tuning). */
typedef struct {
    int n_crit;              /* leaf size in use                                                 */
    int p2p_rows;            /* rows per lane of the float32 P2P tile                            */
    int m2l_blocks_per_sm;   /* float32 M2L grid, blocks per SM                                  */
    int m2l_form;            /* float32 harmonic M2L: 0 mutual blocks, 1 directed by target cell   */
    int candidates;          /* settings timed by the last tg_autotune (0: never tuned)           */
    double objective_ms;     /* objective at the chosen settings                                 */
    double objective_ms_initial; /* objective at the settings the context had before tuning      */
} tg_tuning;
tg_status tg_autotune(tg_ctx *ctx, int64_t n, const double *pos, const double *mass, const uint8_t *is_fast,
                      tg_tuning *out);
tg_status tg_get_tuning(const tg_ctx *ctx, tg_tuning *out);
/* Apply settings found by tg_autotune on another context (n_crit 1..256, p2p_rows 1..3,
 * m2l_blocks_per_sm 1..64; the other fields are ignored).  TG_ERR_ARG for values out of range. */
tg_status tg_set_tuning(tg_ctx *ctx, const tg_tuning *in);

/* ---- live kernel timing (CUDA events on the context's stream) ---- */
typedef enum {
    TG_K_TREE = 0,   /* root cube, Morton keys, radix sort, gather, octree build            */
    TG_K_UP = 1,     /* leaf offsets, P2M, M2M                                             */
    TG_K_WALK = 2,   /* dual tree walk (Algorithm 4)                                        */
    TG_K_M2L = 3,    /* mutual cell-cell interaction                                        */
    TG_K_P2P = 4,    /* mutual particle-particle interaction                                */
    TG_K_DOWN = 5,   /* L2L, L2P, scatter to caller order                                   */
    TG_K_HHS = 6,    /* timestep, split, kick, drift                                        */
    TG_K_OTHER = 7,  /* scans, reductions, direct summation                                 */
    TG_K_COUNT = 8
} tg_kernel_class;

typedef struct {
    double ms[TG_K_COUNT];        /* summed event time per class (classes being timed only)  */
    int64_t launches[TG_K_COUNT]; /* kernel launches per class (always counted)              */
} tg_profile;

/* level 0: off; 1: time the M2L and P2P launches; 2: time every launch.  Launch counts are
 * always kept.  Timing adds an event record before and after each timed launch. */
tg_status tg_set_profiling(tg_ctx *ctx, int level);
/* Totals since the last tg_reset_stats.  Synchronising. */
tg_status tg_get_profile(tg_ctx *ctx, tg_profile *out);

/* Timestep kernel alone (Sec. 2.2): dt[i] = sqrt(eta*eps/(a_old[i] + a_cur[i])), with a_tot
 * given (nullable) and params.eta_tot > 0 capped by Eq. (9): min(dt[i], sqrt(eta_tot*eps/a_tot[i])),
 * and rung[i] = smallest k with dt_max/2^k <= dt[i], capped at k_max.  Device arrays. */
tg_status tg_timesteps(tg_ctx *ctx, int64_t n, const double *a_old, const double *a_cur, const double *a_tot,
                       double *dt, int32_t *rung);

/* ---- allocation-free variant (the paper has no counterpart; this is a library service) ----
 *
 * For callers that must not allocate device memory: applications whose GPU memory is owned by
 * another allocator or held to a fixed budget, and loops that cannot take the device-wide
 * synchronisation a cudaMalloc can cause.  Creating a context allocates, so this call needs no
 * context.  It computes what tg_build_tree computes first -- the root cube, the Morton keys and
 * the stable (key, particle index) radix sort -- and returns the sorted keys and permutation.
 *
 *   n        number of particles, 0 <= n <= TG_NOALLOC_MAX_N; larger n returns TG_ERR_ARG
 *   pos      device, 3*n float64 (SoA x, y, z), read only
 *   keys_out device, n uint64 output: Morton keys in sorted order
 *   perm_out device, n int64 output: perm_out[s] = index of the particle at sorted position s
 *   cuda_stream  the cudaStream_t the work is enqueued on (NULL = legacy default stream)
 *
 * It allocates nothing (no cudaMalloc, cudaFree or allocating library call).  Its scratch is one
 * file-scope device array of about 6.3 MB that every GPU loading the library holds until the
 * process exits.  Every call looks up that array's device address (cudaGetSymbolAddress, which
 * allocates nothing) on the current device, so pos, keys_out and perm_out must be memory of the
 * current device (or managed memory).  All calls share the array, so two calls whose work
 * overlaps on the GPU (different streams, or host threads racing) corrupt each other's results:
 * serialise them.  Returns TG_ERR_ARG for bad sizes or for pointers that are not memory of the
 * current device, and TG_ERR_CUDA if a launch fails; the call is asynchronous otherwise. */
#define TG_NOALLOC_MAX_N 262144
tg_status tg_morton_sort_noalloc(int64_t n, const double *pos, uint64_t *keys_out, int64_t *perm_out,
                                 void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
