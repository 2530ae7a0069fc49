/*
 * taichi_oracle.h -- plain FP64 CPU oracle of the momentum-conserving FMM + HHS scheme
 * (Zhu 2017, "A momentum conserving N-body scheme with individual timesteps").
 *
 * TEST INFRASTRUCTURE ONLY.  This code exists to check the CUDA path; it is slow on
 * purpose and shares no code, header, table or helper with it.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Conventions (all arrays are host memory owned by the caller):
 *   positions / velocities / accelerations are SoA: x[n], y[n], z[n];
 *   G = 1; the potential is negative (phi = -m/r far from a source);
 *   is_fast (nullable) marks the fast set F of a kick pair; NULL = every particle slow.
 *   With is_fast given, slow sinks feel every mass and fast sinks feel slow masses
 *   only (one kickFS2S + one kickS2F of Algorithm 2/3 evaluated on one tree).
 */
#ifndef TAICHI_ORACLE_H
#define TAICHI_ORACLE_H
#include <stdint.h>

#define ORC_PMAX 20
#define ORC_MAX_LEVEL 21

enum { ORC_WENDLAND_C2 = 0, ORC_PLUMMER = 1 };

typedef struct {
    int p;            /* expansion order (total degree of the Taylor terms kept) */
    int n_crit;       /* a cell with more than n_crit particles is split         */
    int kernel;       /* ORC_WENDLAND_C2 or ORC_PLUMMER                            */
    int max_level;    /* deepest octree level, <= 21                              */
    double theta;     /* opening angle of the MAC, Eq. (1)                        */
    double kappa;     /* R = kappa * cell side in Eq. (1)                          */
    double eps;       /* softening length                                          */
    int mac;          /* 0: R = kappa * side (the paper's Eq. 1); 1: R = radius of a  */
                      /* sphere about the cell centre enclosing its particles        */
} orc_params;

typedef struct {
    double eta;       /* timestep parameter of dt_i = sqrt(eta*eps/|a|)           */
    double dt_max;    /* step of rung 0                                            */
    int k_max;        /* deepest rung                                              */
    double eta_tot;   /* eta_1 of the Eq. (9) minimum-timestep constraint; 0 = off */
} orc_hhs_params;

#ifdef __cplusplus
extern "C" {
#endif

int orc_num_coeffs(int p);
void orc_multi_index(int idx, int *nx, int *ny, int *nz);

void orc_softened(int kernel, double eps, double r, double *phi, double *g);
void orc_dtensor(int p, const double d[3], int kernel, double eps, double *D);

void orc_direct(int64_t n, const double *x, const double *y, const double *z,
                const double *m, const uint8_t *is_fast, int kernel, double eps,
                int64_t n_sink, const int64_t *sink_idx,
                double *ax, double *ay, double *az, double *pot);

int orc_root_cube(int64_t n, const double *x, const double *y, const double *z,
                  double lo[3], double *L);
void orc_morton_keys(int64_t n, const double *x, const double *y, const double *z,
                     const double lo[3], double L, uint64_t *keys);
void orc_sort_keys(int64_t n, const uint64_t *keys, int64_t *perm);

/* Octree + interaction lists of one evaluation, for tests.  Cells are in BFS order. */
typedef struct orc_tree orc_tree;
orc_tree *orc_tree_build(int64_t n, const double *x, const double *y, const double *z,
                         const orc_params *prm);
void orc_tree_free(orc_tree *t);
int64_t orc_tree_ncell(const orc_tree *t);
void orc_tree_cells(const orc_tree *t, int32_t *level, int64_t *cx, int64_t *cy, int64_t *cz,
                    int64_t *first, int64_t *count, int64_t *child_first, int32_t *nchild);
void orc_tree_perm(const orc_tree *t, int64_t *perm, uint64_t *sorted_keys);
void orc_tree_geometry(const orc_tree *t, double lo[3], double *L);
/* Algorithm 4 from (root, root); directed lists.  Returns counts; pass NULL to query. */
void orc_tree_walk(orc_tree *t, int64_t *n_m2l, int64_t *n_p2p);
void orc_tree_lists(const orc_tree *t, int64_t *m2l_a, int64_t *m2l_b, int64_t *p2p_a, int64_t *p2p_b);
int orc_well_separated(const orc_tree *t, int64_t a, int64_t b);
/* enclosing radius of every cell (used by mac = 1): leaves the largest particle distance from the
 * cell centre, parents max over children of (|z_child - z_parent| + R_child) */
void orc_tree_radii(const orc_tree *t, double *r);

/* expansion operators on one cell (for pinning): coefficient arrays of length orc_num_coeffs(p) */
void orc_p2m(int p, int64_t n, const double *x, const double *y, const double *z, const double *m,
             const double zc[3], double *M);
void orc_m2m(int p, const double *Mc, const double delta[3], double *Mp);
void orc_m2l(int p, const double *MB, const double d[3], int kernel, double eps, double *LA);
void orc_l2l(int p, const double *Lp, const double delta[3], double *Lc);
void orc_l2p(int p, const double *L, const double rho[3], double *phi, double a[3]);

/* Full FMM evaluation, directed, per sink cell. */
int orc_fmm(int64_t n, const double *x, const double *y, const double *z, const double *m,
            const uint8_t *is_fast, const orc_params *prm,
            double *ax, double *ay, double *az, double *pot);
/* Same evaluation, but only for the sinks listed in sample (computed one by one). */
int orc_fmm_sample(int64_t n, const double *x, const double *y, const double *z, const double *m,
                   const uint8_t *is_fast, const orc_params *prm,
                   int64_t n_sample, const int64_t *sample,
                   double *ax, double *ay, double *az, double *pot);

/* Timestep function of Sec. 2.2 and the rung of a particle. */
double orc_timestep(double eta, double eps, double a_old, double a_cur);
/* The same with the minimum-timestep constraint of Eq. (9): min(dt_i, sqrt(eta_tot eps / |a|_tot)),
 * |a|_tot the acceleration from all particles; eta_tot <= 0 or |a|_tot <= 0 leaves dt_i alone. */
double orc_timestep_tot(double eta, double eps, double a_old, double a_cur, double eta_tot, double a_tot);
int orc_rung(double dt_i, double dt_max, int k_max);

/* HHS / HOLD integrator, Algorithms 1-3, with the two masked Poisson calls per kick pair. */
typedef struct {
    int64_t poisson_calls;   /* Poisson-solver calls made (each masked call counts once) */
    int64_t sink_forces;     /* sum over calls of the number of sinks that received forces */
    int64_t kdk_frames;      /* number of KDK frames executed                                */
    int32_t max_rung;        /* deepest rung that held a slow particle                      */
    int32_t trace_len;       /* entries written to trace                                    */
} orc_hhs_stats;

/* a_tot (nullable): |a| of every particle from all masses, as kept for Eq. (9). */
int orc_hhs_init(int64_t n, const double *x, const double *y, const double *z, const double *m,
                 const orc_params *prm, double *a_old, double *a_cur, double *a_tot);
/* One rung-0 step of EVOLVE_HOLD.  trace (nullable, capacity trace_cap entries of 4 int64):
 * (kind, rung, n_sinks, n_sources) per Poisson call, kind 0 = kickS2F, 1 = kickFS2S; drifts are
 * recorded as kind 2 with (2, rung, n_slow, 0).  a_tot (nullable): the second kickFS2S of rung 0
 * passes the whole system to the Poisson solver with all masses, and records |a| of every particle
 * of it there; with hp->eta_tot > 0 the timesteps then follow orc_timestep_tot. */
int orc_hhs_step(int64_t n, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                 const double *m, const orc_params *prm, const orc_hhs_params *hp,
                 double *a_old, double *a_cur, double *a_tot, int32_t *rung_out,
                 orc_hhs_stats *stats, int64_t *trace, int32_t trace_cap);

/* The traditional integrator with individual (block) timesteps that the paper sets beside HHS
 * (Sec. 2.3): each particle steps dt_max / 2^rung with kick-drift-kick over its own step; at the end
 * of a particle's step it drifts, gets its force from all masses at their stored positions (the
 * inactive particles' positions are not synchronised to the current time), closes its step with a
 * half kick, takes a new rung from dt_i = sqrt(eta eps / |a_i|) (deepened until its step starts on
 * a multiple of the new step; at most k_max) and opens the next step with a half kick.  One call
 * advances all particles by dt_max (every rung then ends together).
 * acc (3n, x then y then z) and rung hold the state between calls: orc_trad_init evaluates the
 * forces and picks the first rungs; the opening half kicks happen at the start of each step.
 * stats (nullable): poisson_calls counts the force evaluations, sink_forces the active particles. */
int orc_trad_init(int64_t n, const double *x, const double *y, const double *z, const double *m,
                  const orc_params *prm, const orc_hhs_params *hp, double *acc, int32_t *rung);
int orc_trad_step(int64_t n, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                  const double *m, const orc_params *prm, const orc_hhs_params *hp,
                  double *acc, int32_t *rung, orc_hhs_stats *stats);

void orc_diagnostics(int64_t n, const double *x, const double *y, const double *z,
                     const double *vx, const double *vy, const double *vz,
                     const double *m, const double *pot, double out[7]);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
