/*
 * taichi_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * A slow, direct restatement of what the method computes, written from the paper
 * (Zhu 2017) and the published methods it builds on.  It is never on the product path:
 * only tests, the smoke check and the benchmark's CPU-baseline leg load it.  It shares no
 * code with the CUDA library.
 *
 * Sections followed:
 *   Sec. 2.1, Eq. (1)      multipole acceptance criterion |z_A - z_B| > (R_A + R_B)/theta
 *   Sec. 2.1, Eq. (2)      F_ij = -F_ji (mutual forces)
 *   Sec. 2.3, Eq. (8)      Wendland C2 softened potential
 *   Sec. 2.3               octree with n_crit, "open both cells", softening-distance rule
 *   Sec. 2.3, Algorithm 4  dual tree walk GET_INTERACTION_LIST
 *   Sec. 2.2, Algorithms 1-3  HOLD integrator: split, KDK, masked kicks, timestep function
 * Expansions are Cartesian Taylor series truncated at total degree p (the paper's solver
 * uses spherical harmonics; for G = -1/r both truncations give the same approximation).
 * Derivative tensors follow the McMurchie & Davidson (1978) auxiliary recurrence.
 *
 * Readings of points the paper leaves open:
 *   R in Eq. (1) = kappa * side (kappa = 1: the paper calls R the cell side length), or with mac = 1
 *   the radius of a sphere about the cell centre that encloses the cell's particles;
 *   a cell is split iff it holds more than n_crit particles (leaves hold <= n_crit);
 *   expansion centres are geometric cell centres;
 *   "distance larger than eps" = the gap between the two cubes exceeds eps (Wendland only);
 *   Algorithm 4's well_seperated(Ci, Ci) is read as well_seperated(Ci, Cj);
 *   self-interaction is excluded from the potential.
 *
 * Compile with -ffp-contract=off so results do not depend on FMA contraction.
 */
#include "taichi_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------------------ */
/* Multi-indices n = (nx, ny, nz) with |n| <= ORC_PMAX, ordered by total degree, then   */
/* nx descending, then ny descending.  The first orc_num_coeffs(p) entries are |n|<=p.  */
/* ------------------------------------------------------------------------------------ */
#define MI_TOTAL (((ORC_PMAX + 1) * (ORC_PMAX + 2) * (ORC_PMAX + 3)) / 6)
static int mi_x[MI_TOTAL], mi_y[MI_TOTAL], mi_z[MI_TOTAL];
static int mi_lookup[ORC_PMAX + 1][ORC_PMAX + 1][ORC_PMAX + 1];
static double fact_tab[2 * ORC_PMAX + 2];
static int mi_ready = 0;

static void mi_init(void)
{
    if (mi_ready) return;
    int c = 0;
    for (int o = 0; o <= ORC_PMAX; ++o)
        for (int nx = o; nx >= 0; --nx)
            for (int ny = o - nx; ny >= 0; --ny) {
                int nz = o - nx - ny;
                mi_x[c] = nx; mi_y[c] = ny; mi_z[c] = nz;
                mi_lookup[nx][ny][nz] = c;
                ++c;
            }
    fact_tab[0] = 1.0;
    for (int i = 1; i < 2 * ORC_PMAX + 2; ++i) fact_tab[i] = fact_tab[i - 1] * i;
    mi_ready = 1;
}

int orc_num_coeffs(int p) { return ((p + 1) * (p + 2) * (p + 3)) / 6; }

void orc_multi_index(int idx, int *nx, int *ny, int *nz)
{
    mi_init();
    *nx = mi_x[idx]; *ny = mi_y[idx]; *nz = mi_z[idx];
}

static int mi_order(int i) { return mi_x[i] + mi_y[i] + mi_z[i]; }
static int mi_of(int nx, int ny, int nz) { return mi_lookup[nx][ny][nz]; }
static double mi_fact(int i) { return fact_tab[mi_x[i]] * fact_tab[mi_y[i]] * fact_tab[mi_z[i]]; }

static double ipow(double b, int e)
{
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

/* x^n for a multi-index n */
static double mono(const double v[3], int i) { return ipow(v[0], mi_x[i]) * ipow(v[1], mi_y[i]) * ipow(v[2], mi_z[i]); }

static double binom(int n, int k)
{
    return fact_tab[n] / (fact_tab[k] * fact_tab[n - k]);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------------------ */
/* Pair kernels.  phi(r) is the potential of a unit mass (negative), g(r) = phi'(r)/r so */
/* that the acceleration of i due to j is m_j g(r) (x_j - x_i).                          */
/* ------------------------------------------------------------------------------------ */
void orc_softened(int kernel, double eps, double r, double *phi, double *g)
{
    if (kernel == ORC_PLUMMER) {
        double s2 = r * r + eps * eps;
        double s = sqrt(s2);
        *phi = -1.0 / s;
        *g = 1.0 / (s2 * s);
        return;
    }
    /* Wendland C2, Eq. (8): for u = r/eps < 1,
     *   phi = (1/eps) (3u^7 - 15u^6 + 28u^5 - 21u^4 + 7u^2 - 3),
     *   phi'(r) = (1/eps^2) (21u^6 - 90u^5 + 140u^4 - 84u^3 + 14u),  g = phi'/r.
     * Beyond eps the potential is the Newtonian -1/r. */
    if (r < eps) {
        double u = r / eps;
        double u2 = u * u, u3 = u2 * u, u4 = u2 * u2, u5 = u4 * u, u6 = u3 * u3, u7 = u6 * u;
        *phi = (3.0 * u7 - 15.0 * u6 + 28.0 * u5 - 21.0 * u4 + 7.0 * u2 - 3.0) / eps;
        *g = (21.0 * u5 - 90.0 * u4 + 140.0 * u3 - 84.0 * u2 + 14.0) / (eps * eps * eps);
    } else {
        *phi = -1.0 / r;
        *g = 1.0 / (r * r * r);
    }
}

/* Direct O(N^2) summation (ground truth).  Slow sinks feel every mass, fast sinks feel
 * slow masses only; i = j is skipped. */
void orc_direct(int64_t n, const double *x, const double *y, const double *z,
                const double *m, const uint8_t *is_fast, int kernel, double eps,
                int64_t n_sink, const int64_t *sink_idx,
                double *ax, double *ay, double *az, double *pot)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < n_sink; ++s) {
        int64_t i = sink_idx ? sink_idx[s] : s;
        double sx = 0, sy = 0, sz = 0, sp = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (is_fast && is_fast[i] && is_fast[j]) continue;
            double dx = x[j] - x[i], dy = y[j] - y[i], dz = z[j] - z[i];
            double r = sqrt(dx * dx + dy * dy + dz * dz);
            double phi, g;
            orc_softened(kernel, eps, r, &phi, &g);
            sx += m[j] * g * dx; sy += m[j] * g * dy; sz += m[j] * g * dz;
            sp += m[j] * phi;
        }
        ax[s] = sx; ay[s] = sy; az[s] = sz;
        if (pot) pot[s] = sp;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Derivative tensor D^k(d) = d^k G / dd^k, |k| <= p.                                   */
/* G(d) = -1/|d| (Newton) or -(|d|^2 + eps^2)^(-1/2) (Plummer).  With rho = |d|^2/2 and */
/* f_m = h^(m)(rho), h(rho) = G: R^(m)_0 = f_m, R^(m)_{k+e_a} = d_a R^(m+1)_k +          */
/* k_a R^(m+1)_{k-e_a}, D^k = R^(0)_k  (McMurchie & Davidson 1978).                      */
/* For h = -(2 rho + c)^(-1/2): f_m = -(-1)^m (2m-1)!! s^-(2m+1), s = sqrt(|d|^2 + c).   */
/* ------------------------------------------------------------------------------------ */
void orc_dtensor(int p, const double d[3], int kernel, double eps, double *D)
{
    mi_init();
    int nc = orc_num_coeffs(p);
    double *R = (double *)malloc(sizeof(double) * (size_t)(p + 1) * nc);
    double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (kernel == ORC_PLUMMER) s2 += eps * eps;
    double sinv = 1.0 / sqrt(s2);
    double sinv2 = sinv * sinv;
    double f = -sinv;              /* m = 0 */
    for (int m = 0; m <= p; ++m) {
        R[(size_t)m * nc + 0] = f;
        f = -f * (2.0 * m + 1.0) * sinv2;   /* f_{m+1} = -(2m+1) f_m / s^2 */
    }
    for (int k = 1; k < nc; ++k) {
        int kx = mi_x[k], ky = mi_y[k], kz = mi_z[k];
        int a, ka, km, kmm = -1;
        if (kx > 0) { a = 0; ka = kx; km = mi_of(kx - 1, ky, kz); if (kx >= 2) kmm = mi_of(kx - 2, ky, kz); }
        else if (ky > 0) { a = 1; ka = ky; km = mi_of(kx, ky - 1, kz); if (ky >= 2) kmm = mi_of(kx, ky - 2, kz); }
        else { a = 2; ka = kz; km = mi_of(kx, ky, kz - 1); if (kz >= 2) kmm = mi_of(kx, ky, kz - 2); }
        int o = kx + ky + kz;
        for (int m = 0; m <= p - o; ++m) {
            double v = d[a] * R[(size_t)(m + 1) * nc + km];
            if (kmm >= 0) v += (double)(ka - 1) * R[(size_t)(m + 1) * nc + kmm];
            R[(size_t)m * nc + k] = v;
        }
    }
    for (int k = 0; k < nc; ++k) D[k] = R[k];
    free(R);
}

/* ------------------------------------------------------------------------------------ */
/* Expansion operators (Cartesian, total degree <= p).                                   */
/*   M^j = sum_i m_i (x_i - z)^j                                                        */
/*   phi(x) = sum_n L^n (x - z)^n / n!                                                  */
/* ------------------------------------------------------------------------------------ */
void orc_p2m(int p, int64_t n, const double *x, const double *y, const double *z, const double *m,
             const double zc[3], double *M)
{
    mi_init();
    int nc = orc_num_coeffs(p);
    for (int k = 0; k < nc; ++k) M[k] = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r[3] = {x[i] - zc[0], y[i] - zc[1], z[i] - zc[2]};
        for (int k = 0; k < nc; ++k) M[k] += m[i] * mono(r, k);
    }
}

/* Mp^n += sum_{k <= n} C(n,k) delta^(n-k) Mc^k, delta = z_child - z_parent */
void orc_m2m(int p, const double *Mc, const double delta[3], double *Mp)
{
    mi_init();
    int nc = orc_num_coeffs(p);
    for (int n = 0; n < nc; ++n) {
        double s = 0.0;
        for (int k = 0; k < nc; ++k) {
            if (mi_x[k] > mi_x[n] || mi_y[k] > mi_y[n] || mi_z[k] > mi_z[n]) continue;
            int dx = mi_x[n] - mi_x[k], dy = mi_y[n] - mi_y[k], dz = mi_z[n] - mi_z[k];
            double c = binom(mi_x[n], mi_x[k]) * binom(mi_y[n], mi_y[k]) * binom(mi_z[n], mi_z[k]);
            s += c * ipow(delta[0], dx) * ipow(delta[1], dy) * ipow(delta[2], dz) * Mc[k];
        }
        Mp[n] += s;
    }
}

/* Directed M2L, source cell B -> sink cell A, d = z_A - z_B:
 *   L_A^n += sum_{|j| <= p-|n|} (-1)^|j| / j!  M_B^j  D^{n+j}(d).
 * (Taylor expansion of G(x - y) about d, with x - z_A and y - z_B small.) */
void orc_m2l(int p, const double *MB, const double d[3], int kernel, double eps, double *LA)
{
    mi_init();
    int nc = orc_num_coeffs(p);
    double *D = (double *)malloc(sizeof(double) * nc);
    orc_dtensor(p, d, kernel, eps, D);
    for (int n = 0; n < nc; ++n) {
        double s = 0.0;
        int on = mi_order(n);
        for (int j = 0; j < nc; ++j) {
            int oj = mi_order(j);
            if (on + oj > p) continue;
            double sign = (oj & 1) ? -1.0 : 1.0;
            int nj = mi_of(mi_x[n] + mi_x[j], mi_y[n] + mi_y[j], mi_z[n] + mi_z[j]);
            s += sign / mi_fact(j) * MB[j] * D[nj];
        }
        LA[n] += s;
    }
    free(D);
}

/* Lc^n += sum_{k >= n, |k| <= p} Lp^k delta^(k-n) / (k-n)!, delta = z_child - z_parent */
void orc_l2l(int p, const double *Lp, const double delta[3], double *Lc)
{
    mi_init();
    int nc = orc_num_coeffs(p);
    for (int n = 0; n < nc; ++n) {
        double s = 0.0;
        for (int k = 0; k < nc; ++k) {
            if (mi_x[k] < mi_x[n] || mi_y[k] < mi_y[n] || mi_z[k] < mi_z[n]) continue;
            int dx = mi_x[k] - mi_x[n], dy = mi_y[k] - mi_y[n], dz = mi_z[k] - mi_z[n];
            s += Lp[k] * ipow(delta[0], dx) * ipow(delta[1], dy) * ipow(delta[2], dz)
                 / (fact_tab[dx] * fact_tab[dy] * fact_tab[dz]);
        }
        Lc[n] += s;
    }
}

/* phi = sum_n L^n rho^n/n!;  a = -grad phi:  a_e = -sum_{|m| <= p-1} L^{m+e} rho^m/m! */
void orc_l2p(int p, const double *L, const double rho[3], double *phi, double a[3])
{
    mi_init();
    int nc = orc_num_coeffs(p);
    double ph = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int n = 0; n < nc; ++n) {
        double t = mono(rho, n) / mi_fact(n);
        ph += L[n] * t;
        if (mi_order(n) <= p - 1) {
            gx += L[mi_of(mi_x[n] + 1, mi_y[n], mi_z[n])] * t;
            gy += L[mi_of(mi_x[n], mi_y[n] + 1, mi_z[n])] * t;
            gz += L[mi_of(mi_x[n], mi_y[n], mi_z[n] + 1)] * t;
        }
    }
    *phi = ph;
    a[0] = -gx; a[1] = -gy; a[2] = -gz;
}

/* ------------------------------------------------------------------------------------ */
/* Root cube and Morton keys.                                                           */
/*   L = smallest power of two >= (largest bbox extent) * (1 + 2^-20)  (1 if extent 0)  */
/*   h = L / 2^21, lo_k = floor(min_k / h) * h                                          */
/*   integer coordinate c_k = floor((x_k - lo_k) * 2^21 / L) clamped to [0, 2^21 - 1]  */
/*   key = bit-interleave, x the most significant bit of each 3-bit group              */
/* ------------------------------------------------------------------------------------ */
int orc_root_cube(int64_t n, const double *x, const double *y, const double *z, double lo[3], double *L)
{
    if (n <= 0) { lo[0] = lo[1] = lo[2] = 0.0; *L = 1.0; return 0; }
    double mn[3] = {x[0], y[0], z[0]}, mx[3] = {x[0], y[0], z[0]};
    for (int64_t i = 1; i < n; ++i) {
        const double v[3] = {x[i], y[i], z[i]};
        for (int k = 0; k < 3; ++k) {
            if (v[k] < mn[k]) mn[k] = v[k];
            if (v[k] > mx[k]) mx[k] = v[k];
        }
    }
    double ext = 0.0;
    for (int k = 0; k < 3; ++k) {
        double e = mx[k] - mn[k];
        if (e > ext) ext = e;
    }
    double Lv = 1.0;
    if (ext > 0.0) {
        double t = ext * (1.0 + ldexp(1.0, -20));
        int e;
        double f = frexp(t, &e);          /* t = f 2^e, f in [0.5, 1) */
        Lv = (f == 0.5) ? t : ldexp(1.0, e);
    }
    double h = ldexp(Lv, -ORC_MAX_LEVEL);
    for (int k = 0; k < 3; ++k) lo[k] = floor(mn[k] / h) * h;
    *L = Lv;
    return 0;
}

static uint64_t spread3(uint64_t v)
{
    uint64_t r = 0;
    for (int b = 0; b < ORC_MAX_LEVEL; ++b) r |= ((v >> b) & 1ull) << (3 * b);
    return r;
}

static uint64_t cell_coord(double xv, double lo, double inv_h)
{
    double t = floor((xv - lo) * inv_h);
    if (t < 0.0) t = 0.0;
    double top = (double)((1 << ORC_MAX_LEVEL) - 1);
    if (t > top) t = top;
    return (uint64_t)t;
}

void orc_morton_keys(int64_t n, const double *x, const double *y, const double *z,
                     const double lo[3], double L, uint64_t *keys)
{
    double inv_h = ldexp(1.0 / L, ORC_MAX_LEVEL);   /* exact: L is a power of two */
    for (int64_t i = 0; i < n; ++i) {
        uint64_t cx = cell_coord(x[i], lo[0], inv_h);
        uint64_t cy = cell_coord(y[i], lo[1], inv_h);
        uint64_t cz = cell_coord(z[i], lo[2], inv_h);
        keys[i] = (spread3(cx) << 2) | (spread3(cy) << 1) | spread3(cz);
    }
}

static const uint64_t *sort_keys_ptr;
static int cmp_key_index(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    uint64_t ka = sort_keys_ptr[a], kb = sort_keys_ptr[b];
    if (ka < kb) return -1;
    if (ka > kb) return 1;
    return (a < b) ? -1 : (a > b);
}

/* perm[s] = original index of the s-th particle in (key, original index) order */
void orc_sort_keys(int64_t n, const uint64_t *keys, int64_t *perm)
{
    for (int64_t i = 0; i < n; ++i) perm[i] = i;
    sort_keys_ptr = keys;
    qsort(perm, (size_t)n, sizeof(int64_t), cmp_key_index);
}

/* ------------------------------------------------------------------------------------ */
/* Octree (Sec. 2.3): top-down, BFS order; a cell splits iff count > n_crit.            */
/* ------------------------------------------------------------------------------------ */
typedef struct { int64_t *a, *b; int64_t n, cap; } pair_list;

static void pl_push(pair_list *l, int64_t a, int64_t b)
{
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 1024;
        l->a = (int64_t *)realloc(l->a, sizeof(int64_t) * l->cap);
        l->b = (int64_t *)realloc(l->b, sizeof(int64_t) * l->cap);
    }
    l->a[l->n] = a; l->b[l->n] = b; l->n++;
}

struct orc_tree {
    orc_params prm;
    int64_t n;
    double lo[3], L;
    int64_t *perm;          /* sorted position -> original index */
    uint64_t *keys;         /* sorted keys */
    int64_t ncell, cap;
    int32_t *level;
    int64_t *c[3];          /* integer coordinates at the cell's own level */
    int64_t *first, *count, *child_first, *parent;
    int32_t *nchild;
    double *radius;         /* enclosing radius per cell (mac = 1) */
    pair_list m2l, p2p;     /* directed lists from Algorithm 4 */
    int walked;
    /* optional pruning for one-sink evaluation: only cells with on_path set may be the
     * first member of a pair */
    uint8_t *on_path;
};

static int64_t tree_add_cell(orc_tree *t, int lvl, int64_t cx, int64_t cy, int64_t cz,
                             int64_t first, int64_t count, int64_t parent)
{
    if (t->ncell == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 1024;
        t->level = (int32_t *)realloc(t->level, sizeof(int32_t) * t->cap);
        for (int k = 0; k < 3; ++k) t->c[k] = (int64_t *)realloc(t->c[k], sizeof(int64_t) * t->cap);
        t->first = (int64_t *)realloc(t->first, sizeof(int64_t) * t->cap);
        t->count = (int64_t *)realloc(t->count, sizeof(int64_t) * t->cap);
        t->child_first = (int64_t *)realloc(t->child_first, sizeof(int64_t) * t->cap);
        t->parent = (int64_t *)realloc(t->parent, sizeof(int64_t) * t->cap);
        t->nchild = (int32_t *)realloc(t->nchild, sizeof(int32_t) * t->cap);
    }
    int64_t id = t->ncell++;
    t->level[id] = lvl;
    t->c[0][id] = cx; t->c[1][id] = cy; t->c[2][id] = cz;
    t->first[id] = first; t->count[id] = count;
    t->child_first[id] = -1; t->nchild[id] = 0; t->parent[id] = parent;
    return id;
}

orc_tree *orc_tree_build(int64_t n, const double *x, const double *y, const double *z, const orc_params *prm)
{
    mi_init();
    orc_tree *t = (orc_tree *)calloc(1, sizeof(orc_tree));
    t->prm = *prm;
    if (t->prm.max_level > ORC_MAX_LEVEL || t->prm.max_level <= 0) t->prm.max_level = ORC_MAX_LEVEL;
    t->n = n;
    orc_root_cube(n, x, y, z, t->lo, &t->L);
    uint64_t *raw = (uint64_t *)malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    orc_morton_keys(n, x, y, z, t->lo, t->L, raw);
    t->perm = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    orc_sort_keys(n, raw, t->perm);
    t->keys = (uint64_t *)malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    for (int64_t s = 0; s < n; ++s) t->keys[s] = raw[t->perm[s]];
    free(raw);

    tree_add_cell(t, 0, 0, 0, 0, 0, n, -1);
    for (int64_t head = 0; head < t->ncell; ++head) {
        if (t->count[head] <= prm->n_crit || t->level[head] >= t->prm.max_level) continue;
        int lvl = t->level[head] + 1;
        int shift = 3 * (ORC_MAX_LEVEL - lvl);
        int64_t s = t->first[head], e = s + t->count[head];
        int64_t first_child = -1;
        int nch = 0;
        while (s < e) {
            int digit = (int)((t->keys[s] >> shift) & 7u);
            int64_t q = s;
            while (q < e && (int)((t->keys[q] >> shift) & 7u) == digit) ++q;
            int64_t cx = 2 * t->c[0][head] + ((digit >> 2) & 1);
            int64_t cy = 2 * t->c[1][head] + ((digit >> 1) & 1);
            int64_t cz = 2 * t->c[2][head] + (digit & 1);
            int64_t id = tree_add_cell(t, lvl, cx, cy, cz, s, q - s, head);
            if (first_child < 0) first_child = id;
            ++nch;
            s = q;
        }
        t->child_first[head] = first_child;
        t->nchild[head] = nch;
    }
    /* enclosing radii about the cell centres: leaves from their particles, parents bottom-up from
     * their children (cells are in BFS order, so children come after their parent) */
    t->radius = (double *)calloc((size_t)(t->ncell > 0 ? t->ncell : 1), sizeof(double));
    for (int64_t c = t->ncell - 1; c >= 0; --c) {
        double side = ldexp(t->L, -t->level[c]);
        double zc[3];
        for (int k = 0; k < 3; ++k) zc[k] = t->lo[k] + ((double)t->c[k][c] + 0.5) * side;
        double r = 0.0;
        if (t->nchild[c] == 0) {
            for (int64_t s2 = t->first[c]; s2 < t->first[c] + t->count[c]; ++s2) {
                int64_t i = t->perm[s2];
                double dx = x[i] - zc[0], dy = y[i] - zc[1], dz = z[i] - zc[2];
                double d = sqrt(dx * dx + dy * dy + dz * dz);
                if (d > r) r = d;
            }
        } else {
            /* |z_child - z_parent| = sqrt(3) side / 4 */
            double dcp = sqrt(3.0) * ldexp(t->L, -(t->level[c] + 2));
            for (int64_t q = t->child_first[c]; q < t->child_first[c] + t->nchild[c]; ++q) {
                double v = dcp + t->radius[q];
                if (v > r) r = v;
            }
        }
        t->radius[c] = r;
    }
    return t;
}

void orc_tree_radii(const orc_tree *t, double *r)
{
    for (int64_t c = 0; c < t->ncell; ++c) r[c] = t->radius[c];
}

void orc_tree_free(orc_tree *t)
{
    if (!t) return;
    free(t->perm); free(t->keys); free(t->level);
    for (int k = 0; k < 3; ++k) free(t->c[k]);
    free(t->first); free(t->count); free(t->child_first); free(t->parent); free(t->nchild);
    free(t->radius);
    free(t->m2l.a); free(t->m2l.b); free(t->p2p.a); free(t->p2p.b);
    free(t->on_path);
    free(t);
}

int64_t orc_tree_ncell(const orc_tree *t) { return t->ncell; }

void orc_tree_cells(const orc_tree *t, int32_t *level, int64_t *cx, int64_t *cy, int64_t *cz,
                    int64_t *first, int64_t *count, int64_t *child_first, int32_t *nchild)
{
    for (int64_t i = 0; i < t->ncell; ++i) {
        level[i] = t->level[i];
        cx[i] = t->c[0][i]; cy[i] = t->c[1][i]; cz[i] = t->c[2][i];
        first[i] = t->first[i]; count[i] = t->count[i];
        child_first[i] = t->child_first[i]; nchild[i] = t->nchild[i];
    }
}

void orc_tree_perm(const orc_tree *t, int64_t *perm, uint64_t *sorted_keys)
{
    for (int64_t s = 0; s < t->n; ++s) { perm[s] = t->perm[s]; sorted_keys[s] = t->keys[s]; }
}

void orc_tree_geometry(const orc_tree *t, double lo[3], double *L)
{
    lo[0] = t->lo[0]; lo[1] = t->lo[1]; lo[2] = t->lo[2]; *L = t->L;
}

static void cell_centre(const orc_tree *t, int64_t c, double zc[3])
{
    double side = ldexp(t->L, -t->level[c]);
    for (int k = 0; k < 3; ++k) zc[k] = t->lo[k] + ((double)t->c[k][c] + 0.5) * side;
}

/* Eq. (1) with R = kappa * side, plus (Wendland) the rule that the two cubes must be
 * farther apart than eps.  Evaluated exactly in integer units of half the finer side. */
int orc_well_separated(const orc_tree *t, int64_t a, int64_t b)
{
    int la = t->level[a], lb = t->level[b];
    int lf = la > lb ? la : lb;
    int64_t ha = (int64_t)1 << (lf - la), hb = (int64_t)1 << (lf - lb);
    int64_t d2 = 0, g2 = 0;
    for (int k = 0; k < 3; ++k) {
        int64_t ca = (2 * t->c[k][a] + 1) * ha;
        int64_t cb = (2 * t->c[k][b] + 1) * hb;
        int64_t dk = ca - cb;
        if (dk < 0) dk = -dk;
        d2 += dk * dk;
        int64_t gk = dk - (ha + hb);
        if (gk > 0) g2 += gk * gk;
    }
    int mac;
    if (t->prm.mac == 1) {
        /* enclosing spheres: R_a + R_b < theta |z_a - z_b|, the distance from the exact integer offset
         * (units of L / 2^(lf+1), a power of two) */
        double d = sqrt((double)d2) * ldexp(t->L, -(lf + 1));
        mac = t->radius[a] + t->radius[b] < t->prm.theta * d;
    } else {
        double theta2 = t->prm.theta * t->prm.theta;
        double kappa2 = t->prm.kappa * t->prm.kappa;
        double rsum = (double)(2 * (ha + hb));
        mac = (double)d2 * theta2 > kappa2 * (rsum * rsum);
    }
    if (!mac) return 0;
    if (t->prm.kernel == ORC_WENDLAND_C2) {
        /* eps in units of u = L / 2^(lf+1): exact power-of-two scaling */
        double eu = t->prm.eps * ldexp(1.0 / t->L, lf + 1);
        if (!((double)g2 > eu * eu)) return 0;
    }
    return 1;
}

static int is_leaf(const orc_tree *t, int64_t c) { return t->nchild[c] == 0; }

/* Algorithm 4, GET_INTERACTION_LIST(Ci, Cj), directed. */
static void walk(orc_tree *t, int64_t ci, int64_t cj)
{
    if (orc_well_separated(t, ci, cj)) {
        pl_push(&t->m2l, ci, cj);
    } else if (is_leaf(t, ci) && is_leaf(t, cj)) {
        pl_push(&t->p2p, ci, cj);
    } else if (is_leaf(t, ci)) {
        for (int k = 0; k < t->nchild[cj]; ++k) walk(t, ci, t->child_first[cj] + k);
    } else if (is_leaf(t, cj)) {
        for (int k = 0; k < t->nchild[ci]; ++k) {
            int64_t c = t->child_first[ci] + k;
            if (t->on_path && !t->on_path[c]) continue;
            walk(t, c, cj);
        }
    } else {
        for (int k = 0; k < t->nchild[ci]; ++k) {
            int64_t c = t->child_first[ci] + k;
            if (t->on_path && !t->on_path[c]) continue;
            for (int l = 0; l < t->nchild[cj]; ++l) walk(t, c, t->child_first[cj] + l);
        }
    }
}

void orc_tree_walk(orc_tree *t, int64_t *n_m2l, int64_t *n_p2p)
{
    if (!t->walked) {
        t->m2l.n = 0; t->p2p.n = 0;
        if (t->ncell > 0) walk(t, 0, 0);
        t->walked = 1;
    }
    if (n_m2l) *n_m2l = t->m2l.n;
    if (n_p2p) *n_p2p = t->p2p.n;
}

void orc_tree_lists(const orc_tree *t, int64_t *m2l_a, int64_t *m2l_b, int64_t *p2p_a, int64_t *p2p_b)
{
    for (int64_t i = 0; i < t->m2l.n; ++i) { m2l_a[i] = t->m2l.a[i]; m2l_b[i] = t->m2l.b[i]; }
    for (int64_t i = 0; i < t->p2p.n; ++i) { p2p_a[i] = t->p2p.a[i]; p2p_b[i] = t->p2p.b[i]; }
}

/* ------------------------------------------------------------------------------------ */
/* One FMM evaluation.                                                                  */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    orc_tree *t;
    int nc;                 /* coefficients per expansion */
    double *xs, *ys, *zs, *ms;
    uint8_t *fs;            /* fast flag in sorted order */
    double *M;              /* [cell][class S=0, F=1][nc] */
} fmm_state;

static void fmm_upward(fmm_state *st, int64_t n, const double *x, const double *y, const double *z,
                       const double *m, const uint8_t *is_fast, const orc_params *prm)
{
    orc_tree *t = orc_tree_build(n, x, y, z, prm);
    st->t = t;
    int p = prm->p;
    int nc = orc_num_coeffs(p);
    st->nc = nc;
    st->xs = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    st->ys = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    st->zs = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    st->ms = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    st->fs = (uint8_t *)malloc(n > 0 ? n : 1);
    for (int64_t s = 0; s < n; ++s) {
        int64_t i = t->perm[s];
        st->xs[s] = x[i]; st->ys[s] = y[i]; st->zs[s] = z[i]; st->ms[s] = m[i];
        st->fs[s] = is_fast ? (is_fast[i] != 0) : 0;
    }
    st->M = (double *)calloc((size_t)t->ncell * 2 * nc, sizeof(double));
    /* P2M on leaves, separately for the slow and fast classes */
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t c = 0; c < t->ncell; ++c) {
        if (!is_leaf(t, c)) continue;
        double zc[3];
        cell_centre(t, c, zc);
        double *MS = st->M + ((size_t)c * 2 + 0) * nc;
        double *MF = st->M + ((size_t)c * 2 + 1) * nc;
        for (int64_t s = t->first[c]; s < t->first[c] + t->count[c]; ++s) {
            double r[3] = {st->xs[s] - zc[0], st->ys[s] - zc[1], st->zs[s] - zc[2]};
            double *Mt = st->fs[s] ? MF : MS;
            for (int k = 0; k < nc; ++k) Mt[k] += st->ms[s] * mono(r, k);
        }
    }
    /* M2M, children before parents (reverse BFS order) */
    for (int64_t c = t->ncell - 1; c >= 1; --c) {
        int64_t par = t->parent[c];
        double zc[3], zp[3], dlt[3];
        cell_centre(t, c, zc);
        cell_centre(t, par, zp);
        for (int k = 0; k < 3; ++k) dlt[k] = zc[k] - zp[k];
        for (int cls = 0; cls < 2; ++cls)
            orc_m2m(p, st->M + ((size_t)c * 2 + cls) * nc, dlt, st->M + ((size_t)par * 2 + cls) * nc);
    }
}

static void fmm_free(fmm_state *st)
{
    orc_tree_free(st->t);
    free(st->xs); free(st->ys); free(st->zs); free(st->ms); free(st->fs); free(st->M);
}

/* M2L from source cell b into both local classes of sink cell a:
 * L_all (slow sinks) from M_S + M_F, L_S (fast sinks) from M_S. */
static void m2l_both(const fmm_state *st, const orc_params *prm, int64_t a, int64_t b, double *L_all, double *L_s)
{
    int nc = st->nc;
    double za[3], zb[3], d[3];
    cell_centre(st->t, a, za);
    cell_centre(st->t, b, zb);
    for (int k = 0; k < 3; ++k) d[k] = za[k] - zb[k];
    const double *MS = st->M + ((size_t)b * 2 + 0) * nc;
    const double *MF = st->M + ((size_t)b * 2 + 1) * nc;
    double *Mall = (double *)malloc(sizeof(double) * nc);
    for (int k = 0; k < nc; ++k) Mall[k] = MS[k] + MF[k];
    /* M2L uses the Newtonian tensor for Wendland (pairs are beyond eps by construction)
     * and the Plummer-softened tensor for Plummer softening. */
    orc_m2l(prm->p, Mall, d, prm->kernel, prm->eps, L_all);
    orc_m2l(prm->p, MS, d, prm->kernel, prm->eps, L_s);
    free(Mall);
}

/* P2P contribution from the particles of leaf b to sorted particle s */
static void p2p_one(const fmm_state *st, const orc_params *prm, int64_t s, int64_t b, double acc[4])
{
    const orc_tree *t = st->t;
    for (int64_t q = t->first[b]; q < t->first[b] + t->count[b]; ++q) {
        if (q == s) continue;
        if (st->fs[s] && st->fs[q]) continue;
        double dx = st->xs[q] - st->xs[s], dy = st->ys[q] - st->ys[s], dz = st->zs[q] - st->zs[s];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        double phi, g;
        orc_softened(prm->kernel, prm->eps, r, &phi, &g);
        acc[0] += st->ms[q] * g * dx; acc[1] += st->ms[q] * g * dy; acc[2] += st->ms[q] * g * dz;
        acc[3] += st->ms[q] * phi;
    }
}

int orc_fmm(int64_t n, const double *x, const double *y, const double *z, const double *m,
            const uint8_t *is_fast, const orc_params *prm,
            double *ax, double *ay, double *az, double *pot)
{
    mi_init();
    if (prm->p < 1 || prm->p > ORC_PMAX) return -1;
    if (n <= 0) return 0;
    fmm_state st;
    fmm_upward(&st, n, x, y, z, m, is_fast, prm);
    orc_tree *t = st.t;
    int nc = st.nc;
    orc_tree_walk(t, NULL, NULL);

    /* directed lists grouped by sink cell (counting sort keeps list order) */
    int64_t *m2l_off = (int64_t *)calloc(t->ncell + 1, sizeof(int64_t));
    int64_t *p2p_off = (int64_t *)calloc(t->ncell + 1, sizeof(int64_t));
    for (int64_t i = 0; i < t->m2l.n; ++i) m2l_off[t->m2l.a[i] + 1]++;
    for (int64_t i = 0; i < t->p2p.n; ++i) p2p_off[t->p2p.a[i] + 1]++;
    for (int64_t c = 0; c < t->ncell; ++c) { m2l_off[c + 1] += m2l_off[c]; p2p_off[c + 1] += p2p_off[c]; }
    int64_t *m2l_src = (int64_t *)malloc(sizeof(int64_t) * (t->m2l.n + 1));
    int64_t *p2p_src = (int64_t *)malloc(sizeof(int64_t) * (t->p2p.n + 1));
    {
        int64_t *fill = (int64_t *)calloc(t->ncell, sizeof(int64_t));
        for (int64_t i = 0; i < t->m2l.n; ++i) { int64_t a = t->m2l.a[i]; m2l_src[m2l_off[a] + fill[a]++] = t->m2l.b[i]; }
        memset(fill, 0, sizeof(int64_t) * t->ncell);
        for (int64_t i = 0; i < t->p2p.n; ++i) { int64_t a = t->p2p.a[i]; p2p_src[p2p_off[a] + fill[a]++] = t->p2p.b[i]; }
        free(fill);
    }

    /* local expansions: [cell][0 = all sources (slow sinks), 1 = slow sources (fast sinks)][nc] */
    double *L = (double *)calloc((size_t)t->ncell * 2 * nc, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t a = 0; a < t->ncell; ++a) {
        for (int64_t q = m2l_off[a]; q < m2l_off[a + 1]; ++q)
            m2l_both(&st, prm, a, m2l_src[q], L + ((size_t)a * 2 + 0) * nc, L + ((size_t)a * 2 + 1) * nc);
    }
    /* L2L, parents before children (BFS order) */
    for (int64_t c = 1; c < t->ncell; ++c) {
        int64_t par = t->parent[c];
        double zc[3], zp[3], dlt[3];
        cell_centre(t, c, zc);
        cell_centre(t, par, zp);
        for (int k = 0; k < 3; ++k) dlt[k] = zc[k] - zp[k];
        for (int cls = 0; cls < 2; ++cls)
            orc_l2l(prm->p, L + ((size_t)par * 2 + cls) * nc, dlt, L + ((size_t)c * 2 + cls) * nc);
    }
    /* L2P + P2P per leaf, then back to the caller's order */
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t c = 0; c < t->ncell; ++c) {
        if (!is_leaf(t, c)) continue;
        double zc[3];
        cell_centre(t, c, zc);
        for (int64_t s = t->first[c]; s < t->first[c] + t->count[c]; ++s) {
            double rho[3] = {st.xs[s] - zc[0], st.ys[s] - zc[1], st.zs[s] - zc[2]};
            double phi, a3[3];
            orc_l2p(prm->p, L + ((size_t)c * 2 + (st.fs[s] ? 1 : 0)) * nc, rho, &phi, a3);
            double acc[4] = {a3[0], a3[1], a3[2], phi};
            for (int64_t q = p2p_off[c]; q < p2p_off[c + 1]; ++q) p2p_one(&st, prm, s, p2p_src[q], acc);
            int64_t i = t->perm[s];
            ax[i] = acc[0]; ay[i] = acc[1]; az[i] = acc[2];
            if (pot) pot[i] = acc[3];
        }
    }
    free(L); free(m2l_off); free(p2p_off); free(m2l_src); free(p2p_src);
    fmm_free(&st);
    return 0;
}

/* One-sink evaluation: the walk is restricted to pairs whose first member lies on the
 * path from the root to the sink's leaf (every other pair cannot reach this sink), the
 * M2L contributions are translated down that path with L2L and evaluated with L2P. */
int orc_fmm_sample(int64_t n, const double *x, const double *y, const double *z, const double *m,
                   const uint8_t *is_fast, const orc_params *prm,
                   int64_t n_sample, const int64_t *sample,
                   double *ax, double *ay, double *az, double *pot)
{
    mi_init();
    if (prm->p < 1 || prm->p > ORC_PMAX) return -1;
    if (n <= 0 || n_sample <= 0) return 0;
    fmm_state st;
    fmm_upward(&st, n, x, y, z, m, is_fast, prm);
    orc_tree *t0 = st.t;
    int nc = st.nc;
    int64_t *inv = (int64_t *)malloc(sizeof(int64_t) * n);
    for (int64_t s = 0; s < n; ++s) inv[t0->perm[s]] = s;
    int64_t *leaf_of = (int64_t *)malloc(sizeof(int64_t) * n);
    for (int64_t c = 0; c < t0->ncell; ++c)
        if (is_leaf(t0, c))
            for (int64_t s = t0->first[c]; s < t0->first[c] + t0->count[c]; ++s) leaf_of[s] = c;

#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n_sample; ++q) {
        /* private shallow copy of the tree with its own lists and path marks */
        orc_tree tq = *t0;
        memset(&tq.m2l, 0, sizeof(pair_list));
        memset(&tq.p2p, 0, sizeof(pair_list));
        tq.on_path = (uint8_t *)calloc(t0->ncell, 1);
        int64_t s = inv[sample[q]];
        int64_t leaf = leaf_of[s];
        int64_t path[ORC_MAX_LEVEL + 2];
        int depth = 0;
        for (int64_t c = leaf; c >= 0; c = t0->parent[c]) { tq.on_path[c] = 1; path[depth++] = c; }
        walk(&tq, 0, 0);
        /* local expansion accumulated down the path, root first */
        double *Lall = (double *)calloc(nc, sizeof(double)), *Ls = (double *)calloc(nc, sizeof(double));
        double *Tall = (double *)calloc(nc, sizeof(double)), *Ts = (double *)calloc(nc, sizeof(double));
        for (int k = depth - 1; k >= 0; --k) {
            int64_t c = path[k];
            if (k != depth - 1) {
                double zc[3], zp[3], dlt[3];
                cell_centre(t0, c, zc);
                cell_centre(t0, path[k + 1], zp);
                for (int a = 0; a < 3; ++a) dlt[a] = zc[a] - zp[a];
                memset(Tall, 0, sizeof(double) * nc); memset(Ts, 0, sizeof(double) * nc);
                orc_l2l(prm->p, Lall, dlt, Tall);
                orc_l2l(prm->p, Ls, dlt, Ts);
                memcpy(Lall, Tall, sizeof(double) * nc); memcpy(Ls, Ts, sizeof(double) * nc);
            }
            for (int64_t e = 0; e < tq.m2l.n; ++e)
                if (tq.m2l.a[e] == c) m2l_both(&st, prm, c, tq.m2l.b[e], Lall, Ls);
        }
        double zc[3];
        cell_centre(t0, leaf, zc);
        double rho[3] = {st.xs[s] - zc[0], st.ys[s] - zc[1], st.zs[s] - zc[2]};
        double phi, a3[3];
        orc_l2p(prm->p, st.fs[s] ? Ls : Lall, rho, &phi, a3);
        double acc[4] = {a3[0], a3[1], a3[2], phi};
        for (int64_t e = 0; e < tq.p2p.n; ++e)
            if (tq.p2p.a[e] == leaf) p2p_one(&st, prm, s, tq.p2p.b[e], acc);
        ax[q] = acc[0]; ay[q] = acc[1]; az[q] = acc[2];
        if (pot) pot[q] = acc[3];
        free(Lall); free(Ls); free(Tall); free(Ts);
        free(tq.m2l.a); free(tq.m2l.b); free(tq.p2p.a); free(tq.p2p.b); free(tq.on_path);
    }
    free(inv); free(leaf_of);
    fmm_free(&st);
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* HOLD integrator (Sec. 2.2).                                                          */
/* ------------------------------------------------------------------------------------ */
/* dt_i = sqrt(eta eps / |a|), |a| ~ |a_old| + |a_current| (Sec. 2.2, Fig. 1 caption) */
double orc_timestep(double eta, double eps, double a_old, double a_cur)
{
    double a = a_old + a_cur;
    if (!(a > 0.0)) return INFINITY;
    return sqrt(eta * eps / a);
}

/* Eq. (9): a minimum timestep from the total acceleration, imposed on the function above */
double orc_timestep_tot(double eta, double eps, double a_old, double a_cur, double eta_tot, double a_tot)
{
    double dt = orc_timestep(eta, eps, a_old, a_cur);
    if (eta_tot > 0.0 && a_tot > 0.0) {
        double dt_tot = sqrt(eta_tot * eps / a_tot);
        if (dt_tot < dt) dt = dt_tot;
    }
    return dt;
}

/* smallest k with dt_max / 2^k <= dt_i, capped at k_max */
int orc_rung(double dt_i, double dt_max, int k_max)
{
    int k = 0;
    while (k < k_max && !(dt_i >= ldexp(dt_max, -k))) ++k;
    return k;
}

typedef struct {
    int64_t n;
    double *x, *y, *z, *vx, *vy, *vz;
    const double *m;
    const orc_params *prm;
    const orc_hhs_params *hp;
    double *a_old, *a_cur, *a_tot, *dt;
    int32_t *rung;
    orc_hhs_stats *stats;
    int64_t *trace;
    int32_t trace_cap;
    int status;
} hhs_ctx;

static void trace_push(hhs_ctx *h, int64_t kind, int64_t rung, int64_t a, int64_t b)
{
    if (!h->trace || h->stats->trace_len >= h->trace_cap) return;
    int64_t *e = h->trace + 4 * (int64_t)h->stats->trace_len;
    e[0] = kind; e[1] = rung; e[2] = a; e[3] = b;
    h->stats->trace_len++;
}

/* Algorithm 3, KICK(rung, system1, system2, dt, kickFS, secondkick).  The Poisson solver
 * is called on the joint set system1 + system2; for kickS2F (kickFS = 1) the masses of
 * system1 are set to zero so that only system2 acts on it. */
static void kick(hhs_ctx *h, int rung, const int64_t *s1, int64_t n1, const int64_t *s2, int64_t n2,
                 double dt, int kick_fs, int second)
{
    if (n1 == 0) return;                       /* no sinks */
    if (kick_fs && n2 == 0) return;            /* no sources */
    int64_t nj = n1 + n2;
    double *jx = (double *)malloc(sizeof(double) * nj), *jy = (double *)malloc(sizeof(double) * nj);
    double *jz = (double *)malloc(sizeof(double) * nj), *jm = (double *)malloc(sizeof(double) * nj);
    double *ax = (double *)malloc(sizeof(double) * nj), *ay = (double *)malloc(sizeof(double) * nj);
    double *az = (double *)malloc(sizeof(double) * nj);
    /* joint_pos_mass in index order of the current system (a merge of the two sorted sets) */
    int64_t i1 = 0, i2 = 0, q = 0;
    int64_t *src = (int64_t *)malloc(sizeof(int64_t) * nj);
    uint8_t *in1 = (uint8_t *)malloc(nj);
    while (i1 < n1 || i2 < n2) {
        if (i2 >= n2 || (i1 < n1 && s1[i1] < s2[i2])) { src[q] = s1[i1++]; in1[q] = 1; }
        else { src[q] = s2[i2++]; in1[q] = 0; }
        ++q;
    }
    for (q = 0; q < nj; ++q) {
        int64_t i = src[q];
        jx[q] = h->x[i]; jy[q] = h->y[i]; jz[q] = h->z[i];
        jm[q] = (kick_fs && in1[q]) ? 0.0 : h->m[i];       /* mask_mass_to_zero(system1) */
    }
    if (orc_fmm(nj, jx, jy, jz, jm, NULL, h->prm, ax, ay, az, NULL) != 0) h->status = -1;
    h->stats->poisson_calls++;
    h->stats->sink_forces += n1;
    trace_push(h, kick_fs ? 0 : 1, rung, n1, kick_fs ? n2 : nj);
    /* rung 0, second kickFS2S: the whole system with all masses, |a|_tot of every particle (Eq. 9) */
    if (h->a_tot && !kick_fs && second && rung == 0)
        for (q = 0; q < nj; ++q) h->a_tot[src[q]] = sqrt(ax[q] * ax[q] + ay[q] * ay[q] + az[q] * az[q]);
    for (q = 0; q < nj; ++q) {
        if (!in1[q]) continue;
        int64_t i = src[q];
        h->vx[i] += ax[q] * dt; h->vy[i] += ay[q] * dt; h->vz[i] += az[q] * dt;
        double amag = sqrt(ax[q] * ax[q] + ay[q] * ay[q] + az[q] * az[q]);
        if (kick_fs) { if (second) h->a_old[i] = amag; }   /* most recent kick from lower rungs */
        else h->a_cur[i] = amag;                           /* most recent kick from same/faster rungs */
    }
    free(jx); free(jy); free(jz); free(jm); free(ax); free(ay); free(az); free(src); free(in1);
}

static void drift(hhs_ctx *h, int rung, const int64_t *s, int64_t ns, double dt)
{
    for (int64_t q = 0; q < ns; ++q) {
        int64_t i = s[q];
        h->x[i] += h->vx[i] * dt; h->y[i] += h->vy[i] * dt; h->z[i] += h->vz[i] * dt;
    }
    trace_push(h, 2, rung, ns, 0);
}

/* Algorithm 2 */
static void kdk(hhs_ctx *h, int rung, const int64_t *S, int64_t nS, const int64_t *F, int64_t nF, double dt)
{
    h->stats->kdk_frames++;
    if (nF > 0) kick(h, rung, F, nF, S, nS, dt / 2, 1, 0);   /* kickS2F  */
    kick(h, rung, S, nS, F, nF, dt / 2, 0, 0);               /* kickFS2S */
    drift(h, rung, S, nS, dt);
    kick(h, rung, S, nS, F, nF, dt / 2, 0, 1);               /* kickFS2S */
    if (nF > 0) kick(h, rung, F, nF, S, nS, dt / 2, 1, 1);   /* kickS2F  */
}

/* Algorithm 1 */
static void evolve_hold(hhs_ctx *h, int rung, const int64_t *sys, int64_t ns, double dt, int calc)
{
    if (calc)
        for (int64_t q = 0; q < ns; ++q) {
            int64_t i = sys[q];
            h->dt[i] = h->a_tot ? orc_timestep_tot(h->hp->eta, h->prm->eps, h->a_old[i], h->a_cur[i],
                                                   h->hp->eta_tot, h->a_tot[i])
                                : orc_timestep(h->hp->eta, h->prm->eps, h->a_old[i], h->a_cur[i]);
        }
    /* split_slow_fast: slow = {dt_i >= dt}; at the deepest rung everything is slow */
    int64_t *S = (int64_t *)malloc(sizeof(int64_t) * (ns > 0 ? ns : 1));
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * (ns > 0 ? ns : 1));
    int64_t nS = 0, nF = 0;
    for (int64_t q = 0; q < ns; ++q) {
        int64_t i = sys[q];
        if (rung >= h->hp->k_max || h->dt[i] >= dt) S[nS++] = i;
        else F[nF++] = i;
    }
    for (int64_t q = 0; q < nS; ++q) h->rung[S[q]] = rung;
    if (nS > 0 && rung > h->stats->max_rung) h->stats->max_rung = rung;
    if (nF > 0) evolve_hold(h, rung + 1, F, nF, dt / 2, 0);
    kdk(h, rung, S, nS, F, nF, dt);
    if (nF > 0) evolve_hold(h, rung + 1, F, nF, dt / 2, 1);
    free(S); free(F);
}

int orc_hhs_init(int64_t n, const double *x, const double *y, const double *z, const double *m,
                 const orc_params *prm, double *a_old, double *a_cur, double *a_tot)
{
    double *ax = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *ay = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *az = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    int rc = orc_fmm(n, x, y, z, m, NULL, prm, ax, ay, az, NULL);
    for (int64_t i = 0; i < n; ++i) {
        a_old[i] = 0.0;
        a_cur[i] = sqrt(ax[i] * ax[i] + ay[i] * ay[i] + az[i] * az[i]);
        if (a_tot) a_tot[i] = a_cur[i];
    }
    free(ax); free(ay); free(az);
    return rc;
}

int orc_hhs_step(int64_t n, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                 const double *m, const orc_params *prm, const orc_hhs_params *hp,
                 double *a_old, double *a_cur, double *a_tot, int32_t *rung_out,
                 orc_hhs_stats *stats, int64_t *trace, int32_t trace_cap)
{
    hhs_ctx h;
    memset(&h, 0, sizeof(h));
    orc_hhs_stats local;
    memset(&local, 0, sizeof(local));
    h.n = n; h.x = x; h.y = y; h.z = z; h.vx = vx; h.vy = vy; h.vz = vz; h.m = m;
    h.prm = prm; h.hp = hp; h.a_old = a_old; h.a_cur = a_cur; h.a_tot = a_tot;
    h.dt = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    h.rung = rung_out ? rung_out : (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    h.stats = stats ? stats : &local;
    memset(h.stats, 0, sizeof(orc_hhs_stats));
    h.trace = trace; h.trace_cap = trace_cap;
    int64_t *all = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) all[i] = i;
    evolve_hold(&h, 0, all, n, hp->dt_max, 1);
    free(all); free(h.dt);
    if (!rung_out) free(h.rung);
    return h.status;
}

/* ------------------------------------------------------------------------------------ */
/* Traditional individual timesteps (Sec. 2.3), the comparison integrator.              */
/* ------------------------------------------------------------------------------------ */
/* deepest rung allowed for a step that starts at substep m of a 2^k_max grid: the step must start on
 * a multiple of itself, i.e. 2^(k_max - r) divides m */
static int trad_aligned_rung(int64_t m, int k_max)
{
    if (m == 0) return 0;
    int tz = 0;
    while (tz < k_max && ((m >> tz) & 1) == 0) ++tz;
    return k_max - tz;
}

static int trad_rung(const orc_hhs_params *hp, double eps, double amag, int64_t m)
{
    int r = orc_rung(orc_timestep(hp->eta, eps, 0.0, amag), hp->dt_max, hp->k_max);
    int ra = trad_aligned_rung(m, hp->k_max);
    return r > ra ? r : ra;
}

int orc_trad_init(int64_t n, const double *x, const double *y, const double *z, const double *m,
                  const orc_params *prm, const orc_hhs_params *hp, double *acc, int32_t *rung)
{
    int rc = orc_fmm(n, x, y, z, m, NULL, prm, acc, acc + n, acc + 2 * n, NULL);
    for (int64_t i = 0; i < n; ++i) {
        double a = sqrt(acc[i] * acc[i] + acc[n + i] * acc[n + i] + acc[2 * n + i] * acc[2 * n + i]);
        rung[i] = trad_rung(hp, prm->eps, a, 0);
    }
    return rc;
}

int orc_trad_step(int64_t n, double *x, double *y, double *z, double *vx, double *vy, double *vz,
                  const double *m, const orc_params *prm, const orc_hhs_params *hp,
                  double *acc, int32_t *rung, orc_hhs_stats *stats)
{
    orc_hhs_stats local;
    if (!stats) stats = &local;
    memset(stats, 0, sizeof(*stats));
    const int K = hp->k_max;
    const int64_t M = (int64_t)1 << K;            /* substeps of dt_max / 2^K in one call */
    const double dt_min = ldexp(hp->dt_max, -K);
    int64_t *end = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));   /* substep where i's step ends */
    double *ax = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *ay = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *az = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    int rc = 0;
    /* opening half kicks at the start of the step, with the forces and rungs held from before */
    for (int64_t i = 0; i < n; ++i) {
        double h = 0.5 * ldexp(hp->dt_max, -rung[i]);
        vx[i] += acc[i] * h; vy[i] += acc[n + i] * h; vz[i] += acc[2 * n + i] * h;
        end[i] = (int64_t)1 << (K - rung[i]);
        if (rung[i] > stats->max_rung) stats->max_rung = rung[i];
    }
    for (int64_t t = 1; t <= M; ++t) {
        int64_t na = 0;
        for (int64_t i = 0; i < n; ++i) na += end[i] == t;
        if (na == 0) continue;
        /* drift the particles whose step ends now over their whole step */
        for (int64_t i = 0; i < n; ++i)
            if (end[i] == t) {
                double dt = ldexp(hp->dt_max, -rung[i]);
                x[i] += vx[i] * dt; y[i] += vy[i] * dt; z[i] += vz[i] * dt;
            }
        /* forces on them from all masses at the stored positions */
        if (orc_fmm(n, x, y, z, m, NULL, prm, ax, ay, az, NULL) != 0) rc = -1;
        stats->poisson_calls++;
        stats->sink_forces += na;
        for (int64_t i = 0; i < n; ++i) {
            if (end[i] != t) continue;
            double h = 0.5 * ldexp(hp->dt_max, -rung[i]);
            vx[i] += ax[i] * h; vy[i] += ay[i] * h; vz[i] += az[i] * h;     /* closing half kick */
            acc[i] = ax[i]; acc[n + i] = ay[i]; acc[2 * n + i] = az[i];
            double a = sqrt(ax[i] * ax[i] + ay[i] * ay[i] + az[i] * az[i]);
            int r = trad_rung(hp, prm->eps, a, t == M ? 0 : t);
            rung[i] = r;
            if (t < M) {                                                     /* opening half kick */
                double h2 = 0.5 * ldexp(hp->dt_max, -r);
                vx[i] += ax[i] * h2; vy[i] += ay[i] * h2; vz[i] += az[i] * h2;
                end[i] = t + ((int64_t)1 << (K - r));
                if (r > stats->max_rung) stats->max_rung = r;
            }
        }
    }
    (void)dt_min;
    free(end); free(ax); free(ay); free(az);
    return rc;
}

/* P = sum m v, L = sum m x cross v, E = sum m v^2/2 + sum m phi / 2 */
void orc_diagnostics(int64_t n, const double *x, const double *y, const double *z,
                     const double *vx, const double *vy, const double *vz,
                     const double *m, const double *pot, double out[7])
{
    double P[3] = {0, 0, 0}, Lm[3] = {0, 0, 0}, K = 0, W = 0;
    for (int64_t i = 0; i < n; ++i) {
        P[0] += m[i] * vx[i]; P[1] += m[i] * vy[i]; P[2] += m[i] * vz[i];
        Lm[0] += m[i] * (y[i] * vz[i] - z[i] * vy[i]);
        Lm[1] += m[i] * (z[i] * vx[i] - x[i] * vz[i]);
        Lm[2] += m[i] * (x[i] * vy[i] - y[i] * vx[i]);
        K += 0.5 * m[i] * (vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i]);
        if (pot) W += 0.5 * m[i] * pot[i];
    }
    out[0] = P[0]; out[1] = P[1]; out[2] = P[2];
    out[3] = Lm[0]; out[4] = Lm[1]; out[5] = Lm[2];
    out[6] = K + W;
}
