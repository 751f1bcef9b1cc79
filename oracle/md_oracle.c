/*
 * md_oracle.c -- plain, slow, double-precision CPU oracle for the short-range
 * molecular-dynamics hot path of "A hybrid algorithm for parallel molecular
 * dynamics simulations" (Mangiardi & Meyer).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only tests/, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py use it.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * Every routine is written for readability, not speed: loops in the order the
 * paper states them, fp64 throughout, no blocking, no fusion, and compiled
 * with -ffp-contract=off so that no multiply-add is fused.  OpenMP pragmas only
 * split the outer per-atom loops over threads; each atom's sum still runs in
 * ascending neighbour order, so the result does not depend on the thread count.
 *
 * Conventions (the paper's problem statement, Sec. 2.2 and Sec. 3.3):
 *   - positions/velocities/forces: n x 3 doubles, xyz interleaved, original
 *     atom order; orthorhombic periodic box box[3], positions in [0, L).
 *   - minimum image: d = x_j - x_i; if d > L/2 then d -= L, else if d < -L/2
 *     then d += L (valid for L > 2 r_list).
 *   - squared distance r^2 = dx*dx + dy*dy + dz*dz, left to right.
 *   - a pair is inside a cutoff r_x when r^2 < r_x^2 (strict).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_CAPACITY (-4)

/* ------------------------------------------------------------------------ */
/* geometry                                                                  */
/* ------------------------------------------------------------------------ */

static double min_image(double d, double L) {
    double h = 0.5 * L;
    if (d > h) d -= L;
    else if (d < -h) d += L;
    return d;
}

/* Squared minimum-image distance between atoms i and j, plus the components
 * of d = r_j - r_i (the paper's R = r_i - r_j is its negative). */
static double pair_r2(const double *pos, const double *box, int64_t i, int64_t j,
                      double *dx, double *dy, double *dz) {
    double ax = min_image(pos[3 * j + 0] - pos[3 * i + 0], box[0]);
    double ay = min_image(pos[3 * j + 1] - pos[3 * i + 1], box[1]);
    double az = min_image(pos[3 * j + 2] - pos[3 * i + 2], box[2]);
    double r2 = ax * ax;
    r2 = r2 + ay * ay;
    r2 = r2 + az * az;
    *dx = ax; *dy = ay; *dz = az;
    return r2;
}

double orc_pair_r2(const double *pos, const double *box, int64_t i, int64_t j) {
    double dx, dy, dz;
    return pair_r2(pos, box, i, j, &dx, &dy, &dz);
}

/* ------------------------------------------------------------------------ */
/* cell decomposition (Sec. 2.1: the volume is divided into small cells and  */
/* one task covers all atoms of one cell)                                    */
/* ------------------------------------------------------------------------ */

/* Cells per dimension n_d = floor(L_d / r_list), and inv_w_d = n_d / L_d. */
int orc_cell_grid(const double *box, double r_list, int32_t *ncell, double *inv_w) {
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0.0) || !(r_list > 0.0)) return ORC_ERR_INVALID;
        double q = floor(box[d] / r_list);
        if (q < 1.0) return ORC_ERR_INVALID;
        ncell[d] = (int32_t)q;
        inv_w[d] = (double)ncell[d] / box[d];
    }
    return ORC_OK;
}

/* Cell index of one coordinate: floor(x * inv_w), clamped to [0, n-1]. */
static int32_t cell_coord(double x, double inv_w, int32_t n) {
    double q = floor(x * inv_w);
    int32_t c = (int32_t)q;
    if (q < 0.0) c = 0;
    if (c > n - 1) c = n - 1;
    return c;
}

/* Linear cell id with x fastest: (cz * ny + cy) * nx + cx. */
static int64_t cell_id(int32_t cx, int32_t cy, int32_t cz, const int32_t *ncell) {
    return ((int64_t)cz * ncell[1] + cy) * ncell[0] + cx;
}

/* Assign every atom to its cell and produce the stable order by (cell, id):
 *   cell_of_atom[i]  cell of original atom i
 *   cell_start[c]    first slot of cell c in the order (ncells + 1 entries)
 *   order[k]         original id of the atom in slot k
 * A plain counting sort: count, exclusive prefix sum, then place atoms in
 * ascending original id, which makes the order stable. */
int orc_bin(int64_t n, const double *pos, const int32_t *ncell, const double *inv_w,
            int32_t *cell_of_atom, int64_t *cell_start, int64_t *order) {
    int64_t ncells = (int64_t)ncell[0] * ncell[1] * ncell[2];
    for (int64_t c = 0; c <= ncells; ++c) cell_start[c] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t cx = cell_coord(pos[3 * i + 0], inv_w[0], ncell[0]);
        int32_t cy = cell_coord(pos[3 * i + 1], inv_w[1], ncell[1]);
        int32_t cz = cell_coord(pos[3 * i + 2], inv_w[2], ncell[2]);
        int64_t c = cell_id(cx, cy, cz, ncell);
        cell_of_atom[i] = (int32_t)c;
        cell_start[c + 1] += 1;
    }
    for (int64_t c = 0; c < ncells; ++c) cell_start[c + 1] += cell_start[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncells > 0 ? ncells : 1));
    if (!fill) return ORC_ERR_INVALID;
    for (int64_t c = 0; c < ncells; ++c) fill[c] = cell_start[c];
    for (int64_t i = 0; i < n; ++i) order[fill[cell_of_atom[i]]++] = i;
    free(fill);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Verlet neighbour lists (Sec. 2.1 list construction per cell task;         */
/* Sec. 3.3 list radius r_list = r_c + skin)                                 */
/* ------------------------------------------------------------------------ */

/* Brute force O(N^2): N(i) = { j != i : r_ij^2 < r_list^2 }, ascending j.
 * half != 0 keeps only j > i.  offsets has n + 1 entries.  Returns the total
 * number of entries, or ORC_ERR_CAPACITY if it exceeds cap (offsets are then
 * still filled so the caller can size the buffer). */
int64_t orc_neighbors_brute(int64_t n, const double *pos, const double *box, double r_list,
                            int half, int64_t *offsets, int32_t *ids, int64_t cap) {
    double rl2 = r_list * r_list;
    int64_t total = 0;
    int overflow = 0;
    offsets[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            if (j == i || (half && j < i)) continue;
            if (orc_pair_r2(pos, box, i, j) < rl2) {
                if (total < cap) ids[total] = (int32_t)j;
                else overflow = 1;
                total += 1;
            }
        }
        offsets[i + 1] = total;
    }
    return overflow ? ORC_ERR_CAPACITY : total;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Neighbour offsets of one cell along one dimension: the distinct values of
 * (c - 1, c, c + 1) mod n.  For n < 3 some coincide and are kept once. */
static int stencil_1d(int32_t c, int32_t n, int32_t *out) {
    int k = 0;
    for (int d = -1; d <= 1; ++d) {
        int32_t v = ((c + d) % n + n) % n;
        int dup = 0;
        for (int q = 0; q < k; ++q) dup |= (out[q] == v);
        if (!dup) out[k++] = v;
    }
    return k;
}

/* Cell-based list: the same set as orc_neighbors_brute, found by scanning the
 * 27 cells around each atom's cell (Sec. 2.1).  Per-atom entries are sorted by
 * original id so both list routines give identical arrays.  Requires
 * L > 2 r_list (minimum image) and the cell grid of orc_cell_grid. */
int64_t orc_neighbors_cells(int64_t n, const double *pos, const double *box, double r_list,
                            int half, int64_t *offsets, int32_t *ids, int64_t cap) {
    int32_t ncell[3];
    double inv_w[3];
    if (orc_cell_grid(box, r_list, ncell, inv_w) != ORC_OK) return ORC_ERR_INVALID;
    int64_t ncells = (int64_t)ncell[0] * ncell[1] * ncell[2];
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(ncells + 1));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *count = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!cell_of || !start || !order || !count) {
        free(cell_of); free(start); free(order); free(count);
        return ORC_ERR_INVALID;
    }
    orc_bin(n, pos, ncell, inv_w, cell_of, start, order);
    double rl2 = r_list * r_list;

    /* pass 1: count per atom */
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = cell_of[i];
        int32_t cx = (int32_t)(c % ncell[0]);
        int32_t cy = (int32_t)((c / ncell[0]) % ncell[1]);
        int32_t cz = (int32_t)(c / ((int64_t)ncell[0] * ncell[1]));
        int32_t sx[3], sy[3], sz[3];
        int kx = stencil_1d(cx, ncell[0], sx), ky = stencil_1d(cy, ncell[1], sy),
            kz = stencil_1d(cz, ncell[2], sz);
        int64_t cnt = 0;
        for (int a = 0; a < kz; ++a)
            for (int b = 0; b < ky; ++b)
                for (int e = 0; e < kx; ++e) {
                    int64_t cc = cell_id(sx[e], sy[b], sz[a], ncell);
                    for (int64_t s = start[cc]; s < start[cc + 1]; ++s) {
                        int64_t j = order[s];
                        if (j == i || (half && j < i)) continue;
                        if (orc_pair_r2(pos, box, i, j) < rl2) cnt += 1;
                    }
                }
        count[i] = cnt;
    }
    offsets[0] = 0;
    for (int64_t i = 0; i < n; ++i) offsets[i + 1] = offsets[i] + count[i];
    int64_t total = offsets[n];
    if (total > cap) {
        free(cell_of); free(start); free(order); free(count);
        return ORC_ERR_CAPACITY;
    }
    /* pass 2: fill and sort each atom's entries by original id */
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = cell_of[i];
        int32_t cx = (int32_t)(c % ncell[0]);
        int32_t cy = (int32_t)((c / ncell[0]) % ncell[1]);
        int32_t cz = (int32_t)(c / ((int64_t)ncell[0] * ncell[1]));
        int32_t sx[3], sy[3], sz[3];
        int kx = stencil_1d(cx, ncell[0], sx), ky = stencil_1d(cy, ncell[1], sy),
            kz = stencil_1d(cz, ncell[2], sz);
        int64_t w = offsets[i];
        for (int a = 0; a < kz; ++a)
            for (int b = 0; b < ky; ++b)
                for (int e = 0; e < kx; ++e) {
                    int64_t cc = cell_id(sx[e], sy[b], sz[a], ncell);
                    for (int64_t s = start[cc]; s < start[cc + 1]; ++s) {
                        int64_t j = order[s];
                        if (j == i || (half && j < i)) continue;
                        if (orc_pair_r2(pos, box, i, j) < rl2) ids[w++] = (int32_t)j;
                    }
                }
        qsort(ids + offsets[i], (size_t)(w - offsets[i]), sizeof(int32_t), cmp_i32);
    }
    free(cell_of); free(start); free(order); free(count);
    return total;
}

/* ------------------------------------------------------------------------ */
/* potentials                                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t potential;      /* 0 = Lennard-Jones, 1 = Sutton-Chen */
    int32_t rebuild_every;  /* 0 = half-skin displacement rule */
    double eps;             /* LJ epsilon / SC epsilon */
    double sigma;           /* LJ sigma / SC lattice parameter a */
    double c;               /* SC c */
    double n_exp;           /* SC n (pair repulsion exponent) */
    double m_exp;           /* SC m (density exponent) */
    double rc;              /* potential cutoff */
    double skin;            /* list skin; r_list = rc + skin */
    double dt;              /* time step */
    double mass;            /* atom mass */
    const struct orc_eam_s *eam;  /* embedded-atom tables (potential 2), else NULL */
    /* multi-element Lennard-Jones (potential 0 with ntypes > 0): the species
     * of every atom, pair parameters t_eps[a * ntypes + b], t_sigma[...] and
     * masses t_mass[a]; eps, sigma and mass above are then not used */
    int32_t ntypes;
    const int32_t *types;
    const double *t_eps, *t_sigma, *t_mass;
} orc_params;

/* Lennard-Jones, truncated and energy-shifted at r_c:
 *   phi(r) = 4 eps [(s/r)^12 - (s/r)^6] - phi_LJ(r_c),  r < r_c.
 * The pair force follows Sec. 2.2: F = -(1/d) dphi/dr R with R = r_i - r_j,
 * added to f_i and subtracted from f_j.  -(1/d) dphi/dr for LJ is
 * (48 eps / d^2) [(s/d)^12 - (s/d)^6 / 2]. */
static double lj_phi(double r2, double eps, double sigma) {
    double s2 = sigma * sigma / r2;
    double s6 = s2 * s2 * s2;
    return 4.0 * eps * (s6 * s6 - s6);
}
static double lj_fscalar(double r2, double eps, double sigma) {
    double s2 = sigma * sigma / r2;
    double s6 = s2 * s2 * s2;
    return 48.0 * eps / r2 * (s6 * s6 - 0.5 * s6);
}

/* LJ over all pairs i < j (O(N^2)), the definition itself.  f is n x 3
 * (overwritten).  Returns the potential energy. */
double orc_lj_brute(int64_t n, const double *pos, const double *box, double eps, double sigma,
                    double rc, double *f) {
    double rc2 = rc * rc, shift = lj_phi(rc2, eps, sigma), U = 0.0;
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double dx, dy, dz;
            double r2 = pair_r2(pos, box, i, j, &dx, &dy, &dz);
            if (!(r2 < rc2)) continue;
            double fs = lj_fscalar(r2, eps, sigma);
            /* R = r_i - r_j = -(dx, dy, dz); F = fs * R */
            double Fx = -fs * dx, Fy = -fs * dy, Fz = -fs * dz;
            f[3 * i + 0] += Fx; f[3 * i + 1] += Fy; f[3 * i + 2] += Fz;
            f[3 * j + 0] -= Fx; f[3 * j + 1] -= Fy; f[3 * j + 2] -= Fz;
            U += lj_phi(r2, eps, sigma) - shift;
        }
    }
    return U;
}

/* LJ from a full neighbour list (both directions): f_i = sum_j F_ij in list
 * order, U = 1/2 sum_i sum_j phi(r_ij).  Optional per-atom energy e_atom. */
double orc_lj_list(int64_t n, const double *pos, const double *box, double eps, double sigma,
                   double rc, const int64_t *offsets, const int32_t *ids, double *f,
                   double *e_atom) {
    double rc2 = rc * rc, shift = lj_phi(rc2, eps, sigma), U = 0.0;
    #pragma omp parallel for schedule(dynamic, 256) reduction(+ : U)
    for (int64_t i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0, fz = 0.0, ei = 0.0;
        for (int64_t k = offsets[i]; k < offsets[i + 1]; ++k) {
            int64_t j = ids[k];
            double dx, dy, dz;
            double r2 = pair_r2(pos, box, i, j, &dx, &dy, &dz);
            if (!(r2 < rc2)) continue;
            double fs = lj_fscalar(r2, eps, sigma);
            fx -= fs * dx; fy -= fs * dy; fz -= fs * dz;
            ei += 0.5 * (lj_phi(r2, eps, sigma) - shift);
        }
        f[3 * i + 0] = fx; f[3 * i + 1] = fy; f[3 * i + 2] = fz;
        if (e_atom) e_atom[i] = ei;
        U += ei;
    }
    return U;
}

/* Multi-element Lennard-Jones (the Cu-Au alloy and layer systems of
 * Sec. 3.1): the pair (i, j) takes eps and sigma of its two species,
 * eps[t_i * nt + t_j], and its energy is shifted to zero at r_c with those
 * parameters.  Same loops as orc_lj_brute / orc_lj_list otherwise. */
double orc_lj_typed_brute(int64_t n, const double *pos, const double *box, int32_t nt,
                          const int32_t *types, const double *eps, const double *sigma, double rc,
                          double *f) {
    double rc2 = rc * rc, U = 0.0;
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double dx, dy, dz;
            double r2 = pair_r2(pos, box, i, j, &dx, &dy, &dz);
            if (!(r2 < rc2)) continue;
            int t = types[i] * nt + types[j];
            double fs = lj_fscalar(r2, eps[t], sigma[t]);
            double Fx = -fs * dx, Fy = -fs * dy, Fz = -fs * dz;
            f[3 * i + 0] += Fx; f[3 * i + 1] += Fy; f[3 * i + 2] += Fz;
            f[3 * j + 0] -= Fx; f[3 * j + 1] -= Fy; f[3 * j + 2] -= Fz;
            U += lj_phi(r2, eps[t], sigma[t]) - lj_phi(rc2, eps[t], sigma[t]);
        }
    }
    return U;
}

double orc_lj_typed_list(int64_t n, const double *pos, const double *box, int32_t nt,
                         const int32_t *types, const double *eps, const double *sigma, double rc,
                         const int64_t *offsets, const int32_t *ids, double *f, double *e_atom) {
    double rc2 = rc * rc, U = 0.0;
    #pragma omp parallel for schedule(dynamic, 256) reduction(+ : U)
    for (int64_t i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0, fz = 0.0, ei = 0.0;
        for (int64_t k = offsets[i]; k < offsets[i + 1]; ++k) {
            int64_t j = ids[k];
            double dx, dy, dz;
            double r2 = pair_r2(pos, box, i, j, &dx, &dy, &dz);
            if (!(r2 < rc2)) continue;
            int t = types[i] * nt + types[j];
            double fs = lj_fscalar(r2, eps[t], sigma[t]);
            fx -= fs * dx; fy -= fs * dy; fz -= fs * dz;
            ei += 0.5 * (lj_phi(r2, eps[t], sigma[t]) - lj_phi(rc2, eps[t], sigma[t]));
        }
        f[3 * i + 0] = fx; f[3 * i + 1] = fy; f[3 * i + 2] = fz;
        if (e_atom) e_atom[i] = ei;
        U += ei;
    }
    return U;
}

/* Sutton-Chen instance of the many-body form of Eq. 1 and Eq. 2:
 *   U = sum_i F(rho_i) + 1/2 sum_{i != j} Phi(r_ij),  rho_i = sum_{j != i} psi(r_ij)
 *   Phi(r) = eps (a/r)^n,  psi(r) = (a/r)^m,  F(rho) = -eps c sqrt(rho)
 * truncated (no shift) at r_c.  Forces by differentiating U:
 *   f_i = -sum_{j != i} [Phi'(r) + (F'(rho_i) + F'(rho_j)) psi'(r)] (r_i - r_j)/r
 * Evaluated in the paper's three steps (Sec. 3.1): a pair pass for rho, an
 * atom pass for F and F', and a pair pass for Phi and the forces. */
static double sc_pow(double x, double e) { return pow(x, e); }

static void sc_rho_from_list(int64_t n, const double *pos, const double *box, double a,
                             double m_exp, double rc, const int64_t *offsets,
                             const int32_t *ids, double *rho) {
    double rc2 = rc * rc;
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t k = offsets[i]; k < offsets[i + 1]; ++k) {
            double dx, dy, dz;
            double r2 = pair_r2(pos, box, i, ids[k], &dx, &dy, &dz);
            if (!(r2 < rc2)) continue;
            s += sc_pow(a / sqrt(r2), m_exp);
        }
        rho[i] = s;
    }
}

/* SC from a full neighbour list.  rho_out, dF_out (F'(rho_i)) and e_atom are
 * optional outputs.  Returns U. */
double orc_sc_list(int64_t n, const double *pos, const double *box, double eps, double a,
                   double c, double n_exp, double m_exp, double rc, const int64_t *offsets,
                   const int32_t *ids, double *f, double *rho_out, double *dF_out,
                   double *e_atom) {
    double rc2 = rc * rc;
    double *rho = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *dF = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *Femb = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    /* step 1: localization function rho_i (Eq. 2) */
    sc_rho_from_list(n, pos, box, a, m_exp, rc, offsets, ids, rho);
    /* step 2: embedding energy F(rho_i) and its derivative, atom loop */
    for (int64_t i = 0; i < n; ++i) {
        double sr = sqrt(rho[i]);
        Femb[i] = -eps * c * sr;
        dF[i] = (rho[i] > 0.0) ? -eps * c / (2.0 * sr) : 0.0;
    }
    /* step 3: pair interaction and forces */
    double U = 0.0;
    #pragma omp parallel for schedule(dynamic, 256) reduction(+ : U)
    for (int64_t i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0, fz = 0.0, ep = 0.0;
        for (int64_t k = offsets[i]; k < offsets[i + 1]; ++k) {
            int64_t j = ids[k];
            double dx, dy, dz;
            double r2 = pair_r2(pos, box, i, j, &dx, &dy, &dz);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            double Phi = eps * sc_pow(a / r, n_exp);
            double psi = sc_pow(a / r, m_exp);
            double dPhi = -n_exp * Phi / r;
            double dpsi = -m_exp * psi / r;
            double g = dPhi + (dF[i] + dF[j]) * dpsi;  /* dU/dr_ij */
            /* f_i += -g (r_i - r_j)/r = g d / r with d = r_j - r_i */
            fx += g * dx / r; fy += g * dy / r; fz += g * dz / r;
            ep += 0.5 * Phi;
        }
        f[3 * i + 0] = fx; f[3 * i + 1] = fy; f[3 * i + 2] = fz;
        double ei = ep + Femb[i];
        if (e_atom) e_atom[i] = ei;
        U += ei;
    }
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)n);
    if (dF_out) memcpy(dF_out, dF, sizeof(double) * (size_t)n);
    free(rho); free(dF); free(Femb);
    return U;
}

/* SC over all pairs (O(N^2)), same three steps without a list. */
double orc_sc_brute(int64_t n, const double *pos, const double *box, double eps, double a,
                    double c, double n_exp, double m_exp, double rc, double *f,
                    double *rho_out) {
    double rc2 = rc * rc;
    double *rho = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *dF = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double dx, dy, dz;
            double r2 = pair_r2(pos, box, i, j, &dx, &dy, &dz);
            if (!(r2 < rc2)) continue;
            double psi = sc_pow(a / sqrt(r2), m_exp);
            rho[i] += psi;
            rho[j] += psi;
        }
    double U = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double sr = sqrt(rho[i]);
        U += -eps * c * sr;
        dF[i] = (rho[i] > 0.0) ? -eps * c / (2.0 * sr) : 0.0;
    }
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double dx, dy, dz;
            double r2 = pair_r2(pos, box, i, j, &dx, &dy, &dz);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2);
            double Phi = eps * sc_pow(a / r, n_exp);
            double psi = sc_pow(a / r, m_exp);
            double g = -n_exp * Phi / r + (dF[i] + dF[j]) * (-m_exp * psi / r);
            f[3 * i + 0] += g * dx / r; f[3 * i + 1] += g * dy / r; f[3 * i + 2] += g * dz / r;
            f[3 * j + 0] -= g * dx / r; f[3 * j + 1] -= g * dy / r; f[3 * j + 2] -= g * dz / r;
            U += Phi;
        }
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)n);
    free(rho); free(dF);
    return U;
}

/* Embedded-atom method with piecewise functions, the form of the paper's Fe
 * potential (Sec. 3.1: pair and density functions that are sums of truncated
 * cubics, which is why the force step dominates for Fe126 in Table 2):
 *   Phi(r) = sum_k a_k (r_k - r)^3 for the knots with r < r_k
 *   psi(r) = sum_k b_k (s_k - r)^3 for the knots with r < s_k
 *   F(rho) = -A sqrt(rho) + B rho^2
 * in the many-body form of Eq. 1-2, cut at r_c (every knot <= r_c).  Forces
 * by differentiating U as for Sutton-Chen:
 *   f_i = -sum_j [Phi'(r) + (F'(rho_i) + F'(rho_j)) psi'(r)] (r_i - r_j)/r
 * evaluated in the paper's three steps (Sec. 3.1). */
typedef struct orc_eam_s {
    int32_t n_phi, n_psi;
    double phi_r[16], phi_a[16];
    double psi_r[16], psi_a[16];
    double F_sqrt, F_quad;
} orc_eam;

/* value (*d = derivative) of sum_k c_k (k_k - r)^3 over the knots beyond r */
static double piecewise_cubic(int nk, const double *knot, const double *c, double r, double *d) {
    double v = 0.0, dv = 0.0;
    for (int k = 0; k < nk; ++k) {
        if (r < knot[k]) {
            double t = knot[k] - r;
            v += c[k] * t * t * t;
            dv += -3.0 * c[k] * t * t;
        }
    }
    if (d) *d = dv;
    return v;
}
static double eam_F(const orc_eam *t, double rho) {
    return -t->F_sqrt * sqrt(rho) + t->F_quad * rho * rho;
}
static double eam_dF(const orc_eam *t, double rho) {
    double d = 2.0 * t->F_quad * rho;
    if (rho > 0.0) d += -t->F_sqrt / (2.0 * sqrt(rho));
    return d;
}

/* EAM from a full neighbour list; rho_out, dF_out (F'(rho_i)) and e_atom are
 * optional outputs.  Returns U. */
double orc_eam_list(int64_t n, const double *pos, const double *box, const orc_eam *t,
                    double rc, const int64_t *offsets, const int32_t *ids, double *f,
                    double *rho_out, double *dF_out, double *e_atom) {
    double rc2 = rc * rc;
    double *rho = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *dF = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    /* step 1: localization function rho_i (Eq. 2) */
    #pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        double sum = 0.0;
        for (int64_t k = offsets[i]; k < offsets[i + 1]; ++k) {
            double dx, dy, dz;
            double r2 = pair_r2(pos, box, i, ids[k], &dx, &dy, &dz);
            if (!(r2 < rc2)) continue;
            sum += piecewise_cubic(t->n_psi, t->psi_r, t->psi_a, sqrt(r2), NULL);
        }
        rho[i] = sum;
    }
    /* step 2: embedding derivative, atom loop */
    for (int64_t i = 0; i < n; ++i) dF[i] = eam_dF(t, rho[i]);
    /* step 3: pair term and forces */
    double U = 0.0;
    #pragma omp parallel for schedule(dynamic, 256) reduction(+ : U)
    for (int64_t i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0, fz = 0.0, ep = 0.0;
        for (int64_t k = offsets[i]; k < offsets[i + 1]; ++k) {
            int64_t j = ids[k];
            double dx, dy, dz;
            double r2 = pair_r2(pos, box, i, j, &dx, &dy, &dz);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2), dPhi, dpsi;
            double Phi = piecewise_cubic(t->n_phi, t->phi_r, t->phi_a, r, &dPhi);
            piecewise_cubic(t->n_psi, t->psi_r, t->psi_a, r, &dpsi);
            double g = dPhi + (dF[i] + dF[j]) * dpsi;  /* dU/dr_ij */
            fx += g * dx / r; fy += g * dy / r; fz += g * dz / r;
            ep += 0.5 * Phi;
        }
        f[3 * i + 0] = fx; f[3 * i + 1] = fy; f[3 * i + 2] = fz;
        double ei = ep + eam_F(t, rho[i]);
        if (e_atom) e_atom[i] = ei;
        U += ei;
    }
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)n);
    if (dF_out) memcpy(dF_out, dF, sizeof(double) * (size_t)n);
    free(rho); free(dF);
    return U;
}

/* EAM over all pairs i < j (O(N^2)), same three steps without a list. */
double orc_eam_brute(int64_t n, const double *pos, const double *box, const orc_eam *t,
                     double rc, double *f, double *rho_out) {
    double rc2 = rc * rc;
    double *rho = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *dF = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double dx, dy, dz;
            double r2 = pair_r2(pos, box, i, j, &dx, &dy, &dz);
            if (!(r2 < rc2)) continue;
            double psi = piecewise_cubic(t->n_psi, t->psi_r, t->psi_a, sqrt(r2), NULL);
            rho[i] += psi;
            rho[j] += psi;
        }
    double U = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        U += eam_F(t, rho[i]);
        dF[i] = eam_dF(t, rho[i]);
    }
    memset(f, 0, sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double dx, dy, dz;
            double r2 = pair_r2(pos, box, i, j, &dx, &dy, &dz);
            if (!(r2 < rc2)) continue;
            double r = sqrt(r2), dPhi, dpsi;
            double Phi = piecewise_cubic(t->n_phi, t->phi_r, t->phi_a, r, &dPhi);
            piecewise_cubic(t->n_psi, t->psi_r, t->psi_a, r, &dpsi);
            double g = dPhi + (dF[i] + dF[j]) * dpsi;
            f[3 * i + 0] += g * dx / r; f[3 * i + 1] += g * dy / r; f[3 * i + 2] += g * dz / r;
            f[3 * j + 0] -= g * dx / r; f[3 * j + 1] -= g * dy / r; f[3 * j + 2] -= g * dz / r;
            U += Phi;
        }
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)n);
    free(rho); free(dF);
    return U;
}

/* Forces (and per-atom energies) of a sample of atoms, for systems too large
 * for the all-atom routines: the 27 cells around each sampled atom are
 * scanned for pairs with r^2 < r_c^2 (same definitions as above).  For the
 * many-body potential the density of every atom within r_c of a sampled atom
 * is needed, so rho is computed for the sample and for those neighbours.
 * idx[k] are original ids; f_out is nsamp x 3, e_out (optional) nsamp. */
static void sample_cells(int64_t n, const double *pos, const double *box, double r,
                         int32_t *ncell, int32_t **cell_of, int64_t **start, int64_t **order) {
    double inv_w[3];
    orc_cell_grid(box, r, ncell, inv_w);
    int64_t nc = (int64_t)ncell[0] * ncell[1] * ncell[2];
    *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    *start = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc + 1));
    *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    orc_bin(n, pos, ncell, inv_w, *cell_of, *start, *order);
}

/* neighbours of atom i within r (strict), via the cell grid; returns count,
 * writes up to cap original ids into out */
static int64_t cell_neighbors(int64_t i, const double *pos, const double *box, double r,
                              const int32_t *ncell, const int32_t *cell_of, const int64_t *start,
                              const int64_t *order, int64_t *out, int64_t cap) {
    double r2c = r * r;
    int64_t c = cell_of[i];
    int32_t cx = (int32_t)(c % ncell[0]);
    int32_t cy = (int32_t)((c / ncell[0]) % ncell[1]);
    int32_t cz = (int32_t)(c / ((int64_t)ncell[0] * ncell[1]));
    int32_t sx[3], sy[3], sz[3];
    int kx = stencil_1d(cx, ncell[0], sx), ky = stencil_1d(cy, ncell[1], sy),
        kz = stencil_1d(cz, ncell[2], sz);
    int64_t cnt = 0;
    for (int a = 0; a < kz; ++a)
        for (int b = 0; b < ky; ++b)
            for (int e = 0; e < kx; ++e) {
                int64_t cc = cell_id(sx[e], sy[b], sz[a], ncell);
                for (int64_t s = start[cc]; s < start[cc + 1]; ++s) {
                    int64_t j = order[s];
                    if (j == i) continue;
                    if (orc_pair_r2(pos, box, i, j) < r2c) {
                        if (cnt < cap) out[cnt] = j;
                        cnt += 1;
                    }
                }
            }
    return cnt;
}

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

int orc_forces_sample(const orc_params *p, int64_t n, const double *pos, const double *box,
                      int64_t nsamp, const int64_t *idx, double *f_out, double *e_out) {
    int32_t ncell[3];
    int32_t *cell_of;
    int64_t *start, *order;
    sample_cells(n, pos, box, p->rc, ncell, &cell_of, &start, &order);
    const int64_t CAP = 4096;
    int bad = 0;
    #pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
    for (int64_t k = 0; k < nsamp; ++k) {
        int64_t i = idx[k];
        int64_t *nb = (int64_t *)malloc(sizeof(int64_t) * CAP);
        int64_t *nb2 = (int64_t *)malloc(sizeof(int64_t) * CAP);
        int64_t cnt = cell_neighbors(i, pos, box, p->rc, ncell, cell_of, start, order, nb, CAP);
        if (cnt > CAP) { bad = 1; free(nb); free(nb2); continue; }
        qsort(nb, (size_t)cnt, sizeof(int64_t), cmp_i64);  /* ascending j, as the list routines */
        double fx = 0.0, fy = 0.0, fz = 0.0, ei = 0.0;
        if (p->potential == 0 && p->ntypes > 0) {
            double rc2 = p->rc * p->rc;
            for (int64_t q = 0; q < cnt; ++q) {
                double dx, dy, dz;
                double r2 = pair_r2(pos, box, i, nb[q], &dx, &dy, &dz);
                int t = p->types[i] * p->ntypes + p->types[nb[q]];
                double fs = lj_fscalar(r2, p->t_eps[t], p->t_sigma[t]);
                fx -= fs * dx; fy -= fs * dy; fz -= fs * dz;
                ei += 0.5 * (lj_phi(r2, p->t_eps[t], p->t_sigma[t]) -
                             lj_phi(rc2, p->t_eps[t], p->t_sigma[t]));
            }
        } else if (p->potential == 0) {
            double shift = lj_phi(p->rc * p->rc, p->eps, p->sigma);
            for (int64_t q = 0; q < cnt; ++q) {
                double dx, dy, dz;
                double r2 = pair_r2(pos, box, i, nb[q], &dx, &dy, &dz);
                double fs = lj_fscalar(r2, p->eps, p->sigma);
                fx -= fs * dx; fy -= fs * dy; fz -= fs * dz;
                ei += 0.5 * (lj_phi(r2, p->eps, p->sigma) - shift);
            }
        } else if (p->potential == 2) {
            /* EAM: step 1 for i and each neighbour j, step 2 for each, step 3 for i */
            const orc_eam *t = p->eam;
            double rho_i = 0.0;
            for (int64_t q = 0; q < cnt; ++q)
                rho_i += piecewise_cubic(t->n_psi, t->psi_r, t->psi_a,
                                         sqrt(orc_pair_r2(pos, box, i, nb[q])), NULL);
            double dFi = eam_dF(t, rho_i);
            double ep = 0.0;
            for (int64_t q = 0; q < cnt; ++q) {
                int64_t j = nb[q];
                int64_t c2 = cell_neighbors(j, pos, box, p->rc, ncell, cell_of, start, order,
                                            nb2, CAP);
                if (c2 > CAP) { bad = 1; break; }
                qsort(nb2, (size_t)c2, sizeof(int64_t), cmp_i64);
                double rho_j = 0.0;
                for (int64_t u = 0; u < c2; ++u)
                    rho_j += piecewise_cubic(t->n_psi, t->psi_r, t->psi_a,
                                             sqrt(orc_pair_r2(pos, box, j, nb2[u])), NULL);
                double dFj = eam_dF(t, rho_j);
                double dx, dy, dz;
                double r2 = pair_r2(pos, box, i, j, &dx, &dy, &dz);
                double r = sqrt(r2), dPhi, dpsi;
                double Phi = piecewise_cubic(t->n_phi, t->phi_r, t->phi_a, r, &dPhi);
                piecewise_cubic(t->n_psi, t->psi_r, t->psi_a, r, &dpsi);
                double g = dPhi + (dFi + dFj) * dpsi;
                fx += g * dx / r; fy += g * dy / r; fz += g * dz / r;
                ep += 0.5 * Phi;
            }
            ei = ep + eam_F(t, rho_i);
        } else {
            /* step 1 for i and each neighbour j, step 2 for each, step 3 for i */
            double rho_i = 0.0;
            for (int64_t q = 0; q < cnt; ++q)
                rho_i += sc_pow(p->sigma / sqrt(orc_pair_r2(pos, box, i, nb[q])), p->m_exp);
            double dFi = rho_i > 0.0 ? -p->eps * p->c / (2.0 * sqrt(rho_i)) : 0.0;
            double ep = 0.0;
            for (int64_t q = 0; q < cnt; ++q) {
                int64_t j = nb[q];
                int64_t c2 = cell_neighbors(j, pos, box, p->rc, ncell, cell_of, start, order,
                                            nb2, CAP);
                if (c2 > CAP) { bad = 1; break; }
                qsort(nb2, (size_t)c2, sizeof(int64_t), cmp_i64);
                double rho_j = 0.0;
                for (int64_t t = 0; t < c2; ++t)
                    rho_j += sc_pow(p->sigma / sqrt(orc_pair_r2(pos, box, j, nb2[t])), p->m_exp);
                double dFj = rho_j > 0.0 ? -p->eps * p->c / (2.0 * sqrt(rho_j)) : 0.0;
                double dx, dy, dz;
                double r2 = pair_r2(pos, box, i, j, &dx, &dy, &dz);
                double r = sqrt(r2);
                double Phi = p->eps * sc_pow(p->sigma / r, p->n_exp);
                double psi = sc_pow(p->sigma / r, p->m_exp);
                double g = -p->n_exp * Phi / r + (dFi + dFj) * (-p->m_exp * psi / r);
                fx += g * dx / r; fy += g * dy / r; fz += g * dz / r;
                ep += 0.5 * Phi;
            }
            ei = ep - p->eps * p->c * sqrt(rho_i);
        }
        f_out[3 * k + 0] = fx; f_out[3 * k + 1] = fy; f_out[3 * k + 2] = fz;
        if (e_out) e_out[k] = ei;
        free(nb); free(nb2);
    }
    free(cell_of); free(start); free(order);
    return bad ? ORC_ERR_CAPACITY : ORC_OK;
}

/* Neighbour list rows (r < r_list, ascending original id) of sampled atoms.
 * offsets has nsamp + 1 entries; returns the total or ORC_ERR_CAPACITY. */
int64_t orc_neighbors_sample(int64_t n, const double *pos, const double *box, double r_list,
                             int64_t nsamp, const int64_t *idx, int64_t *offsets, int32_t *ids,
                             int64_t cap) {
    int32_t ncell[3];
    int32_t *cell_of;
    int64_t *start, *order;
    sample_cells(n, pos, box, r_list, ncell, &cell_of, &start, &order);
    int64_t *nb = (int64_t *)malloc(sizeof(int64_t) * 4096);
    int64_t total = 0;
    offsets[0] = 0;
    int overflow = 0;
    for (int64_t k = 0; k < nsamp; ++k) {
        int64_t cnt = cell_neighbors(idx[k], pos, box, r_list, ncell, cell_of, start, order, nb, 4096);
        if (cnt > 4096) { overflow = 1; cnt = 4096; }
        qsort(nb, (size_t)cnt, sizeof(int64_t), cmp_i64);
        for (int64_t q = 0; q < cnt; ++q) {
            if (total < cap) ids[total] = (int32_t)nb[q];
            else overflow = 1;
            total += 1;
        }
        offsets[k + 1] = total;
    }
    free(nb); free(cell_of); free(start); free(order);
    return overflow ? ORC_ERR_CAPACITY : total;
}

/* ------------------------------------------------------------------------ */
/* velocity-Verlet MD (Sec. 3.3): half kick, drift, wrap, forces, half kick;  */
/* the list is rebuilt when an atom has moved more than half the skin since   */
/* the last build (or every rebuild_every steps when that is > 0).           */
/* ------------------------------------------------------------------------ */

static double wrap(double x, double L) {
    if (x < 0.0) x += L;
    if (x >= L) x -= L;
    return x;
}

typedef struct {
    int64_t *offsets;
    int32_t *ids;
    int64_t cap;
} orc_list;

static int build_list(int64_t n, const double *pos, const double *box, double r_list,
                      orc_list *L) {
    for (;;) {
        int64_t t = orc_neighbors_cells(n, pos, box, r_list, 0, L->offsets, L->ids, L->cap);
        if (t >= 0) return ORC_OK;
        if (t != ORC_ERR_CAPACITY) return (int)t;
        int64_t need = L->offsets[n];
        L->cap = need + need / 4 + 1024;
        free(L->ids);
        L->ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)L->cap);
        if (!L->ids) return ORC_ERR_INVALID;
    }
}

static double forces(const orc_params *p, int64_t n, const double *pos, const double *box,
                     const orc_list *L, double *f) {
    if (p->potential == 0 && p->ntypes > 0)
        return orc_lj_typed_list(n, pos, box, p->ntypes, p->types, p->t_eps, p->t_sigma, p->rc,
                                 L->offsets, L->ids, f, NULL);
    if (p->potential == 0)
        return orc_lj_list(n, pos, box, p->eps, p->sigma, p->rc, L->offsets, L->ids, f, NULL);
    if (p->potential == 2)
        return orc_eam_list(n, pos, box, p->eam, p->rc, L->offsets, L->ids, f, NULL, NULL, NULL);
    return orc_sc_list(n, pos, box, p->eps, p->sigma, p->c, p->n_exp, p->m_exp, p->rc,
                       L->offsets, L->ids, f, NULL, NULL, NULL);
}

/* mass of atom i: its species' mass for a multi-element system */
static double atom_mass(const orc_params *p, int64_t i) {
    return p->ntypes > 0 ? p->t_mass[p->types[i]] : p->mass;
}

static double kinetic(const orc_params *p, int64_t n, const double *vel) {
    if (p->ntypes == 0) {
        double s = 0.0;
        for (int64_t k = 0; k < 3 * n; ++k) s += vel[k] * vel[k];
        return 0.5 * p->mass * s;
    }
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) s += 0.5 * atom_mass(p, i) * vel[3 * i + d] * vel[3 * i + d];
    return s;
}

/* Runs nsteps velocity-Verlet steps in place on pos/vel (n x 3).  energies
 * (optional) receives (nsteps + 1) x 3 values (KE, PE, KE + PE) at steps
 * 0..nsteps; force_out (optional) receives the final forces.  Returns the
 * number of list builds (including the initial one) or a negative status. */
int64_t orc_md_run(const orc_params *p, int64_t n, double *pos, double *vel, const double *box,
                   int64_t nsteps, double *energies, double *force_out) {
    double r_list = p->rc + p->skin;
    double half_skin2 = 0.25 * p->skin * p->skin;
    orc_list L;
    L.cap = 128 * (n > 0 ? n : 1);
    L.offsets = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    L.ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)L.cap);
    double *f = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *xb = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!L.offsets || !L.ids || !f || !xb) return ORC_ERR_INVALID;
    int64_t builds = 0;
    int st = build_list(n, pos, box, r_list, &L);
    if (st != ORC_OK) return st;
    builds += 1;
    memcpy(xb, pos, sizeof(double) * 3 * (size_t)n);
    int64_t since = 0;
    double U = forces(p, n, pos, box, &L, f);
    if (energies) {
        double K = kinetic(p, n, vel);
        energies[0] = K; energies[1] = U; energies[2] = K + U;
    }
    for (int64_t s = 1; s <= nsteps; ++s) {
        for (int64_t i = 0; i < n; ++i) {
            double h = 0.5 * p->dt / atom_mass(p, i);
            for (int d = 0; d < 3; ++d) {
                vel[3 * i + d] += h * f[3 * i + d];
                pos[3 * i + d] = wrap(pos[3 * i + d] + p->dt * vel[3 * i + d], box[d]);
            }
        }
        since += 1;
        int rebuild = 0;
        if (p->rebuild_every > 0) {
            rebuild = (since >= p->rebuild_every);
        } else {
            for (int64_t i = 0; i < n && !rebuild; ++i) {
                double d2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    double dd = min_image(pos[3 * i + d] - xb[3 * i + d], box[d]);
                    d2 += dd * dd;
                }
                if (d2 > half_skin2) rebuild = 1;
            }
        }
        if (rebuild) {
            st = build_list(n, pos, box, r_list, &L);
            if (st != ORC_OK) return st;
            builds += 1;
            memcpy(xb, pos, sizeof(double) * 3 * (size_t)n);
            since = 0;
        }
        U = forces(p, n, pos, box, &L, f);
        for (int64_t i = 0; i < n; ++i) {
            double h = 0.5 * p->dt / atom_mass(p, i);
            for (int d = 0; d < 3; ++d) vel[3 * i + d] += h * f[3 * i + d];
        }
        if (energies) {
            double K = kinetic(p, n, vel);
            energies[3 * s + 0] = K; energies[3 * s + 1] = U; energies[3 * s + 2] = K + U;
        }
    }
    if (force_out) memcpy(force_out, f, sizeof(double) * 3 * (size_t)n);
    free(L.offsets); free(L.ids); free(f); free(xb);
    return builds;
}

/* One force evaluation (list build + forces) at the given positions, the unit
 * the CPU baseline times.  Returns U, or NaN on failure. */
double orc_forces_once(const orc_params *p, int64_t n, const double *pos, const double *box,
                       double *f) {
    orc_list L;
    L.cap = 128 * (n > 0 ? n : 1);
    L.offsets = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    L.ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)L.cap);
    if (!L.offsets || !L.ids) return NAN;
    if (build_list(n, pos, box, p->rc + p->skin, &L) != ORC_OK) return NAN;
    double U = forces(p, n, pos, box, &L, f);
    free(L.offsets); free(L.ids);
    return U;
}

/* ------------------------------------------------------------------------ */
/* per-cell cost model: 3 -> 32 -> 32 -> 1 multilayer perceptron, ReLU,      */
/* mean-squared-error loss, Adam update (Kingma & Ba).  Parameter layout:    */
/*   W1[32][3], b1[32], W2[32][32], b2[32], W3[32], b3[1]  (1217 values)     */
/* ------------------------------------------------------------------------ */

#define H 32
#define NPAR (H * 3 + H + H * H + H + H + 1)

int orc_mlp_nparams(void) { return NPAR; }

static void mlp_one(const double *P, const double *x, double *z1, double *a1, double *z2,
                    double *a2, double *y) {
    const double *W1 = P, *b1 = P + 3 * H, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H,
                 *b3 = W3 + H;
    for (int u = 0; u < H; ++u) {
        double s = b1[u];
        for (int k = 0; k < 3; ++k) s += W1[3 * u + k] * x[k];
        z1[u] = s;
        a1[u] = s > 0.0 ? s : 0.0;
    }
    for (int u = 0; u < H; ++u) {
        double s = b2[u];
        for (int k = 0; k < H; ++k) s += W2[H * u + k] * a1[k];
        z2[u] = s;
        a2[u] = s > 0.0 ? s : 0.0;
    }
    double s = b3[0];
    for (int k = 0; k < H; ++k) s += W3[k] * a2[k];
    *y = s;
}

void orc_mlp_forward(int64_t ns, const double *X, const double *P, double *y) {
    double z1[H], a1[H], z2[H], a2[H];
    for (int64_t s = 0; s < ns; ++s) mlp_one(P, X + 3 * s, z1, a1, z2, a2, &y[s]);
}

/* Loss = (1/ns) sum_s (y_hat_s - y_s)^2 and its gradient dL/dP by the chain
 * rule (backpropagation), same layout as P. */
double orc_mlp_loss_grad(int64_t ns, const double *X, const double *y, const double *P,
                         double *G) {
    const double *W2 = P + 3 * H + H, *W3 = W2 + H * H + H;
    double *gW1 = G, *gb1 = G + 3 * H, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H,
           *gb3 = gW3 + H;
    memset(G, 0, sizeof(double) * NPAR);
    double z1[H], a1[H], z2[H], a2[H], d2[H], d1[H], yh, loss = 0.0;
    for (int64_t s = 0; s < ns; ++s) {
        const double *x = X + 3 * s;
        mlp_one(P, x, z1, a1, z2, a2, &yh);
        double e = yh - y[s];
        loss += e * e;
        double dy = 2.0 * e / (double)ns;
        gb3[0] += dy;
        for (int k = 0; k < H; ++k) {
            gW3[k] += dy * a2[k];
            d2[k] = (z2[k] > 0.0) ? dy * W3[k] : 0.0;
        }
        for (int u = 0; u < H; ++u) {
            gb2[u] += d2[u];
            for (int k = 0; k < H; ++k) gW2[H * u + k] += d2[u] * a1[k];
        }
        for (int k = 0; k < H; ++k) {
            double s2 = 0.0;
            for (int u = 0; u < H; ++u) s2 += W2[H * u + k] * d2[u];
            d1[k] = (z1[k] > 0.0) ? s2 : 0.0;
        }
        for (int u = 0; u < H; ++u) {
            gb1[u] += d1[u];
            for (int k = 0; k < 3; ++k) gW1[3 * u + k] += d1[u] * x[k];
        }
    }
    return loss / (double)ns;
}

/* One Adam step at step number t (1-based): m = b1 m + (1 - b1) g,
 * v = b2 v + (1 - b2) g^2, P -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + e). */
void orc_adam(int64_t np, double *P, const double *G, double *m, double *v, int64_t t,
              double lr, double beta1, double beta2, double epsilon) {
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (int64_t k = 0; k < np; ++k) {
        m[k] = beta1 * m[k] + (1.0 - beta1) * G[k];
        v[k] = beta2 * v[k] + (1.0 - beta2) * G[k] * G[k];
        P[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + epsilon);
    }
}

/* Contiguous equal-cost partition of cells over nparts workers: part b starts
 * at the first cell k whose inclusive cost prefix P_k satisfies
 * P_k * nparts > b * total (integer arithmetic).  bounds has nparts + 1
 * entries, bounds[0] = 0 and bounds[nparts] = ncells. */
void orc_partition(int64_t ncells, const int64_t *cost, int32_t nparts, int64_t *bounds) {
    int64_t total = 0;
    for (int64_t k = 0; k < ncells; ++k) total += cost[k];
    bounds[0] = 0;
    int64_t prefix = 0, k = 0;
    for (int32_t b = 1; b < nparts; ++b) {
        while (k < ncells && (prefix + cost[k]) * (int64_t)nparts <= (int64_t)b * total) {
            prefix += cost[k];
            k += 1;
        }
        bounds[b] = k;
    }
    bounds[nparts] = ncells;
}
