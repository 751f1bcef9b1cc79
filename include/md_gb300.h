/*
 * md_gb300.h -- C ABI of the GB300 (sm_103a) short-range molecular-dynamics
 * hot path: cell binning, Verlet neighbour lists with skin, pair (Lennard-
 * Jones) and many-body (Sutton-Chen) forces, and velocity-Verlet integration.
 *
 * The problem statement follows Mangiardi & Meyer, "A hybrid algorithm for
 * parallel molecular dynamics simulations": N atoms in a periodic box, a
 * short-range potential with cutoff r_c, Verlet lists of radius
 * r_list = r_c + skin (Sec. 2.1, Sec. 3.3), pair forces
 * F = -(1/d) dPhi/dr R with R = r_i - r_j (Sec. 2.2), many-body energy
 * U = sum_i F_i(rho_i) + 1/2 sum_{i != j} Phi_ij(r_ij) with
 * rho_i = sum_{j != i} psi_ij(r_ij) (Eq. 1, Eq. 2) evaluated in three steps
 * (Sec. 3.1), and velocity-Verlet time stepping with list rebuilds when an
 * atom has moved more than half the skin (Sec. 3.3).
 *
 * Conventions for every call:
 *  - Arrays passed by the caller are caller-owned.  Pointer arguments named
 *    *_dev are DEVICE pointers, *_host are HOST pointers.  Positions,
 *    velocities and forces are n x 3 float64, xyz interleaved, in ORIGINAL
 *    atom order (the order given to md_create).
 *  - The library owns a private, cell-sorted copy of the state on the GPU;
 *    it allocates it in md_create and frees it in md_destroy.
 *  - Work is enqueued on the CUDA stream given to md_create.  Calls that
 *    return host values (md_energy, md_stats, md_get_neighbors' total) or
 *    that must inspect device status (md_step) synchronize that stream.
 *  - Every call returns an md_status.  Nothing calls exit() or traps on the
 *    device.  After MD_ERR_STATE the handle must be destroyed; after any
 *    other error it stays usable, and md_last_error(h) describes the error.
 *  - Not thread-safe per handle; distinct handles are independent.
 */
#ifndef MD_GB300_H
#define MD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct md_system md_system; /* opaque, library-owned */

typedef enum {
    MD_OK = 0,
    MD_ERR_INVALID = -1,       /* bad argument, box or parameter */
    MD_ERR_OOM = -2,           /* device allocation failed */
    MD_ERR_CUDA = -3,          /* a CUDA runtime call failed */
    MD_ERR_LIST_OVERFLOW = -4, /* neighbour capacity exceeded (md_step regrows and retries) */
    MD_ERR_NONFINITE = -5,     /* a position or force became NaN/Inf */
    MD_ERR_TIMEOUT = -6,       /* a bounded device wait gave up (reserved: no kernel of this
                                  library waits on another, so no call returns it) */
    MD_ERR_STATE = -7          /* handle unusable: destroy it */
} md_status;

enum { MD_POT_LJ = 0, MD_POT_SC = 1, MD_POT_EAM = 2 };
enum { MD_FP64 = 0, MD_MIXED = 1 };
/* Newton's-third-law strategy (Sec. 1 race problem, Sec. 2.2 pair loop), and
 * the cluster-pair layout the paper compares its SIMD scheme with (Sec. 4.1):
 * MD_FORCE_CLUSTER evaluates the full pair set from a list of (i-cluster of up
 * to 8 atoms, j-cluster of up to 4 atoms) pairs whose bounding boxes come
 * within r_list, one warp per i-cluster; the per-atom list is still built
 * (for md_get_neighbors).  Mixed-precision one-species Lennard-Jones of one
 * box under MD_SCHED_GRID, n < 2^25.
 * MD_FORCE_PAIRED clusters the home side only, by two (Sec. 4.1's point that
 * grouping atoms saves neighbour loads): each thread owns two consecutive
 * atoms of one cell and walks the union of their lists, so that one gathered
 * neighbour position serves two pair evaluations.  The full pair set, the
 * same forces as MD_FORCE_FULL up to float32 rounding.  Its rebuilds make the
 * slot lists only; md_get_neighbors builds per-atom rows on demand from the
 * positions of the last build.  Mixed precision: one-species Lennard-Jones
 * in one box under any scheduler (the persistent kernel then takes tiles of
 * 32 slots) or in a batch (md_create_batch) under MD_SCHED_GRID, each slot
 * with its box's geometry; multi-element Lennard-Jones (md_create_typed),
 * Sutton-Chen and the embedded-atom potential (both passes over the slots)
 * under MD_SCHED_GRID.  MD_FORCE_CLUSTER is a measured alternative (slower on GB300);
 * MD_FORCE_PAIRED is faster than the per-atom list on large systems. */
enum { MD_FORCE_FULL = 0, MD_FORCE_HALF_COLOR = 1, MD_FORCE_HALF_ATOMIC = 2,
       MD_FORCE_CLUSTER = 3, MD_FORCE_PAIRED = 4 };
/* How force work is spread over the SMs.  The static schedulers cut the
 * cells into equal-cost ranges per persistent CTA and leave the last fifth
 * of the cost as a tail that CTAs claim tile by tile when their ranges are
 * done.  The learned model is trained on the mixed kernel's timings, so the
 * float64 path partitions by list length under MD_SCHED_MLP too. */
enum {
    MD_SCHED_GRID = 0,      /* one thread per atom, hardware block scheduler */
    MD_SCHED_PAIRCOUNT = 1, /* persistent CTAs, static partition by list length */
    MD_SCHED_MLP = 2,       /* persistent CTAs, static partition by the learned cost model */
    MD_SCHED_DYNAMIC = 3    /* persistent CTAs pulling tiles from an atomic queue */
};
enum {
    MD_COST_TRAIN = 0,   /* Adam epochs on the stored samples */
    MD_COST_PREDICT = 1, /* infer per-cell costs, rebuild the partition */
    MD_COST_RESET = 2,   /* re-initialise the weights */
    MD_COST_SAMPLE = 3,  /* timed force passes -> per-cell training samples */
    MD_COST_PROFILE = 4  /* one timed force pass: max / mean CTA busy cycles */
};

typedef struct {
    int32_t potential;     /* MD_POT_LJ or MD_POT_SC */
    int32_t precision;     /* MD_FP64 (plain) or MD_MIXED (fp32 pair math, fp64 state) */
    int32_t force_variant; /* MD_FORCE_* */
    int32_t rebuild_every; /* 0: rebuild when an atom moved > skin/2 (Sec. 3.3); k>0: every k steps */
    int32_t scheduler;     /* MD_SCHED_* */
    int32_t max_neighbors; /* list capacity per atom; 0 = sized from the first build */
    int32_t reserved0;
    int32_t reserved1;
    double eps;            /* LJ epsilon / SC epsilon */
    double sigma;          /* LJ sigma / SC lattice parameter a */
    double c;              /* SC c (ignored for LJ) */
    double n_exp;          /* SC pair exponent n (integer valued, 1..30) */
    double m_exp;          /* SC density exponent m (integer valued, 1..30) */
    double rc;             /* potential cutoff r_c > 0 */
    double skin;           /* list skin >= 0; r_list = rc + skin */
    double dt;             /* time step */
    double mass;           /* atom mass > 0 */
} md_params;

/* Creates a system of n >= 1 atoms in the orthorhombic periodic box
 * box3_host[3] (each side must hold at least 3 list radii, so that the 27
 * cells around any cell are distinct).  pos_dev / vel_dev: n x 3 float64
 * device arrays; both are copied, and positions are wrapped into [0, L) on
 * the way in (any finite value is accepted).  cuda_stream: a
 * cudaStream_t (NULL = legacy default stream).  Bins atoms (Sec. 2.1),
 * builds the first list with capacity from a counting pass, and evaluates
 * forces.  Energy is L/J units of the potential. */
md_status md_create(md_system **out, const md_params *p, int64_t n, const double *box3_host,
                    const double *pos_dev, const double *vel_dev, void *cuda_stream);

/* Piecewise embedded-atom functions, the form of the paper's Fe potential
 * (Sec. 3.1; its force step dominates Table 2 because such pieces
 * vectorise poorly): the many-body energy of Eq. 1-2 with
 *   Phi(r) = sum_k phi_a[k] (phi_r[k] - r)^3   over the knots with r < phi_r[k]
 *   psi(r) = sum_k psi_a[k] (psi_r[k] - r)^3   over the knots with r < psi_r[k]
 *   F(rho) = -F_sqrt sqrt(rho) + F_quad rho^2
 * and forces f_i = -sum_j [Phi'(r) + (F'(rho_i) + F'(rho_j)) psi'(r)]
 * (r_i - r_j) / r over r < r_c.  1 <= n_phi, n_psi <= MD_EAM_MAX_KNOTS, every
 * knot in (0, r_c]. */
#define MD_EAM_MAX_KNOTS 16
typedef struct {
    int32_t n_phi;
    int32_t n_psi;
    double phi_r[MD_EAM_MAX_KNOTS];
    double phi_a[MD_EAM_MAX_KNOTS];
    double psi_r[MD_EAM_MAX_KNOTS];
    double psi_a[MD_EAM_MAX_KNOTS];
    double F_sqrt;
    double F_quad;
} md_eam;

/* md_create for the embedded-atom potential: p->potential must be
 * MD_POT_EAM (p->eps, sigma, c, n_exp and m_exp are not used); eam_host is a
 * host struct, copied.  Full lists under MD_SCHED_GRID; md_get_density
 * reports rho_i and F'(rho_i).  MD_ERR_INVALID for bad tables. */
md_status md_create_eam(md_system **out, const md_params *p, const md_eam *eam_host, int64_t n,
                        const double *box3_host, const double *pos_dev, const double *vel_dev,
                        void *cuda_stream);

/* Multi-element Lennard-Jones, the GPU counterpart of the paper's Cu-Au
 * Alloy and Layer systems (Sec. 3.1), whose SIMD loop reloads each pair's
 * parameters with masks (Sec. 2.2): ntypes species (1..MD_MAX_TYPES); the
 * pair (i, j) uses eps[t_i * ntypes + t_j] and sigma[...] (symmetric
 * matrices) with its energy shifted to zero at r_c, and atom i has mass
 * mass[t_i].  The md_params fields eps, sigma and mass are not used. */
#define MD_MAX_TYPES 4
typedef struct {
    int32_t ntypes;
    int32_t reserved;
    double eps[MD_MAX_TYPES * MD_MAX_TYPES];
    double sigma[MD_MAX_TYPES * MD_MAX_TYPES];
    double mass[MD_MAX_TYPES];
} md_lj_types;

/* md_create for a multi-element Lennard-Jones system: p->potential must be
 * MD_POT_LJ; types_host (copied) holds the species parameters and type_dev
 * (device, n int32 in original order, 0 <= t < ntypes) each atom's species.
 * Full lists under MD_SCHED_GRID, fp64 or mixed precision, or two atoms per
 * thread (MD_FORCE_PAIRED, mixed precision; a slot's atoms may be of two
 * species, each lane of the pair arithmetic with its own parameters).  The species
 * travels with the atom through binning (two spare bits above the original
 * id in its float32 position word), so the pair loop reads j's species from
 * the position it loads anyway and selects the pair's parameters from the
 * row of i's species held in registers.  MD_ERR_INVALID for bad species,
 * asymmetric or non-positive parameters. */
md_status md_create_typed(md_system **out, const md_params *p, const md_lj_types *types_host,
                          const int32_t *type_dev, int64_t n, const double *box3_host,
                          const double *pos_dev, const double *vel_dev, void *cuda_stream);

/* A batch of n_replicas independent systems advanced together: replica r
 * has n_each_host[r] atoms in the box box3_each_host[3r .. 3r+2]; pos_dev /
 * vel_dev hold all replicas' atoms one replica after the other (n = sum of
 * n_each).  Every step of the path runs as one launch over all replicas (the
 * cells of all boxes are numbered consecutively), so small replicas do not
 * pay one launch each.  Batches run mixed-precision Lennard-Jones with full
 * lists under MD_SCHED_GRID or MD_SCHED_DYNAMIC, or two atoms per thread
 * (MD_FORCE_PAIRED) under MD_SCHED_GRID; the list is rebuilt for all
 * replicas when any replica needs it.  All other calls work on the whole
 * batch (original order = the concatenation); md_get_cells reports global
 * cell ids (replica r's cells follow those of replicas 0..r-1, each box in
 * its own x-fastest order) and ncell_host = {total cells, 1, 1}. */
md_status md_create_batch(md_system **out, const md_params *p, int32_t n_replicas,
                          const int64_t *n_each_host, const double *box3_each_host,
                          const double *pos_dev, const double *vel_dev, void *cuda_stream);

/* Kinetic and potential energy of every replica (host arrays of n_replicas;
 * 1 for md_create systems); a fresh force evaluation.  Synchronizes. */
md_status md_energy_batch(md_system *h, double *ke_host, double *pe_host);

/* Cell binning only (Sec. 2.1): assigns each atom to cell
 * c = min(floor(x * n_d / L_d), n_d - 1) per dimension, n_d = floor(L_d /
 * r_list), linear id (cz * ny + cy) * nx + cx, and reorders the private copy
 * stably by (cell, original id).  Under MD_FORCE_PAIRED each cell of up to
 * 32 atoms is put in a pairing order instead (ranked by the Morton code of
 * the position at 1/8 of the cell width; the first unpaired atom takes its
 * nearest unpaired cell mate), so the atoms 2k and 2k + 1 that form slot k
 * are near neighbours.  Either order is deterministic and invisible to the
 * exports, which are in original order.  Invalidates the neighbour list. */
md_status md_bin_cells(md_system *h);

/* Rebuilds the Verlet list from the current positions (bins first).  An
 * entry j of atom i means r_ij^2 < r_list^2 computed in float64 as
 * dx*dx + dy*dy + dz*dz on minimum-image components. */
md_status md_build_neighbors(md_system *h);

/* Forces (and per-atom energies) at the current positions, rebuilding the
 * list first when it is stale.  Pair potentials follow the pair loop of
 * Sec. 2.2, f_i = sum_j -(1/d) dPhi/dr (r_i - r_j) over list entries with
 * r < r_c; the many-body potential follows Eq. 1-2 in the three steps of
 * Sec. 3.1 (density, embedding derivative, forces).  Asynchronous. */
md_status md_forces(md_system *h);

/* Advances nsteps >= 0 velocity-Verlet steps (Sec. 3.3).  Lists are rebuilt
 * on the device when the half-skin rule (or rebuild_every) asks for it; a
 * neighbour-capacity overflow is repaired on the host (capacity grown,
 * list rebuilt) and the remaining steps continue.  On a non-default stream
 * the steps replay CUDA graphs captured on first use, the rebuild chain
 * under a conditional node set from the device's rebuild flag; on the
 * default stream every kernel is launched on its own.  Synchronizes the
 * stream once at the end to read the device status word. */
md_status md_step(md_system *h, int64_t nsteps);

/* Kinetic and potential energy at the current state (host outputs).  The
 * potential energy is U of Eq. 1 (for a pair potential its F term is zero:
 * U = 1/2 sum_{i != j} Phi(r_ij) over r < r_c) from a fresh force
 * evaluation; KE = 1/2 m sum_i |v_i|^2 with the full-step velocities of the
 * velocity-Verlet scheme of Sec. 3.3.  Synchronizes. */
md_status md_energy(md_system *h, double *ke_host, double *pe_host);

/* Copies the state out in original atom order; any pointer may be NULL.
 * The state is that of the velocity-Verlet scheme of Sec. 3.3 between two
 * steps: positions x(t) wrapped into [0, L), full-step velocities v(t), and
 * (force_dev) the forces f(t) of the last force evaluation (Sec. 2.2). */
md_status md_get_state(md_system *h, double *pos_dev, double *vel_dev, double *force_dev);

/* Replaces positions and velocities (original order, device arrays;
 * positions wrapped into [0, L) on the way in): the state x(t), v(t) of the
 * velocity-Verlet scheme of Sec. 3.3.  The next force evaluation rebinds
 * the cells (Sec. 2.1) and rebuilds the list, as after any list-invalidating
 * move (Sec. 3.3), so a restored state continues like an uninterrupted run
 * that rebuilt its list at the same step. */
md_status md_set_state(md_system *h, const double *pos_dev, const double *vel_dev);

/* Exports the current Verlet list (Sec. 2.1: built per cell from the 27
 * surrounding cells; Sec. 3.3: radius r_list = r_c + skin) as CSR in
 * original order: offsets_dev[n + 1] (int64) and ids_dev (int32 original
 * ids, ascending within each row).
 * half != 0 keeps only j > i.  cap = capacity of ids_dev in entries.
 * *total_host receives the entry count; if it exceeds cap nothing is
 * written to ids_dev and MD_ERR_LIST_OVERFLOW is returned.  Synchronizes. */
md_status md_get_neighbors(md_system *h, int32_t half, int64_t *offsets_dev, int32_t *ids_dev,
                           int64_t cap, int64_t *total_host);

/* Cell of every atom (original order, int32 device array of n) and, if
 * cell_start_dev != NULL, the sorted cell starts (int64, ncells + 1).
 * ncell_host[3] receives the cells per dimension.  Synchronizes. */
md_status md_get_cells(md_system *h, int32_t *cell_of_atom_dev, int64_t *cell_start_dev,
                       int32_t *ncell_host);

/* Many-body intermediate results of the last force evaluation (Sutton-
 * Chen or embedded-atom; original order, float64 device arrays of n): rho_i
 * (Eq. 2) and F'(rho_i).  Either pointer may be NULL. */
md_status md_get_density(md_system *h, double *rho_dev, double *dF_dev);

/* Per-atom potential energy of the last force evaluation with energy
 * (md_energy), original order, float64 device array of n. */
md_status md_get_atom_energy(md_system *h, double *e_dev);

/* Switches the force strategy and scheduler of an existing system (same
 * potential and precision) and rebuilds what the new choice needs (the list
 * when switching between full and half lists, the cell partition for the
 * static schedulers).  Half lists (Newton's third law, each pair once, owned
 * by the lower original id) are built for one-species Lennard-Jones on
 * either path and the cluster layout for its mixed path; the two-atom layout
 * serves the mixed path of every potential (multi-element Lennard-Jones,
 * Sutton-Chen and the embedded-atom potential, and batches, under
 * MD_SCHED_GRID); the persistent schedulers drive the one-box, one-species
 * full-list Lennard-Jones pass of either precision and its two-atom pass,
 * and every other combination runs one thread per atom (per slot, per
 * i-cluster). */
md_status md_set_variant(md_system *h, int32_t force_variant, int32_t scheduler);

/* Colour of every cell of an ncell_host[0] x [1] x [2] grid (each >= 3) as
 * used by MD_FORCE_HALF_COLOR: same-colour cells have disjoint 27-cell
 * neighbourhoods, so their force tasks never touch the same atom (the
 * conflict-free schedule of Sec. 2.1).  color_host (may be NULL) receives
 * one int32 per cell in linear cell order; *ncolors_host the colour count.
 * Host-only; touches no GPU. */
md_status md_color_cells(const int32_t *ncell_host, int32_t *color_host, int32_t *ncolors_host);

/* Learned per-cell cost model (3 -> 32 -> 32 -> 1 MLP, ReLU, fp32).
 *  MD_COST_SAMPLE  time one force pass with per-tile clock64 and store
 *                  per-cell (features, log cycles) training samples
 *  MD_COST_TRAIN   run Adam epochs on the stored samples on the GPU;
 *                  *loss_out (host, may be NULL) receives the final loss
 *  MD_COST_PREDICT infer per-cell costs and rebuild the static partition
 *  MD_COST_RESET   re-initialise the network weights */
md_status md_cost_model(md_system *h, int32_t op, float *loss_out);

/* Per-launch timing: with on != 0 the library records a CUDA event after
 * each rebuild chain, force evaluation and integrator launch it enqueues
 * (on the handle's stream) and md_stats reports the summed milliseconds and
 * counts per kind, plus the number of kernels launched (those of a rebuild
 * chain only when it ran).  Resets the sums and the launch count.
 * Synchronizes. */
md_status md_set_timing(md_system *h, int32_t on);

/* The inner/outer split of the force pass that lets the paper's domain
 * decomposition communicate while it computes (Sec. 2.1, the seven-step
 * pair-force algorithm), on one GPU: the cell grid is cut into px x py x pz
 * virtual domains (blocks of cells, floor(c p / n) along each dimension).
 * Each force pass then (1) packs the float32 positions of atoms whose cell
 * touches a domain face into one send buffer, (2-3) copies it into a receive
 * buffer on a second stream -- the stand-in for the transfer between
 * domains --, (4) computes every atom's intra-domain forces meanwhile
 * (interior atoms finish their step there), (5) waits for the copy and
 * (6) adds the inter-domain forces of the boundary atoms, their foreign
 * neighbours read from the receive buffer.  Forces equal the fused pass's up
 * to the order of float32 partial sums.  (1, 1, 1) switches it off.  For the
 * mixed-precision one-species Lennard-Jones full list of one box under
 * MD_SCHED_GRID; MD_ERR_INVALID otherwise or for more domains than cells.
 * Captured step graphs are dropped; the split steps are captured again, both
 * streams joined by events. */
md_status md_set_decomposition(md_system *h, int32_t px, int32_t py, int32_t pz);

/* Shape of the static partition used by MD_SCHED_PAIRCOUNT and MD_SCHED_MLP
 * (the load-balance question of Sec. 1 and Sec. 2.1 for inhomogeneous
 * systems): rounds = equal-cost ranges per persistent CTA (1..16; 0 = sized
 * from the system, about 24 tiles of 32 work items per range), tail_percent
 * = share of the estimated cost left as a tail that CTAs claim tile by tile
 * once their ranges are done (0..80; -1 = the layout's default, measured:
 * 20 for the per-atom list, 40 for two atoms per thread).  tail_percent = 0
 * makes the partition purely static, so the cost estimate alone balances
 * the CTAs.  Recomputes the partition; captured step graphs are dropped.
 * MD_ERR_INVALID outside those ranges. */
md_status md_set_schedule(md_system *h, int32_t rounds, int32_t tail_percent);

/* Per-cell view of the cost model (after MD_COST_SAMPLE), each array of
 * ncells in linear cell order, any pointer may be NULL (device arrays):
 *   cycles_dev     float32 measured force-pass cycles of the cell, summed
 *                  over the sampling passes
 *   predicted_dev  int64 cost the trained network predicts (what the
 *                  MD_SCHED_MLP partition uses)
 *   paircount_dev  int64 list entries of the cell's atoms (what the
 *                  MD_SCHED_PAIRCOUNT partition uses)
 * Synchronizes. */
md_status md_get_cell_costs(md_system *h, float *cycles_dev, int64_t *predicted_dev,
                            int64_t *paircount_dev);

/* Writes a one-line JSON summary (atoms, cells, list capacity, rebuild
 * count, steps, last kernel times) into buf_host (NUL-terminated, at most
 * cap bytes).  Synchronizes. */
md_status md_stats(md_system *h, char *buf_host, size_t cap);

/* Last error message of h (or of the calling thread when h is NULL). */
const char *md_last_error(md_system *h);

void md_destroy(md_system *h);

/* ---- building blocks exposed for parity tests and tools --------------- */

/* Forward pass of the cost model on ns samples: X_dev ns x 3 fp32,
 * P_dev parameters (layout W1[32][3], b1[32], W2[32][32], b2[32], W3[32],
 * b3[1]; 1217 fp32), y_dev ns fp32 outputs.  Asynchronous on stream. */
md_status md_mlp_forward(const float *X_dev, int64_t ns, const float *P_dev, float *y_dev,
                         void *cuda_stream);

/* Mean-squared-error loss and its gradient over ns samples (fp32):
 * G_dev (1217 fp32) receives dL/dP, loss_dev (1 fp32) the loss.
 * Asynchronous on stream. */
md_status md_mlp_loss_grad(const float *X_dev, const float *y_dev, int64_t ns,
                           const float *P_dev, float *G_dev, float *loss_dev,
                           void *cuda_stream);

/* One Adam step (Kingma & Ba) at 1-based step t on np fp32 parameters. */
md_status md_mlp_adam(float *P_dev, const float *G_dev, float *m_dev, float *v_dev, int64_t np,
                      int64_t t, float lr, float beta1, float beta2, float epsilon,
                      void *cuda_stream);

/* Contiguous equal-cost partition of ncells integer costs into nparts:
 * bounds_dev[b] = first cell k with (inclusive prefix of cost through k) *
 * nparts > b * total; bounds_dev[0] = 0, bounds_dev[nparts] = ncells.
 * Costs must be >= 0 with total * nparts < 2^63 (the comparisons are exact
 * int64 products; larger sums give wrong bounds).  Asynchronous on stream. */
md_status md_partition(const int64_t *cost_dev, int64_t ncells, int32_t nparts,
                       int64_t *bounds_dev, void *cuda_stream);

/* md_partition for callers that cannot allocate device memory while they
 * run -- a loop that fixed its memory budget at start-up, a host framework
 * whose allocator owns the device heap, or a setup without stream-ordered
 * allocation.  The paper has no counterpart; this is a service of the
 * library.  Same arguments and result as md_partition, but the scan scratch
 * is a fixed array inside the library's device image (about 8.4 MB, held on
 * every GPU that loads the library until the process exits) instead of a
 * cudaMallocAsync buffer, so the call allocates nothing.
 *  - ncells must be <= 1,048,576; larger sizes return MD_ERR_INVALID and
 *    md_last_error(NULL) says why (use md_partition for them).
 *  - The first call on a device looks up the array's device address with
 *    cudaGetSymbolAddress (once per device, with that device current) and
 *    keeps it for the life of the process; make that first call before any
 *    stream capture.  A device reset (cudaDeviceReset) while the library
 *    stays loaded is not supported: the kept address would be stale.
 *  - Costs must be >= 0 with total * nparts < 2^63, as for md_partition.
 *  - All calls share the one array and nothing in it needs to start at zero
 *    (the scan overwrites every word it reads).  Calls that overlap on the
 *    GPU -- different streams, or different host threads -- race on it; the
 *    caller must order them.
 * Asynchronous on stream. */
md_status md_partition_noalloc(const int64_t *cost_dev, int64_t ncells, int32_t nparts,
                               int64_t *bounds_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* MD_GB300_H */
