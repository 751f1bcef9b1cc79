// md_internal.cuh -- private types and launcher declarations of the GB300
// molecular-dynamics library.  Included by every translation unit of the
// library; never installed.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/md_gb300.h"

namespace mdg {

constexpr int kBlock = 256;       // threads per block of the per-atom kernels
constexpr int kStencil = 27;      // cells scanned around a cell (Sec. 2.1)
constexpr int kIndexBits = 27;    // list entry = (stencil << 27) | sorted index
constexpr uint32_t kIndexMask = (1u << kIndexBits) - 1u;
constexpr int64_t kMaxAtoms = (int64_t)1 << kIndexBits;
// share of the estimated cost in the dynamically claimed tail of the static
// schedulers (percent): default and largest accepted by md_set_schedule
constexpr int kTailPctDefault = 20;  // per-atom layout
constexpr int kTailPctPaired = 40;   // two-atom layout (measured: 20 % left it 15 % slower)
constexpr int kTailPctMax = 80;

// Neighbour-list layout.  Atoms are grouped by 32 (one warp); inside a group
// each atom's entries are stored in quads: uint32 [n/32][cap/4][32][4].  A
// lane reads its quad q with one 16-byte load, and the 32 lanes' loads of quad
// q are 512 contiguous bytes.  cap is a multiple of 4.  Every list is padded
// to a multiple of 4 entries with kPadStencil entries pointing at the atom
// itself: that image lies at (w_x, w_y, w_z), at least sqrt(3) r_list away,
// so every cutoff test rejects it and the pair loops need no tail handling.
constexpr uint32_t kPadStencil = 26;  // stencil cell (+1, +1, +1)

__host__ __device__ __forceinline__ size_t list_group(int i, int cap) {
    return (size_t)(i >> 5) * (size_t)cap * 32;
}
__host__ __device__ __forceinline__ size_t list_idx(int i, int k, int cap) {
    return list_group(i, cap) + (size_t)(k >> 2) * 128 + (size_t)((i & 31) << 2) + (size_t)(k & 3);
}

// Cell colouring for the half-list force pass without atomics.  Per
// dimension of n >= 3 cells, cells below m = 3 floor(n / 3) take colour
// c mod 3 and the (n - m) tail cells take colours 3, 4.  Two distinct cells
// of one colour then differ by >= 3 cells (periodically) in some dimension,
// so their 27-cell neighbourhoods -- everything a cell's atoms may write --
// are disjoint.  Colours per dimension: 3 + n mod 3.
__host__ __device__ __forceinline__ int color_1d(int c, int n) {
    const int m = (n / 3) * 3;
    return c < m ? c % 3 : 3 + (c - m);
}
__host__ __device__ __forceinline__ int colors_1d(int n) { return 3 + n % 3; }
// number of cells of colour k along a dimension of n cells
__host__ __device__ __forceinline__ int color_count_1d(int k, int n) {
    return k < 3 ? n / 3 : 1;
}
// t-th cell of colour k along a dimension
__host__ __device__ __forceinline__ int color_cell_1d(int k, int t, int n) {
    return k < 3 ? k + 3 * t : (n / 3) * 3 + (k - 3);
}

// half lists (Newton's third law: each pair once) as opposed to the full pair
// set of the per-atom or the cluster-pair list
inline bool half_variant(int fv) { return fv == MD_FORCE_HALF_COLOR || fv == MD_FORCE_HALF_ATOMIC; }

// Device status word.  Every kernel of a step returns at entry when `status`
// is non-zero, so an error stops the rest of the enqueued work and the host
// finds the state exactly where it stopped.
struct DevStatus {
    int status;          // md_status of the first device-detected error
    int steps_done;      // last completed time step of the current md_step call
    int rebuild;         // 1: the next gated rebuild chain runs
    int since_build;     // steps since the last list build
    int abs_fresh;       // 1: xabs holds the positions exactly (no drift since)
    int max_count;       // largest neighbour count of the last build
    int max_cell;        // largest cell occupancy of the last binning
    int builds;          // list builds so far
    unsigned int timeouts;  // bounded waits that gave up
    int pad0;
    unsigned long long list_entries;  // entries of the last list build
    unsigned long long pairs_cut;     // pairs inside r_c of the last energy evaluation
    int tile_counter;                 // dynamic scheduler: next unclaimed tile
    unsigned int done_ctas;           // dynamic scheduler: CTAs finished this launch
    long long cond_runs;              // rebuild chains run by a graph's IF node
    unsigned long long cluster_pairs; // (i-cluster, j-cluster) entries of the last cluster list
    unsigned long long pair_entries;  // entries of the last two-atom slot list
    int pair_max;                     // its longest row
    int pair_slots;                   // its slots
};

// What the persistent force kernel needs besides ForceArgs.
struct SchedArgs {
    const int32_t *cell_start;  // ncells + 1
    const long long *bounds;    // partition of cells: rounds * gridDim.x static ranges,
                                // then the tail's parts (bounds[last] = ncells)
    int rounds;                 // ranges per CTA (cyclic assignment)
    const int32_t *cell;        // sorted slot -> cell
    float *cell_cycles;         // TIMING: per-cell cycles (accumulated)
    float *cta_cycles;          // TIMING: per-CTA busy cycles
};

// Geometry of one periodic box and its cells.  A system may hold several
// independent boxes (replicas); their cells are numbered consecutively and
// cell0 is the first global cell id of this box.
struct Grid {
    int nx, ny, nz;
    int wsmall_hi;      // high word of 2^e, the largest power of two <= every cell width
    int ncells;
    int cell0;
    double L[3];
    double w[3];        // cell widths L / n
    double inv_w[3];    // n / L
    float wf[3];        // w and inv_w rounded to float32 (the two-atom layout's
    float inv_wf[3];    // float32 list build and pairing order)
    const double *ctab; // cell centres (c + 0.5) w: nx for x, then ny for y, then nz for z
};

// Periodic wrap into [0, L): x - L*floor(x/L), then one correction each
// way -- the rounded quotient can leave x a period off (a tiny negative x,
// or x just below a multiple of L), and x + L can round up to L itself.
__device__ __forceinline__ double wrap_coord(double x, double L) {
    if (x < 0.0 || x >= L) x -= L * floor(x / L);
    if (x < 0.0) x += L;
    if (x >= L) x -= L;
    return x;
}

// Centre of the box-local cell (cx, cy, cz), read from the box's table.  A
// stored centre makes every kernel that forms centre + offset (or position -
// centre) round the same single addition.
__device__ __forceinline__ double3 cell_centre_of(int cx, int cy, int cz, const Grid &g) {
    return make_double3(g.ctab[cx], g.ctab[g.nx + cy], g.ctab[g.nx + g.ny + cz]);
}

// |v| < 2^e <= the smallest cell width, from the exponent bits alone (false
// for NaN and infinities).
__device__ __forceinline__ bool below_cell_width(double v, const Grid &g) {
    return (__double2hiint(v) & 0x7fffffff) < g.wsmall_hi;
}

// Per-launch scalars of the force kernels.
struct ForceConsts {
    float rc2f, eps4f, eps48f, sig2f, shiftf;  // LJ in fp32
    double rc2, eps4, eps48, sig2, shift;        // LJ in fp64
    // Sutton-Chen
    float sc_af, sc_epsf, sc_ecf;  // a, eps, eps*c
    double sc_a, sc_eps, sc_ec;
    int sc_n, sc_m;
    // integrator
    double dt, inv_m;
    float half_skin2f;
    // multi-element Lennard-Jones: species count (0 = one species) and the
    // inverse mass of each species; an atom's species sits in bits 27-28 of
    // its float32 position's w word, above the original id
    int ntypes;
    double t_inv_m[4];
};

constexpr int kMaxTypes = 4;
// species of a position word: bits 27-28 above the original id
__host__ __device__ __forceinline__ int species_of(uint32_t w) { return (int)(w >> 27) & 3; }
__device__ __forceinline__ double pick4(const double *v, int t) {
    return t < 2 ? (t == 0 ? v[0] : v[1]) : (t == 2 ? v[2] : v[3]);
}

// Pair parameters of a multi-element Lennard-Jones system, [t_i * nt + t_j]:
// 48 eps, 4 eps, sigma^2 and the energy shift at r_c, in float32 and float64.
struct TypeTab {
    float e48[16], e4[16], s2[16], sh[16];
    double e48d[16], e4d[16], s2d[16], shd[16];
};

// Piecewise embedded-atom tables (MD_POT_EAM), passed to the kernels by value
// (parameter space: warp-uniform reads).  Knot radii r_k / s_k and
// coefficients a_k / b_k of Phi and psi, in float32 and float64; F(rho) =
// -A sqrt(rho) + B rho^2.
constexpr int kEamMaxKnots = 16;
struct EamTab {
    int nphi, npsi;
    float pr[kEamMaxKnots], pa[kEamMaxKnots], qr[kEamMaxKnots], qa[kEamMaxKnots];
    double prd[kEamMaxKnots], pad[kEamMaxKnots], qrd[kEamMaxKnots], qad[kEamMaxKnots];
    double A, B;
};

enum ForceMode {
    FM_STORE = 0,       // forces (and optional energies) to f
    FM_FUSED_FULL = 1,  // forces, kick dt, drift dt (two half kicks merged)
    FM_FUSED_HALF = 2,  // forces, closing half kick, store f
};

}  // namespace mdg

// The system handle (host structure; device arrays in sorted order).
struct md_system {
    md_params p;
    int64_t n = 0;
    cudaStream_t stream = nullptr;
    mdg::Grid g{};  // the box (the first box of a batch); g.ncells counts all cells

    // replicas (md_create_batch): R boxes, atoms of replica r are original ids
    // [atom_off[r], atom_off[r+1]) and cells [grids[r].cell0, + grids[r].ncells)
    int R = 1;
    std::vector<mdg::Grid> grids_h;
    std::vector<int64_t> atom_off_h;
    mdg::Grid *grids = nullptr;       // device copy of grids_h
    double *ctab = nullptr;           // cell-centre tables of all boxes (Grid::ctab)
    int64_t *atom_off = nullptr;      // device copy of atom_off_h
    uint16_t *rep = nullptr;          // sorted slot -> replica (batches only)
    float4 *shifts32 = nullptr;       // R x 27 float32 cell shifts (batches only)
    double *rep_ke = nullptr, *rep_pe = nullptr;  // per-replica sums (device)
    mdg::ForceConsts fc{};
    mdg::EamTab eam{};  // MD_POT_EAM only
    mdg::TypeTab types{};        // multi-element Lennard-Jones only
    int32_t *type_orig = nullptr;  // species of each atom, original order (typed only)
    double types_mass[4] = {0, 0, 0, 0};  // mass of each species (typed only)
    double r_list = 0.0;
    float list_lo = 0.f, list_hi = 0.f;  // fp32 prefilter band around r_list^2
    double rl2 = 0.0;

    // state, sorted order
    double4 *xr64[2] = {nullptr, nullptr};  // fp64 position relative to the cell centre
    float4 *xq[2] = {nullptr, nullptr};     // fp32 copy (w = original id bits)
    float4 *xq_build = nullptr;             // fp32 copy at the last build
    double4 *xabs = nullptr;                // absolute positions at the last rebuild
    double *v = nullptr;                    // velocities, 3 x n SoA
    double *f = nullptr;                    // forces of the last evaluation, 3 x n SoA
    double *e_atom = nullptr;               // per-atom potential energy
    int32_t *orig = nullptr;                // sorted slot -> original id
    int32_t *cell = nullptr;                // sorted slot -> cell (-1: xr64 holds absolute)
    int cur = 0;

    // binning
    int32_t *cell_start = nullptr;  // ncells + 1
    int32_t *cell_count = nullptr;  // ncells
    int32_t *new_cell = nullptr, *slot = nullptr, *src = nullptr, *key = nullptr;
    int32_t *scan_bsum = nullptr;
    double4 *tmp_abs = nullptr;  // gather records: (x, y, z, new cell | original id)
    double4 *tmp_v = nullptr;    //                 (vx, vy, vz, replica)

    // neighbour list: warp-interleaved [n/32][cap][32] entries + counts
    uint32_t *nlist = nullptr;
    int32_t *ncount = nullptr;
    int cap = 0;
    size_t nlist_entries = 0;

    // many-body
    double *rho = nullptr;
    float *dF32 = nullptr;
    float4 *xqf = nullptr;  // Sutton-Chen mixed: position with F'(rho) in w
    double *dF64 = nullptr;

    // reductions
    double *partials = nullptr;  // per-block partial sums
    double *red_out = nullptr;   // [0] = PE, [1] = KE
    int nblocks_n = 0;

    int64_t *exp_tmp = nullptr;  // scratch of md_get_neighbors

    // persistent scheduler and learned cost model (allocated on first use)
    int sched_ctas = 0;                 // resident CTAs of the persistent force kernel
    int sched_sms = 0;                  // SMs of the device (0: scheduler not set up)
    int sched_rounds = 1;               // static ranges per CTA (sched_rounds())
    int sched_rounds_set = 0;           // md_set_schedule: fixed ranges per CTA (0 = by size)
    int sched_tail_pct = mdg::kTailPctDefault;  // share of the cost in the tail
    bool sched_tail_set = false;                // md_set_schedule chose it (else the layout's)
    long long *part_bounds = nullptr;   // sched_parts(sched_ctas, sched_rounds) + 1 cell bounds
    long long *cell_cost = nullptr;     // quantised per-cell cost (ncells)
    long long *part_scratch = nullptr;  // prefix sums of the partition
    float *cell_X = nullptr;            // features, ncells x 3
    float *cell_pred = nullptr;         // model outputs, ncells
    float *cell_cycles = nullptr;       // measured per-cell cycles, ncells
    float *cta_cycles = nullptr;        // measured per-CTA cycles, sched_ctas
    int32_t *samp_flag = nullptr;       // ncells + 1 (non-empty flags, then their scan)
    int32_t *samp_bsum = nullptr;
    float *samp_X = nullptr, *samp_y = nullptr;  // training set, compacted
    int64_t samp_n = 0;
    float *mlp_P = nullptr, *mlp_G = nullptr, *mlp_m = nullptr, *mlp_v = nullptr;
    float *mlp_scratch = nullptr;       // gradient partials
    float *mlp_loss = nullptr;          // device scalar
    int64_t mlp_t = 0;                  // Adam step count
    bool partition_valid = false;

    // cluster-pair list (MD_FORCE_CLUSTER)
    int32_t *cl_icnt = nullptr, *cl_jcnt = nullptr;  // clusters per cell
    int32_t *cl_ioff = nullptr, *cl_joff = nullptr;  // their scans (ncells + 1)
    int32_t *cl_bsum = nullptr;
    uint32_t *cl_icl = nullptr;   // i-cluster: first atom | (size - 1) << 27
    int32_t *cl_icell = nullptr;  // i-cluster: cell
    float4 *cl_jbox = nullptr;    // j-cluster: box lo (w: first atom), hi (w: size)
    int32_t *cl_ntot = nullptr;   // [0] i-clusters, [1] j-clusters (device)
    uint32_t *cl_list = nullptr;  // rows of cl_cap entries per i-cluster
    int32_t *cl_row = nullptr;    // row lengths
    int cl_cap = 0;

    // two home atoms per thread (MD_FORCE_PAIRED)
    int32_t *ps_cnt = nullptr;     // slots per cell
    int32_t *ps_start = nullptr;   // their scan (ncells + 1)
    int32_t *ps_bsum = nullptr;
    uint32_t *ps_atom = nullptr;   // slot: first atom | 2^31 for a one-atom slot
    uint32_t *ps_list = nullptr;   // union lists, per-atom layout over slots
    int32_t *ps_count = nullptr;   // their lengths
    int ps_cap = 0;
    int atom_list_at = -1;         // build count when the per-atom rows were last made

    // inner/outer split of the force pass (md_set_decomposition)
    bool ov_on = false;
    int dd[3] = {1, 1, 1};               // virtual domains per dimension
    uint32_t *ov_cell_outer = nullptr;   // per cell: stencil cells in another domain (27 bits)
    int32_t *ov_flag = nullptr, *ov_pos = nullptr, *ov_bsum = nullptr;  // boundary flags, scan
    int32_t *ov_gidx = nullptr;          // sorted slot -> buffer slot (-1: interior atom)
    int32_t *ov_bidx = nullptr;          // buffer slot -> sorted slot
    int32_t *ov_nb = nullptr;            // boundary atom count (device)
    float4 *ov_send = nullptr, *ov_recv = nullptr;  // the exchange's buffers
    cudaStream_t ov_stream = nullptr;    // the exchange's stream
    cudaEvent_t ov_ev[2] = {nullptr, nullptr};

    mdg::DevStatus *ds = nullptr;       // device
    mdg::DevStatus *ds_host = nullptr;  // pinned mirror
    double *red_host = nullptr;         // pinned

    // captured full steps (one per double-buffer parity)
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};     // one full step, per parity
    cudaGraphExec_t gexec_rb[2] = {nullptr, nullptr};  // the rebuild chain alone, per parity
    long long graph_launches[2] = {0, 0};  // unconditional launches of gexec
    long long body_launches = 0;           // launches of the conditional rebuild chain
    bool graphs_ok = true;

    // per-launch timing (md_set_timing)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_kind;  // kind of the interval that ends at event k
    size_t ev_used = 0;
    double ms_kind[4] = {0, 0, 0, 0};      // rebuild, force, integrate, other
    long long n_kind[4] = {0, 0, 0, 0};
    long long launches = 0;                // kernels enqueued by this handle

    bool forces_valid = false;
    bool list_valid = false;
    int64_t steps_total = 0;
    int64_t rebuilds_host = 0;
    std::string last_error;
};

namespace mdg {

// ---- binning (k_bin.cu) --------------------------------------------------
// Gated chain: count per cell (with the absolute positions and gather
// records), scan, scatter, order each cell by original id, gather the new
// sorted state.  kBinLaunches kernels.
constexpr int kBinLaunches = 8;
cudaError_t launch_bin(md_system *h, bool gated);
// Exclusive scan of int32 counts into int32 starts (starts[n] = total).
cudaError_t launch_scan_i32(const int32_t *in, int32_t *out, int n, int32_t *bsum,
                            const DevStatus *ds, bool gated, cudaStream_t s);
// cell of each atom in original order; cell_start as int64
cudaError_t launch_export_cells(md_system *h, int32_t *cell_of_atom, int64_t *cell_start);

// ---- neighbour list (k_nlist.cu) ------------------------------------------
// positions: the float32 positions the list is built from (default: the
// current buffer, right after binning)
cudaError_t launch_build_list(md_system *h, bool write, bool gated,
                              const float4 *positions = nullptr);
cudaError_t launch_finish_rebuild(md_system *h, bool gated);
cudaError_t launch_export_list(md_system *h, int half, int64_t *offsets, int32_t *ids,
                               int64_t *row_counts_tmp);

// ---- forces (k_lj.cu, k_sc.cu) -------------------------------------------
cudaError_t launch_lj(md_system *h, int mode, bool energy, bool store_f);
// half-list LJ (mixed precision): zero f, force pass(es), integrate
cudaError_t launch_lj_half(md_system *h, int mode, bool energy, int *launches);
// persistent LJ kernel (mixed precision, full list); timing only with FM_STORE
cudaError_t launch_lj_persist(md_system *h, int mode, bool store_f, bool dynamic, bool timing);
int persist_ctas_per_sm(bool f64, bool paired);
cudaError_t launch_sc_density(md_system *h);
cudaError_t launch_sc_force(md_system *h, int mode, bool energy, bool store_f);
// cluster-pair list (k_cluster.cu): tables and list after a rebuild (10 kernels),
// one force kernel
int cluster_cap(int max_cell);
int64_t cluster_rows(int64_t n, int ncells);
cudaError_t launch_cluster_build(md_system *h, bool gated);
cudaError_t launch_cluster_forces(md_system *h, int mode, bool energy, bool store_f);
// inner/outer split (k_overlap.cu): boundary index after a rebuild (5 kernels),
// then per force pass assemble, exchange, inner and outer passes (4 kernels)
cudaError_t launch_overlap_index(md_system *h, bool gated);
cudaError_t launch_overlap_forces(md_system *h, int mode, bool energy, bool store_f);
// two atoms per thread (k_pair.cu): slot tables and union lists after a
// rebuild (7 kernels), one force kernel; the padding entries point at a
// dummy position at index n of both position buffers
int64_t pair_slots_max(int64_t n, int ncells);
cudaError_t launch_pair_dummy(md_system *h);
cudaError_t launch_pair_build(md_system *h, bool write, bool gated);
cudaError_t launch_pair_forces(md_system *h, int mode, bool energy, bool store_f);
cudaError_t launch_eam_density(md_system *h);  // k_eam.cu
cudaError_t launch_eam_force(md_system *h, int mode, bool energy, bool store_f);

// ---- integrator and state (k_integrate.cu) --------------------------------
cudaError_t launch_kick_drift(md_system *h);
cudaError_t launch_load_state(md_system *h, const double *pos, const double *vel);
cudaError_t launch_get_state(md_system *h, double *pos, double *vel, double *force);
cudaError_t launch_scatter_orig(md_system *h, const double *src_sorted, double *dst_orig);
cudaError_t launch_scatter_orig_f32(md_system *h, const float *src_sorted, double *dst_orig);
cudaError_t launch_replica_energy(md_system *h);  // per-replica PE and KE
cudaError_t launch_reduce_pe(md_system *h);
cudaError_t launch_reduce_ke(md_system *h);
cudaError_t launch_set_rebuild(md_system *h);

// ---- scheduler and cost model (k_sched.cu, k_mlp.cu) ----------------------
constexpr int kMlpParams = 1217;
// The static schedulers cut the cells into `rounds` ranges per CTA, plus a
// tail of sched_tail_parts() further equal-cost parts (a fifth of the total)
// that the persistent kernel hands out dynamically.  Rounds grow with the
// system so that a range keeps about kTilesPerRange 32-atom tiles, up to
// kSchedRounds (measured: one round at 1 M atoms, eight at 9.8 M).
constexpr int kSchedRounds = 16;
constexpr int kTilesPerRange = 24;
inline int sched_rounds(int64_t n, int ctas) {
    const int64_t r = ((n + 31) / 32) / ((int64_t)ctas * kTilesPerRange);
    return r < 1 ? 1 : (r > kSchedRounds ? kSchedRounds : (int)r);
}
// The tail holds tail_pct percent of the predicted cost: ctas * rounds equal
// static parts plus ctas * rounds * tail_pct / (100 - tail_pct) tail parts of
// the same cost (20 % by default: a quarter as many tail parts as static ones).
inline int sched_tail_parts(int ctas, int rounds, int tail_pct) {
    return (int)((long long)ctas * rounds * tail_pct / (100 - tail_pct));
}
inline int sched_parts(int ctas, int rounds, int tail_pct) {
    return ctas * rounds + sched_tail_parts(ctas, rounds, tail_pct);
}
// features of every cell; with paircount != 0 also cell_cost = list entries
cudaError_t launch_cell_features(md_system *h, bool paircount, bool gated);
// model inference on cell_X, quantised into cell_cost
cudaError_t launch_predict_costs(md_system *h, bool gated);
// equal-cost partition of cell_cost into part_bounds
cudaError_t launch_partition_cells(md_system *h, bool gated);
// training set: non-empty cells' features and log cycles (count to samp_count_dev)
cudaError_t launch_make_samples(md_system *h, int passes, int32_t *samp_count_dev);
cudaError_t launch_mlp_init(float *P, unsigned long long seed, cudaStream_t s);
cudaError_t launch_mlp_forward(const float *X, long long ns, const float *P, float *y,
                               cudaStream_t s, const DevStatus *ds = nullptr, bool gated = false);
size_t mlp_grad_scratch_floats(long long ns);
cudaError_t launch_mlp_loss_grad(const float *X, const float *Y, long long ns, const float *P,
                                 float *G, float *loss, float *scratch, cudaStream_t s);
cudaError_t launch_adam(float *P, const float *G, float *m, float *v, long long np, long long t,
                        float lr, float b1, float b2, float eps, cudaStream_t s);
cudaError_t launch_partition(const long long *cost, long long ncells, int nparts,
                             long long *bounds, long long *scratch, cudaStream_t s,
                             const DevStatus *ds = nullptr, bool gated = false);

// Message returned by md_last_error(NULL) on the calling thread.
void set_thread_error(const std::string &msg);

inline int nblocks(int64_t n, int b = kBlock) { return (int)((n + b - 1) / b); }

// Grids of the grid-stride kernels (rebuild chain): enough blocks to fill the
// GPU, few enough that a launch whose gate is closed costs microseconds.
constexpr int kGridCap = 152 * 8;
inline int gs_blocks(int64_t n) {
    const int b = nblocks(n);
    return b < 1 ? 1 : (b < kGridCap ? b : kGridCap);
}

}  // namespace mdg
