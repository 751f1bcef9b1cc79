// k_sched.cu -- per-cell work estimates for the persistent force kernel.
//
// The paper balances the force work of inhomogeneous systems by running one
// task per cell under a dynamic schedule (Sec. 2.1) and reports how density
// fluctuations unbalance static decompositions (Sec. 1).  Here the cells are
// split into contiguous ranges of (predicted) equal cost, one range per
// resident CTA, by one of two estimates:
//   pair count  cost(c) = list entries of the atoms of c (of the two-atom
//               slots of c under MD_FORCE_PAIRED: the work units there)
//   learned     cost(c) = exp(10 y) - 1, y = MLP(features of c)
// Features of cell c, scaled to O(1):
//   x0 = log1p(atoms in c) / 3
//   x1 = log1p(list entries of c's atoms, or of its slots) / 8
//   x2 = log1p(atoms in the 26 neighbour cells) / 6
// Training targets come from the persistent kernel's clock64 timing:
//   y = log1p(cycles of c) / 10.
#include <cmath>

#include "k_scan.cuh"

namespace mdg {

namespace {

constexpr float kX0 = 1.f / 3.f, kX1 = 1.f / 8.f, kX2 = 1.f / 6.f, kY = 10.f;

__device__ __forceinline__ bool chain_off(const DevStatus *ds, bool gated) {
    return ds != nullptr && (ds->status != 0 || (gated && ds->rebuild == 0));
}

// start: first atom of every cell; item_start / item_count: the force pass's
// work units (atoms, or two-atom slots) of every cell and their list lengths
__global__ void cell_features_kernel(int ncells, Grid g, const int32_t *__restrict__ start,
                                     const int32_t *__restrict__ item_start,
                                     const int32_t *__restrict__ item_count, int cap,
                                     float *__restrict__ X, long long *__restrict__ paircost,
                                     const DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
    const int b = start[c], e = start[c + 1];
    long long np = 0;
    for (int i = item_start[c]; i < item_start[c + 1]; ++i) np += min(item_count[i], cap);
    const int cx = c % g.nx, cy = (c / g.nx) % g.ny, cz = c / (g.nx * g.ny);
    int occ = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                const int xx = (cx + dx + g.nx) % g.nx, yy = (cy + dy + g.ny) % g.ny,
                          zz = (cz + dz + g.nz) % g.nz;
                const int cn = (zz * g.ny + yy) * g.nx + xx;
                occ += start[cn + 1] - start[cn];
            }
    X[3 * (size_t)c] = log1pf((float)(e - b)) * kX0;
    X[3 * (size_t)c + 1] = log1pf((float)np) * kX1;
    X[3 * (size_t)c + 2] = log1pf((float)occ) * kX2;
    if (paircost) paircost[c] = np;
    }
}

__global__ void quantize_kernel(int ncells, const float *__restrict__ y,
                                const int32_t *__restrict__ start, long long *__restrict__ cost,
                                const DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        if (start[c + 1] == start[c]) {
            cost[c] = 0;
            continue;
        }
        const float v = expm1f(kY * fminf(y[c], 3.f));  // cap at e^30 against a diverged model
        cost[c] = (v >= 1.f) ? (long long)llrintf(v) : 1ll;
    }
}

__global__ void sample_flags_kernel(int ncells, const int32_t *__restrict__ start,
                                    int32_t *__restrict__ flag) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncells) flag[c] = (start[c + 1] > start[c]) ? 1 : 0;
}

__global__ void sample_scatter_kernel(int ncells, const int32_t *__restrict__ flag,
                                      const int32_t *__restrict__ pos,
                                      const float *__restrict__ X,
                                      const float *__restrict__ cycles, float inv_passes,
                                      float *__restrict__ sX, float *__restrict__ sy,
                                      int32_t *__restrict__ count) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) *count = pos[ncells];
    if (c >= ncells || !flag[c]) return;
    const int k = pos[c];
    sX[3 * (size_t)k] = X[3 * (size_t)c];
    sX[3 * (size_t)k + 1] = X[3 * (size_t)c + 1];
    sX[3 * (size_t)k + 2] = X[3 * (size_t)c + 2];
    sy[k] = log1pf(cycles[c] * inv_passes) / kY;
}

}  // namespace

cudaError_t launch_cell_features(md_system *h, bool paircount, bool gated) {
    const int nc = h->g.ncells;
    const bool slots = (h->p.force_variant == MD_FORCE_PAIRED);
    cell_features_kernel<<<gs_blocks(nc), kBlock, 0, h->stream>>>(
        nc, h->g, h->cell_start, slots ? h->ps_start : h->cell_start,
        slots ? h->ps_count : h->ncount, slots ? h->ps_cap : h->cap, h->cell_X,
        paircount ? h->cell_cost : nullptr, h->ds, gated);
    return cudaGetLastError();
}

cudaError_t launch_predict_costs(md_system *h, bool gated) {
    const int nc = h->g.ncells;
    cudaError_t e = launch_mlp_forward(h->cell_X, nc, h->mlp_P, h->cell_pred, h->stream, h->ds,
                                       gated);
    if (e != cudaSuccess) return e;
    quantize_kernel<<<gs_blocks(nc), kBlock, 0, h->stream>>>(nc, h->cell_pred, h->cell_start,
                                                          h->cell_cost, h->ds, gated);
    return cudaGetLastError();
}

cudaError_t launch_partition_cells(md_system *h, bool gated) {
    return launch_partition(h->cell_cost, h->g.ncells, sched_parts(h->sched_ctas, h->sched_rounds, h->sched_tail_pct), h->part_bounds,
                            h->part_scratch, h->stream, h->ds, gated);
}

cudaError_t launch_make_samples(md_system *h, int passes, int32_t *samp_count_dev) {
    const int nc = h->g.ncells;
    int32_t *flag = h->samp_flag;
    int32_t *pos = h->samp_flag + (nc + 1);
    sample_flags_kernel<<<nblocks(nc), kBlock, 0, h->stream>>>(nc, h->cell_start, flag);
    cudaError_t e = launch_scan<int32_t>(flag, pos, nc, h->samp_bsum, nullptr, false, h->stream);
    if (e != cudaSuccess) return e;
    sample_scatter_kernel<<<nblocks(nc), kBlock, 0, h->stream>>>(
        nc, flag, pos, h->cell_X, h->cell_cycles, 1.f / (float)passes, h->samp_X, h->samp_y,
        samp_count_dev);
    return cudaGetLastError();
}

}  // namespace mdg
