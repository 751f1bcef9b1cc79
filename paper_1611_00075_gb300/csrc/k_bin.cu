// k_bin.cu -- cell binning by counting sort (Sec. 2.1: the volume is divided
// into small cells; a cell's atoms are processed together).
//
// Atoms are assigned to cell c = min(floor(x * n_d / L_d), n_d - 1) per
// dimension, counted with atomics, the counts are scanned into cell starts,
// atoms are scattered into their cell's range and each cell's range is put in
// ascending original-id order, so the sorted layout is deterministic and
// equals a stable sort by (cell, original id).  For the two-atom layout,
// whose slots take a cell's atoms two at a time, each cell is instead put in
// a pairing order (cell_pair_order_kernel), also deterministic, that places
// near neighbours next to each other.  The gather then rewrites the
// state in the new order as float64 positions relative to the cell centre
// plus their float32 copy (the layout the force kernels read).
//
// Traffic: the counting pass also writes each atom's absolute position and
// velocity (with its original id, new cell and replica packed into the spare
// fourth words) into two 32-byte records, so the gather reads two aligned
// sectors per atom instead of seven scattered words.
//
// A system of several boxes (replicas) numbers its cells consecutively, box
// after box, so each box's atoms stay one contiguous range of the sorted
// order; every kernel reads the geometry of the atom's own box.
#include "k_scan.cuh"

#include <algorithm>
#include <climits>

namespace mdg {

namespace {

__device__ __forceinline__ bool chain_off(const DevStatus *ds, bool gated) {
    return ds->status != 0 || (gated && ds->rebuild == 0);
}

// floor(x * inv_w) clamped to [0, n-1] (one float64 floor-convert: the
// conversion saturates, and a NaN coordinate converts to 0, so an exploding
// state can never index outside the cell arrays; the drift check reports it
// as MD_ERR_NONFINITE).
__device__ __forceinline__ int cell_coord(double x, double inv_w, int n) {
    const int q = __double2int_rd(x * inv_w);
    return q < 0 ? 0 : (q > n - 1 ? n - 1 : q);
}

// Absolute position of sorted atom i: exact in xabs right after a build or a
// load (abs_fresh); otherwise the cell centre plus the relative position.  An
// atom of an interior cell whose offset is below the cell width lies strictly
// inside the box, so only boundary cells and stray offsets need the periodic
// wrap.  cell < 0: xr holds the absolute position (a loaded state).
__device__ __forceinline__ double3 absolute_position(int i, const Grid &g, bool fresh,
                                                     const double4 *__restrict__ xr,
                                                     const int32_t *__restrict__ cell,
                                                     const double4 *__restrict__ xabs) {
    if (fresh) {
        const double4 a = xabs[i];
        return make_double3(a.x, a.y, a.z);
    }
    const double4 r = xr[i];
    const int c = cell[i];
    double x = r.x, y = r.y, z = r.z;
    if (c >= 0) {
        const int cl = c - g.cell0;
        const int cx = cl % g.nx, cy = (cl / g.nx) % g.ny, cz = cl / (g.nx * g.ny);
        const double3 C = cell_centre_of(cx, cy, cz, g);
        x = C.x + x; y = C.y + y; z = C.z + z;
        if (cx == 0 || cx == g.nx - 1 || !below_cell_width(r.x, g)) x = wrap_coord(x, g.L[0]);
        if (cy == 0 || cy == g.ny - 1 || !below_cell_width(r.y, g)) y = wrap_coord(y, g.L[1]);
        if (cz == 0 || cz == g.nz - 1 || !below_cell_width(r.z, g)) z = wrap_coord(z, g.L[2]);
    } else {
        x = wrap_coord(x, g.L[0]); y = wrap_coord(y, g.L[1]); z = wrap_coord(z, g.L[2]);
    }
    return make_double3(x, y, z);
}

// Spare fourth words of the gather records: (new cell << 32 | original id)
// beside the position, the replica beside the velocity.
__device__ __forceinline__ double pack2(int hi, int lo) {
    return __longlong_as_double(((long long)hi << 32) | (long long)(unsigned)lo);
}

__global__ void zero_counts_kernel(int ncells, int32_t *count, DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ds->max_cell = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x)
        count[c] = 0;
}

// Cell of every atom, its slot in the cell (atomic count) and its gather
// records: (x, y, z, new cell | original id) and (v, replica).
__global__ void bin_count_kernel(int n, const Grid *__restrict__ grids,
                                 const uint16_t *__restrict__ rep,
                                 const double4 *__restrict__ xr,
                                 const int32_t *__restrict__ cell,
                                 const double4 *__restrict__ xabs,
                                 const double *__restrict__ v, const int32_t *__restrict__ orig,
                                 int32_t *__restrict__ count, int32_t *__restrict__ new_cell,
                                 int32_t *__restrict__ slot, double4 *__restrict__ tabs,
                                 double4 *__restrict__ tv, DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    const bool fresh = ds->abs_fresh != 0;
    int maxs = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = rep ? rep[i] : 0;
        const Grid &g = grids[r];
        const double3 x = absolute_position(i, g, fresh, xr, cell, xabs);
        const int cx = cell_coord(x.x, g.inv_w[0], g.nx);
        const int cy = cell_coord(x.y, g.inv_w[1], g.ny);
        const int cz = cell_coord(x.z, g.inv_w[2], g.nz);
        const int c = g.cell0 + (cz * g.ny + cy) * g.nx + cx;
        new_cell[i] = c;
        const int sl = atomicAdd(&count[c], 1);
        slot[i] = sl;
        maxs = max(maxs, sl + 1);
        tabs[i] = make_double4(x.x, x.y, x.z, pack2(c, orig[i]));
        tv[i] = make_double4(v[i], v[n + i], v[2 * (size_t)n + i], pack2(0, r));
    }
    // all lanes arrive here (grid-stride loop): one atomic per warp
    maxs = __reduce_max_sync(0xffffffffu, (unsigned)maxs);
    if ((threadIdx.x & 31) == 0 && maxs) atomicMax(&ds->max_cell, maxs);
}

__global__ void scatter_kernel(int n, const int32_t *__restrict__ new_cell,
                               const int32_t *__restrict__ slot,
                               const int32_t *__restrict__ start, const int32_t *__restrict__ orig,
                               int32_t *__restrict__ src, int32_t *__restrict__ key,
                               const DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int p = start[new_cell[i]] + slot[i];
        src[p] = i;
        key[p] = orig[i];
    }
}

// Orders each cell's range by original id.  One warp per cell: a cell of up
// to 32 atoms is ranked by shuffles (lane l's rank = how many keys of the cell
// are smaller; the keys are distinct original ids); a larger cell (dense
// systems) is insertion-sorted by one lane.
constexpr int kSortBlock = 256;

__device__ void insertion_sort_cell(int b, int m, int32_t *__restrict__ key,
                                    int32_t *__restrict__ src) {
    for (int a = b + 1; a < b + m; ++a) {
        const int k = key[a], sv = src[a];
        int q = a - 1;
        while (q >= b && key[q] > k) {
            key[q + 1] = key[q];
            src[q + 1] = src[q];
            --q;
        }
        key[q + 1] = k;
        src[q + 1] = sv;
    }
}

__global__ void __launch_bounds__(kSortBlock)
cell_sort_kernel(int ncells, const int32_t *__restrict__ start, int32_t *__restrict__ key,
                 int32_t *__restrict__ src, const DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (kSortBlock / 32);
    for (int c = blockIdx.x * (kSortBlock / 32) + (threadIdx.x >> 5); c < ncells; c += nw) {
        const int b = start[c], m = start[c + 1] - b;
        if (m <= 1) continue;
        if (m <= 32) {
            const int k = lane < m ? key[b + lane] : 0x7fffffff;
            const int sv = lane < m ? src[b + lane] : 0;
            int rank = 0;
            for (int q = 0; q < m; ++q) rank += (__shfl_sync(0xffffffffu, k, q) < k) ? 1 : 0;
            if (lane < m) {
                key[b + rank] = k;
                src[b + rank] = sv;
            }
        } else if (lane == 0) {
            insertion_sort_cell(b, m, key, src);
        }
    }
}

// three bits per axis interleaved (x lowest): the octree position of a point
// in its cell at 1/8 of the cell width
__device__ __forceinline__ unsigned morton9(unsigned qx, unsigned qy, unsigned qz) {
    auto spread = [](unsigned v) { return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4); };
    return spread(qx) | (spread(qy) << 1) | (spread(qz) << 2);
}

// the octree coordinate, from float32 position and inverse width (products
// and differences rounded one by one)
__device__ __forceinline__ unsigned octree_coord(float x, float inv_w) {
    const float t = __fmul_rn(x, inv_w);
    const int q = (int)__fmul_rn(__fsub_rn(t, floorf(t)), 8.0f);
    return (unsigned)min(max(q, 0), 7);
}

// float64 to float32 rounded toward zero, from the IEEE-754 fields with
// integer operations (the float64 pipe is slow on this part); a value below
// the float32 normal range, zero included, gives 0
__device__ __forceinline__ float f32_toward_zero(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    return e <= 0 ? 0.0f : __uint_as_float((hi & 0x80000000u) | ((unsigned)e << 23) | m);
}

// Pairing order for the two-atom layout, whose slot k of a cell holds the
// cell's sorted atoms 2k and 2k + 1: the union of two cut-off spheres grows
// with the distance between their centres, and a warp's loop runs as long as
// its longest slot list, so the pairs should be near neighbours.  One warp
// per cell of up to 32 atoms: the atoms are ranked by the Morton code of
// their octree position in the cell (ties by original id) and moved to the
// lane of their rank; then, while two or more are left, the first unpaired
// atom in rank takes the nearest unpaired atom (squared distance with its low
// 5 bits replaced by the rank, so ties go to the lower rank), and the two
// fill the next two places.  A cell of odd occupancy ends with the atom left
// over.  Positions are float32 (rounded toward zero from float64) and every
// product and sum is rounded on its own, so the order depends on positions
// and ids only and is deterministic; a larger cell falls back to the
// original-id order.
__global__ void __launch_bounds__(kSortBlock)
cell_pair_order_kernel(int ncells, const Grid *__restrict__ grids,
                       const uint16_t *__restrict__ rep, const int32_t *__restrict__ start,
                       const double4 *__restrict__ tabs, int32_t *__restrict__ key,
                       int32_t *__restrict__ src, const DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    constexpr unsigned full = 0xffffffffu;
    __shared__ int s_lane_of[kSortBlock / 32][32];
    int *lane_of = s_lane_of[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (kSortBlock / 32);
    for (int c = blockIdx.x * (kSortBlock / 32) + (threadIdx.x >> 5); c < ncells; c += nw) {
        const int b = start[c], m = start[c + 1] - b;
        if (m <= 1) continue;
        if (m > 32) {
            if (lane == 0) insertion_sort_cell(b, m, key, src);
            continue;
        }
        const bool on = lane < m;
        int o = on ? key[b + lane] : 0x7fffffff;
        int sv = on ? src[b + lane] : 0;
        const double4 a = on ? tabs[sv] : make_double4(0.0, 0.0, 0.0, 0.0);
        float px = f32_toward_zero(a.x), py = f32_toward_zero(a.y), pz = f32_toward_zero(a.z);
        // the cell's box (a cell's atoms share it; lane 0 always holds one)
        const Grid &g = grids[rep ? __shfl_sync(full, (int)rep[sv], 0) : 0];
        const float iwx = g.inv_wf[0], iwy = g.inv_wf[1], iwz = g.inv_wf[2];
        const unsigned mk =
            morton9(octree_coord(px, iwx), octree_coord(py, iwy), octree_coord(pz, iwz));
        const long long K = on ? (((long long)mk << 32) | (long long)o) : LLONG_MAX;
        int rank = 0;
        for (int q = 0; q < m; ++q) rank += (__shfl_sync(full, K, q) < K) ? 1 : 0;
        // lane r takes the atom of rank r
        if (on) lane_of[rank] = lane;
        __syncwarp();
        const int from = on ? lane_of[lane] : lane;
        __syncwarp();
        o = __shfl_sync(full, o, from);
        sv = __shfl_sync(full, sv, from);
        px = __shfl_sync(full, px, from);
        py = __shfl_sync(full, py, from);
        pz = __shfl_sync(full, pz, from);
        unsigned left = (m == 32) ? full : ((1u << m) - 1u);
        int dst = 0, next = 0;
        while (__popc(left) >= 2) {
            const int first = __ffs(left) - 1;
            const float fx = __shfl_sync(full, px, first), fy = __shfl_sync(full, py, first),
                        fz = __shfl_sync(full, pz, first);
            // atoms of one cell need no periodic image
            const float dx = __fsub_rn(px, fx), dy = __fsub_rn(py, fy), dz = __fsub_rn(pz, fz);
            const float d2 =
                __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
            const bool cand = ((left >> lane) & 1u) && lane != first;
            const unsigned k2 = cand ? ((__float_as_uint(d2) & ~31u) | (unsigned)lane) : full;
            const int mate = (int)(__reduce_min_sync(full, k2) & 31u);
            if (lane == first) dst = next;
            if (lane == mate) dst = next + 1;
            next += 2;
            left &= ~((1u << first) | (1u << mate));
        }
        if ((left >> lane) & 1u) dst = next;
        if (on) {
            key[b + dst] = o;
            src[b + dst] = sv;
        }
    }
}

__global__ void gather_kernel(int n, const Grid *__restrict__ grids,
                              const int32_t *__restrict__ src, const double4 *__restrict__ tabs,
                              const double4 *__restrict__ tv, double4 *__restrict__ xr,
                              float4 *__restrict__ xq, float4 *__restrict__ xq_build,
                              double4 *__restrict__ xabs, double *__restrict__ v,
                              int32_t *__restrict__ orig, int32_t *__restrict__ cell,
                              uint16_t *__restrict__ rep, const int32_t *__restrict__ type_orig,
                              DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ds->abs_fresh = 1;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int s = src[k];
        const double4 a = tabs[s];
        const double4 u = tv[s];
        const long long pa = __double_as_longlong(a.w);
        const int o = (int)(unsigned)(pa & 0xffffffffll);
        const int c = (int)(pa >> 32);
        const int r = (int)(__double_as_longlong(u.w) & 0xffff);
        const Grid &g = grids[r];
        const int cl = c - g.cell0;
        const double3 C = cell_centre_of(cl % g.nx, (cl / g.nx) % g.ny, cl / (g.nx * g.ny), g);
        const double rx = a.x - C.x, ry = a.y - C.y, rz = a.z - C.z;
        xr[k] = make_double4(rx, ry, rz, 0.0);
        // the float32 word carries the original id and, for a multi-element
        // system, the species above it
        const uint32_t w = (uint32_t)o | (type_orig ? (uint32_t)type_orig[o] << kIndexBits : 0u);
        const float4 q = make_float4((float)rx, (float)ry, (float)rz, __uint_as_float(w));
        xq[k] = q;
        xq_build[k] = q;
        xabs[k] = make_double4(a.x, a.y, a.z, 0.0);
        v[k] = u.x;
        v[n + k] = u.y;
        v[2 * (size_t)n + k] = u.z;
        orig[k] = o;
        cell[k] = c;
        if (rep) rep[k] = (uint16_t)r;
    }
}

__global__ void export_cells_kernel(int n, int ncells, const int32_t *__restrict__ orig,
                                    const int32_t *__restrict__ cell,
                                    const int32_t *__restrict__ start, int32_t *cell_of_atom,
                                    int64_t *cell_start) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && cell_of_atom) cell_of_atom[orig[i]] = cell[i];
    if (i <= ncells && cell_start) cell_start[i] = start[i];
}

}  // namespace

cudaError_t launch_scan_i32(const int32_t *in, int32_t *out, int n, int32_t *bsum,
                            const DevStatus *ds, bool gated, cudaStream_t s) {
    return launch_scan<int32_t>(in, out, n, bsum, ds, gated, s);
}

cudaError_t launch_bin(md_system *h, bool gated) {
    int n = (int)h->n;
    cudaStream_t s = h->stream;
    int cur = h->cur;
    zero_counts_kernel<<<gs_blocks(h->g.ncells), kBlock, 0, s>>>(h->g.ncells, h->cell_count,
                                                                 h->ds, gated);
    bin_count_kernel<<<gs_blocks(n), kBlock, 0, s>>>(n, h->grids, h->rep, h->xr64[cur], h->cell,
                                                     h->xabs, h->v, h->orig, h->cell_count,
                                                     h->new_cell, h->slot, h->tmp_abs, h->tmp_v,
                                                     h->ds, gated);
    cudaError_t e = launch_scan_i32(h->cell_count, h->cell_start, h->g.ncells, h->scan_bsum,
                                    h->ds, gated, s);
    if (e != cudaSuccess) return e;
    scatter_kernel<<<gs_blocks(n), kBlock, 0, s>>>(n, h->new_cell, h->slot, h->cell_start,
                                                   h->orig, h->src, h->key, h->ds, gated);
    const int sort_blocks = std::min((h->g.ncells + kSortBlock / 32 - 1) / (kSortBlock / 32),
                                     kGridCap * 2);
    if (h->p.force_variant == MD_FORCE_PAIRED)
        cell_pair_order_kernel<<<std::max(sort_blocks, 1), kSortBlock, 0, s>>>(
            h->g.ncells, h->grids, h->rep, h->cell_start, h->tmp_abs, h->key, h->src, h->ds,
            gated);
    else
        cell_sort_kernel<<<std::max(sort_blocks, 1), kSortBlock, 0, s>>>(
            h->g.ncells, h->cell_start, h->key, h->src, h->ds, gated);
    gather_kernel<<<gs_blocks(n), kBlock, 0, s>>>(n, h->grids, h->src, h->tmp_abs, h->tmp_v,
                                                  h->xr64[cur], h->xq[cur], h->xq_build, h->xabs,
                                                  h->v, h->orig, h->cell, h->rep, h->type_orig,
                                                  h->ds, gated);
    return cudaGetLastError();
}

cudaError_t launch_export_cells(md_system *h, int32_t *cell_of_atom, int64_t *cell_start) {
    int m = (int)(h->n > h->g.ncells + 1 ? h->n : h->g.ncells + 1);
    export_cells_kernel<<<nblocks(m), kBlock, 0, h->stream>>>(
        (int)h->n, h->g.ncells, h->orig, h->cell, h->cell_start, cell_of_atom, cell_start);
    return cudaGetLastError();
}

}  // namespace mdg
