// k_pair.cu -- two home atoms per thread (MD_FORCE_PAIRED).
//
// Sec. 4.1 contrasts the paper's per-atom SIMD pair loop with clustering:
// grouping atoms lets one neighbour load serve several pair evaluations,
// which avoids the gather cost that dominates light potentials.  Full 8 x 4
// cluster pairs waste most of their slots at r_c = 2.5 sigma (their bounding
// boxes are as large as the cut-off sphere); this layout clusters only the
// home side, and only by two: the atoms of each cell, in their sorted order,
// are taken two at a time into slots (a cell of odd occupancy ends with a
// one-atom slot).  A slot's list is the union of its two atoms' lists, so one
// gather of a neighbour position feeds two pair evaluations: the union of two
// r_list spheres about one atom spacing apart holds about 1.3 times the
// entries of one, for twice the pairs.
//
// Slot s holds sorted atoms i0 = slot_atom[s] & 0x7fffffff and, unless bit 31
// is set, i1 = i0 + 1 (the same cell).  Its list uses the per-atom layout
// (groups of 32 slots, quads of entries; entry = (stencil << 27) | j, j never
// i0 or i1) and is padded to whole quads with entries that point at a far
// away dummy position stored after the last atom (index n).  The list is a
// superset of both atoms' lists: it accepts j when the float32 distance to
// either atom is below r_list^2 (1 + 2^-14), which covers every pair within
// r_list -- and so, by the half-skin rule, every pair within r_c until the
// next rebuild.  The force pass evaluates the slot's own pair once
// (f_i0 += F, f_i1 -= F), then both atoms against each list entry in
// float32 -- packed: one f32x2 instruction serves the two atoms -- with the
// per-atom kernel's velocity-Verlet epilogue.  Each atom's
// force is summed in float32 over the whole list (about 55 entries per atom
// at rho* = 0.8442, so one chunk of the per-atom kernel's float32-then-
// float64 sums) and converted once: without the float64 accumulators the
// kernel fits 9 CTAs of 128 threads per SM.
#include "k_pair.cuh"
#include "k_scan.cuh"

namespace mdg {

namespace {

constexpr uint32_t kHomeStencil = 13;       // stencil cell (0, 0, 0)
constexpr int kPairBlock = 128;

__device__ __forceinline__ bool chain_off(const DevStatus *ds, bool gated) {
    return ds->status != 0 || (gated && ds->rebuild == 0);
}

__device__ __forceinline__ int row_off(int k) { return k + (k >> 2) * 124; }

// slots per cell: ceil(atoms / 2)
__global__ void slot_count_kernel(int ncells, const int32_t *__restrict__ start,
                                  int32_t *__restrict__ cnt, const DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x)
        cnt[c] = (start[c + 1] - start[c] + 1) >> 1;
}

// the first atom of every slot, flagged when the slot holds one atom
__global__ void slot_fill_kernel(int n, const int32_t *__restrict__ cell,
                                 const int32_t *__restrict__ start,
                                 const int32_t *__restrict__ slot_start,
                                 uint32_t *__restrict__ slot_atom, const DevStatus *ds,
                                 bool gated) {
    if (chain_off(ds, gated)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c = cell[i];
        const int k = i - start[c];
        if (k & 1) continue;
        const uint32_t single = (i + 1 >= start[c + 1]) ? kSingle : 0u;
        slot_atom[slot_start[c] + (k >> 1)] = (uint32_t)i | single;
    }
}

// One stencil cell of a slot's union-list scan (HOME: the slot's own cell,
// the only one holding i0 and i1); returns the running entry count.
template <bool WRITE, bool HOME>
__device__ __forceinline__ int scan_cell(int cnt, int b, int e, const float4 *__restrict__ xq,
                                         float sx, float sy, float sz, float ux, float uy,
                                         float uz, float lim, int i0, int i1, uint32_t *row,
                                         int cap, uint32_t sbits) {
#pragma unroll 4
    for (int j = b; j < e; ++j) {
        const float4 qj = xq[j];
        const float ex = qj.x - sx, ey = qj.y - sy, ez = qj.z - sz;
        const float r2 = ex * ex + ey * ey + ez * ez;
        const float p = ex * ux + ey * uy + ez * uz;
        bool acc = fmaf(-2.0f, fabsf(p), r2) < lim;
        if (HOME) acc = acc & (j != i0) & (j != i1);
        // past the capacity the row's last entry is overwritten: the
        // overflow status discards the list
        if (WRITE && acc) row[row_off(min(cnt, cap - 1))] = sbits | (uint32_t)j;
        cnt += acc ? 1 : 0;
    }
    return cnt;
}

// The union list of each slot: the 27 cells around the slot's cell, in
// stencil order.  A candidate j is tested against both atoms at once from
// the slot's midpoint m = (x0 + x1) / 2 and half separation u = (x1 - x0) / 2:
// with e = x_j - m, the nearer atom's squared distance is
// |e|^2 + |u|^2 - 2 |e.u|, so the test is |e|^2 - 2 |e.u| < hi - |u|^2 (one
// difference vector and two dot products instead of two distances).  In
// float32 the terms stay below about 16 sigma^2, so the rounding error of
// this form is about 1e-5 sigma^2 at most, against the 2^-14 r_list^2
// (5e-4 sigma^2) margin of hi: the list stays a superset of both atoms'
// r_list spheres.
// Only the home cell holds i0 and i1, so only its scan excludes them.
//
// Measured on GB300 (porous LJ, 9.8 M atoms, 300 steps from the generated
// state, one build of the union lists): 3.68 ms against 4.19 ms for two
// direct distances per candidate.  Seven CTAs per SM (71 registers) against
// 3.93 ms at eight and 4.16 ms at nine; the candidate loop unrolled by 4
// against 4.13 ms by 2 and 4.30 ms by 8 (at eight CTAs).  Packed f32x2
// distances for the two atoms were slower (4.98 against 4.45 ms).
// MULTI (a batch of boxes): each slot takes the geometry of its atoms' box
// (cells numbered box after box from the box's cell0).
template <bool WRITE, bool MULTI = false>
__global__ void __launch_bounds__(kPairBlock, 7)
pair_list_kernel(int n, Grid g, const Grid *__restrict__ grids, const uint16_t *__restrict__ rep,
                 float hi, const float4 *__restrict__ xq,
                 const int32_t *__restrict__ cell, const int32_t *__restrict__ start,
                 const int32_t *__restrict__ slot_start, const uint32_t *__restrict__ slot_atom,
                 uint32_t *__restrict__ list, int32_t *__restrict__ count, int cap, DevStatus *ds,
                 bool gated) {
    if (chain_off(ds, gated)) return;
    const int nslots = slot_start[g.ncells];
    if (blockIdx.x == 0 && threadIdx.x == 0) ds->pair_slots = nslots;
    unsigned long long tot = 0;
    int overflow = 0, maxc = 0;
    const uint32_t pad = (kHomeStencil << kIndexBits) | (uint32_t)n;
    // grid-stride over whole warps, so every lane reaches the reductions below
    const int stride = gridDim.x * blockDim.x;
    const int send = ((nslots + 31) & ~31);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < send; s += stride) {
        if (s < nslots) {
            const uint32_t sa = slot_atom[s];
            const int i0 = (int)(sa & ~kSingle);
            const int i1 = (sa & kSingle) ? i0 : i0 + 1;
            const float4 q0 = xq[i0], q1 = xq[i1];
            const float ux = 0.5f * (q1.x - q0.x), uy = 0.5f * (q1.y - q0.y),
                        uz = 0.5f * (q1.z - q0.z);
            const float mx = q0.x + ux, my = q0.y + uy, mz = q0.z + uz;
            const float lim = hi - (ux * ux + uy * uy + uz * uz);
            int nx = g.nx, ny = g.ny, nz = g.nz, c0 = 0;
            float wx = g.wf[0], wy = g.wf[1], wz = g.wf[2];
            if (MULTI) {
                const Grid &gb = grids[rep[i0]];
                nx = gb.nx; ny = gb.ny; nz = gb.nz; c0 = gb.cell0;
                wx = gb.wf[0]; wy = gb.wf[1]; wz = gb.wf[2];
            }
            const int c = cell[i0] - c0;
            const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
            uint32_t *row = list + list_group(s, cap) + ((s & 31) << 2);
            int cnt = 0;
            for (int dz = -1; dz <= 1; ++dz) {
                const int zz = (cz + dz + nz) % nz;
                for (int dy = -1; dy <= 1; ++dy) {
                    const int yy = (cy + dy + ny) % ny;
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int xx = (cx + dx + nx) % nx;
                        const int cn = c0 + (zz * ny + yy) * nx + xx;
                        const uint32_t st = (uint32_t)((dz + 1) * 9 + (dy + 1) * 3 + (dx + 1));
                        // the midpoint moved against the cell shift
                        const float sx = mx - (float)dx * wx, sy = my - (float)dy * wy,
                                    sz = mz - (float)dz * wz;
                        const int b = start[cn], e = start[cn + 1];
                        const uint32_t sbits = st << kIndexBits;
                        if (st == kHomeStencil)
                            cnt = scan_cell<WRITE, true>(cnt, b, e, xq, sx, sy, sz, ux, uy, uz,
                                                         lim, i0, i1, row, cap, sbits);
                        else
                            cnt = scan_cell<WRITE, false>(cnt, b, e, xq, sx, sy, sz, ux, uy, uz,
                                                          lim, i0, i1, row, cap, sbits);
                    }
                }
            }
            if (WRITE && cnt <= cap)
                for (int k = cnt; k & 3; ++k) row[row_off(k)] = pad;
            if (WRITE) count[s] = cnt;
            maxc = max(maxc, cnt);
            tot += (unsigned long long)cnt;
            overflow |= (cnt > cap);
        }
    }
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
    maxc = (int)__reduce_max_sync(0xffffffffu, (unsigned)maxc);
    if ((threadIdx.x & 31) == 0) {
        if (tot) atomicAdd(&ds->pair_entries, tot);
        if (maxc) atomicMax(&ds->pair_max, maxc);
    }
    if (WRITE && overflow) atomicCAS(&ds->status, 0, (int)MD_ERR_LIST_OVERFLOW);
}

__global__ void pair_reset_kernel(DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    ds->pair_max = 0;
    ds->pair_entries = 0;
}

// the dummy neighbour of the padding entries, past the last atom of both
// position buffers and of the many-body passes' (x, F') records
__global__ void pair_dummy_kernel(float4 *xq0, float4 *xq1, float4 *xqf, int n) {
    const float4 far = make_float4(3.0e18f, 3.0e18f, 3.0e18f, 0.f);
    xq0[n] = far;
    xq1[n] = far;
    if (xqf) xqf[n] = far;
}

// Measured on GB300 (porous LJ, 9.8 M atoms, one force launch): this form
// (packed pairs, float32 sums, 56 registers, 9 CTAs per SM) 1.232 ms against
// 1.304 ms for the per-atom kernel from the generated state, 1.342 against
// 1.440 ms on the equilibrated one; the same arithmetic unpacked 1.387 ms
// (issue-bound: the second atom's pair terms cost as many instructions as
// the first's); with float64 chunk accumulators at 72 registers (7 CTAs)
// 1.498 ms unpacked and 1.551 ms packed (latency-bound).  At 1 M atoms the
// two layouts tie (porous) or the per-atom kernel leads by 2 % (liquid).
//
// MULTI (a batch of boxes): a block's slots are consecutive, so their atoms
// belong to one or two boxes (more only when a box holds fewer slots than a
// block); the shift tables of those boxes go to shared memory like a single
// box's, and a block that spans more boxes reads the global R x 27 table.
template <int MODE, bool ENERGY, bool MULTI = false>
__global__ void __launch_bounds__(kPairBlock, 9) lj_pair_kernel(ForceArgs a, PairArgs p,
                                                                int store_f) {
    __shared__ ShiftTab sh[MULTI ? 2 : 1];
    __shared__ int s_r0, s_span;
    const int nslots = p.slot_start[p.ncells];
    if (!MULTI) {
        load_shifts_f32(a.g, &sh[0]);
    } else {
        const int sb = blockIdx.x * blockDim.x;
        const int se = min(nslots, sb + (int)blockDim.x) - 1;
        const int r0 = sb <= se ? (int)a.rep[p.slot_atom[sb] & ~kSingle] : 0;
        const int r1 = sb <= se ? (int)a.rep[p.slot_atom[se] & ~kSingle] : 0;
        if (threadIdx.x < 2 * kStencil) {
            const int t = threadIdx.x / kStencil, st = threadIdx.x % kStencil;
            if (t <= r1 - r0) {
                const float4 v = a.shifts32[kStencil * (r0 + t) + st];
                sh[t].x[st] = v.x;
                sh[t].y[st] = v.y;
                sh[t].z[st] = v.z;
            }
        }
        if (threadIdx.x == 0) {
            s_r0 = r0;
            s_span = r1 - r0;
        }
    }
    __syncthreads();
    if (a.ds->status != 0) return;
    step_bookkeeping<MODE>(a);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    if (MULTI && s_span <= 1) {
        const int r = (int)a.rep[p.slot_atom[s] & ~kSingle];
        lj_pair_slot<MODE, ENERGY, false>(a, p, &sh[r - s_r0], s, store_f);
    } else {
        lj_pair_slot<MODE, ENERGY, MULTI>(a, p, &sh[0], s, store_f);
    }
}

}  // namespace

int64_t pair_slots_max(int64_t n, int ncells) { return (n + ncells) / 2 + 1; }

cudaError_t launch_pair_dummy(md_system *h) {
    pair_dummy_kernel<<<1, 1, 0, h->stream>>>(h->xq[0], h->xq[1], h->xqf, (int)h->n);
    return cudaGetLastError();
}

cudaError_t launch_pair_build(md_system *h, bool write, bool gated) {
    const int n = (int)h->n, nc = h->g.ncells;
    cudaStream_t s = h->stream;
    slot_count_kernel<<<gs_blocks(nc), kBlock, 0, s>>>(nc, h->cell_start, h->ps_cnt, h->ds, gated);
    cudaError_t e = launch_scan_i32(h->ps_cnt, h->ps_start, nc, h->ps_bsum, h->ds, gated, s);
    if (e != cudaSuccess) return e;
    slot_fill_kernel<<<gs_blocks(n), kBlock, 0, s>>>(n, h->cell, h->cell_start, h->ps_start,
                                                     h->ps_atom, h->ds, gated);
    pair_reset_kernel<<<1, 1, 0, s>>>(h->ds, gated);
    const int64_t smax = pair_slots_max(h->n, nc);
    const int blocks = (int)std::min<int64_t>((smax + kPairBlock - 1) / kPairBlock, 152 * 16);
#define MDG_PAIR_LIST(W, M)                                                                  \
    pair_list_kernel<W, M><<<blocks, kPairBlock, 0, s>>>(                                    \
        n, h->g, h->grids, h->rep, h->list_hi, h->xq[h->cur], h->cell, h->cell_start,        \
        h->ps_start, h->ps_atom, h->ps_list, h->ps_count, h->ps_cap, h->ds, gated)
    if (h->R > 1) {
        if (write) MDG_PAIR_LIST(true, true);
        else MDG_PAIR_LIST(false, true);
    } else {
        if (write) MDG_PAIR_LIST(true, false);
        else MDG_PAIR_LIST(false, false);
    }
#undef MDG_PAIR_LIST
    return cudaGetLastError();
}

// the multi-element variant (k_pair_typed.cu)
cudaError_t launch_pair_typed_forces(md_system *h, int mode, bool energy, bool store_f);

cudaError_t launch_pair_forces(md_system *h, int mode, bool energy, bool store_f) {
    if (h->fc.ntypes > 0) return launch_pair_typed_forces(h, mode, energy, store_f);
    ForceArgs a = make_force_args(h);
    const PairArgs p = make_pair_args(h);
    const int sf = store_f ? 1 : 0;
    const int blocks = pair_grid_blocks(h, kPairBlock);
    const bool multi = h->R > 1;
    cudaStream_t s = h->stream;
#define MDG_PAIR(M)                                                                         \
    do {                                                                                    \
        if (multi) {                                                                        \
            if (energy) lj_pair_kernel<M, true, true><<<blocks, kPairBlock, 0, s>>>(a, p, sf); \
            else lj_pair_kernel<M, false, true><<<blocks, kPairBlock, 0, s>>>(a, p, sf);       \
        } else {                                                                            \
            if (energy) lj_pair_kernel<M, true><<<blocks, kPairBlock, 0, s>>>(a, p, sf);    \
            else lj_pair_kernel<M, false><<<blocks, kPairBlock, 0, s>>>(a, p, sf);          \
        }                                                                                   \
    } while (0)
    switch (mode) {
        case FM_STORE: MDG_PAIR(FM_STORE); break;
        case FM_FUSED_FULL: MDG_PAIR(FM_FUSED_FULL); break;
        default: MDG_PAIR(FM_FUSED_HALF); break;
    }
#undef MDG_PAIR
    return cudaGetLastError();
}

}  // namespace mdg
