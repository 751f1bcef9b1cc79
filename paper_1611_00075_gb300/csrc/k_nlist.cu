// k_nlist.cu -- Verlet neighbour lists with skin (Sec. 2.1: lists are built
// per cell from the 27 surrounding cells; Sec. 3.3: list radius
// r_list = r_c + skin, rebuilt on the half-skin displacement rule).
//
// One thread per sorted atom scans the 27 cells around its cell.  The lanes
// of a warp hold consecutive sorted atoms, so they walk the same cells and
// their candidate loads coalesce in L1.  The acceptance test r^2 < r_list^2
// is decided exactly as the float64 definition (minimum-image components,
// dx*dx + dy*dy + dz*dz left to right, no fused multiply-add), but the
// float64 arithmetic only runs for candidates whose float32 distance lies in
// a thin band around r_list^2; outside the band the float32 result cannot
// decide differently (its error bound is far below the band's half width).
//
// List layout: see list_idx() -- per warp group of 32 atoms, quads of four
// entries per atom, written here with one 16-byte store per quad.  An entry is
// (stencil cell s << 27) | sorted index j; s selects the cell shift
// (dx, dy, dz) * w that turns cell-relative coordinates into the pair vector.
#include "md_internal.cuh"

namespace mdg {

namespace {

__device__ __forceinline__ bool chain_off(const DevStatus *ds, bool gated) {
    return ds->status != 0 || (gated && ds->rebuild == 0);
}

// r^2 < r_list^2 by the float64 definition, operation for operation.
__device__ __forceinline__ bool exact_within(const double4 &ai, const double4 &aj, double shx,
                                             double shy, double shz, double rl2) {
    const double ddx = __dadd_rn(__dadd_rn(aj.x, -ai.x), shx);
    const double ddy = __dadd_rn(__dadd_rn(aj.y, -ai.y), shy);
    const double ddz = __dadd_rn(__dadd_rn(aj.z, -ai.z), shz);
    double r2 = __dmul_rn(ddx, ddx);
    r2 = __dadd_rn(r2, __dmul_rn(ddy, ddy));
    r2 = __dadd_rn(r2, __dmul_rn(ddz, ddz));
    return r2 < rl2;
}

// The same test for the rare candidates of the float32 band, kept out of line
// so that the compiler cannot turn it into predicated code that every
// candidate of the hot loop would issue.
__device__ __noinline__ bool exact_within_band(const double4 *__restrict__ xabs, int i, int j,
                                               double shx, double shy, double shz, double rl2) {
    return exact_within(xabs[i], xabs[j], shx, shy, shz, rl2);
}

// Float64 periodic shift of stencil cell s (dx, dy, dz in {-1, 0, 1}) seen
// from cell (cx, cy, cz): +-L where the neighbour wraps, else 0.
__device__ __forceinline__ void stencil_shift64(const Grid &g, int cx, int cy, int cz, int s,
                                                double &shx, double &shy, double &shz) {
    const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
    const int xx = cx + dx, yy = cy + dy, zz = cz + dz;
    shx = xx < 0 ? -g.L[0] : (xx >= g.nx ? g.L[0] : 0.0);
    shy = yy < 0 ? -g.L[1] : (yy >= g.ny ? g.L[1] : 0.0);
    shz = zz < 0 ? -g.L[2] : (zz >= g.nz ? g.L[2] : 0.0);
}

// How the acceptance r^2 < r_list^2 is decided for one atom's candidates.
enum ListMode {
    LM_EXACT = 0,  // float64 definition for every candidate (float64 path)
    LM_BAND = 1,   // float32 prefilter; band candidates tested in float64 at once
    LM_DEFER = 2,  // float32 prefilter; band candidates accepted, verified after
};

struct BandNote {
    int count;    // band candidates met
    int k, j, s;  // the last one: its slot in the row; its index and stencil cell
                  // (kept only when the row is not written: a written row holds them)
};

// Offset of entry k in a row of the quad layout: (k / 4) * 128 + k % 4.
__device__ __forceinline__ int row_off(int k) { return k + (k >> 2) * 124; }

// The list of sorted atom i: scans the 27 cells around its cell and writes
// its row (entries in stencil order, then ascending index).  Returns the
// entry count; in LM_DEFER the band candidates are counted in `band`.
template <int LM, bool WRITE, bool HALF>
__device__ __forceinline__ int list_atom(int i, const Grid &g, float lo, float hi, double rl2,
                                         const float4 *__restrict__ xq,
                                         const double4 *__restrict__ xabs, int c,
                                         const int32_t *__restrict__ start, uint32_t *row,
                                         int cap, BandNote &band) {
    int cnt = 0;
    // float32 cell widths: stencil shift (dx, dy, dz) * w, exact for dx in {-1, 0, 1}
    const float wx = (float)g.w[0], wy = (float)g.w[1], wz = (float)g.w[2];
    const int cx = c % g.nx, cy = (c / g.nx) % g.ny, cz = c / (g.nx * g.ny);
    const float4 qi = xq[i];
    const int myo = __float_as_int(qi.w);
    const double4 ai = (LM == LM_EXACT) ? xabs[i] : make_double4(0.0, 0.0, 0.0, 0.0);
    for (int dz = -1; dz <= 1; ++dz) {
        int zz = cz + dz;
        double shz = 0.0;
        if (zz < 0) { zz += g.nz; shz = -g.L[2]; }
        else if (zz >= g.nz) { zz -= g.nz; shz = g.L[2]; }
        for (int dy = -1; dy <= 1; ++dy) {
            int yy = cy + dy;
            double shy = 0.0;
            if (yy < 0) { yy += g.ny; shy = -g.L[1]; }
            else if (yy >= g.ny) { yy -= g.ny; shy = g.L[1]; }
            for (int dx = -1; dx <= 1; ++dx) {
                int xx = cx + dx;
                double shx = 0.0;
                if (xx < 0) { xx += g.nx; shx = -g.L[0]; }
                else if (xx >= g.nx) { xx -= g.nx; shx = g.L[0]; }
                const int cn = g.cell0 + (zz * g.ny + yy) * g.nx + xx;
                const int s = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                const uint32_t sbits = (uint32_t)s << kIndexBits;
                // home position moved against the cell shift: e = q_j - (q_i - shift)
                const float hx = qi.x - (float)dx * wx, hy = qi.y - (float)dy * wy,
                            hz = qi.z - (float)dz * wz;
                const int b = start[cn], e = start[cn + 1];
                const int skip = (s == 13) ? i : -1;  // the atom itself, home cell only
                if (LM == LM_DEFER) {
                    // branch-free acceptance: a predicated store, a counted
                    // slot; a band candidate only notes its slot (the row
                    // holds its index and stencil cell)
#pragma unroll 4
                    for (int j = b; j < e; ++j) {
                        const float4 qj = xq[j];
                        const float ex = qj.x - hx, ey = qj.y - hy, ez = qj.z - hz;
                        const float r2f = ex * ex + ey * ey + ez * ez;
                        bool acc = (r2f < hi) & (j != skip);
                        if (HALF) acc = acc & (__float_as_int(qj.w) > myo);
                        if (WRITE) {
                            if (acc & (cnt < cap)) row[row_off(cnt)] = sbits | (uint32_t)j;
                        } else {
                            const bool bq = acc & (r2f >= lo);
                            band.j = bq ? j : band.j;
                            band.s = bq ? s : band.s;
                        }
                        const bool bnd = acc & (r2f >= lo);
                        band.k = bnd ? cnt : band.k;
                        band.count += bnd ? 1 : 0;
                        cnt += acc ? 1 : 0;
                    }
                } else {
#pragma unroll 4
                    for (int j = b; j < e; ++j) {
                        const float4 qj = xq[j];
                        float r2f = 0.f;
                        bool cand = true;
                        if (LM == LM_BAND) {
                            const float ex = qj.x - hx, ey = qj.y - hy, ez = qj.z - hz;
                            r2f = ex * ex + ey * ey + ez * ez;
                            cand = r2f < hi;
                        }
                        cand = cand && (j != skip);
                        if (HALF) cand = cand && (__float_as_int(qj.w) > myo);
                        if (!cand) continue;
                        bool acc = true;
                        if (LM == LM_EXACT) acc = exact_within(ai, xabs[j], shx, shy, shz, rl2);
                        else if (r2f >= lo) acc = exact_within_band(xabs, i, j, shx, shy, shz, rl2);
                        if (!acc) continue;
                        if (WRITE && cnt < cap)
                            row[(size_t)(((cnt >> 2) << 7) | (cnt & 3))] = sbits | (uint32_t)j;
                        ++cnt;
                    }
                }
            }
        }
    }
    return cnt;
}

// A second band candidate in one atom is rare enough (about 1 in 10^5 atoms
// at rho* = 0.8442) to redo that atom with the band tested in place.
template <bool WRITE, bool HALF>
__device__ __noinline__ int list_atom_band(int i, const Grid &g, float lo, float hi, double rl2,
                                           const float4 *__restrict__ xq,
                                           const double4 *__restrict__ xabs, int c,
                                           const int32_t *__restrict__ start, uint32_t *row,
                                           int cap) {
    BandNote unused{0, 0, 0, 0};
    return list_atom<LM_BAND, WRITE, HALF>(i, g, lo, hi, rl2, xq, xabs, c, start, row, cap,
                                           unused);
}

// 128-thread blocks measured 1 % faster than 256 for this kernel.
constexpr int kListBlock = 128;

template <bool PREFILTER, bool WRITE, bool HALF>
__global__ void __launch_bounds__(kListBlock)
build_list_kernel(int n, const Grid *__restrict__ grids, const uint16_t *__restrict__ rep,
                  float lo, float hi, double rl2, const float4 *__restrict__ xq,
                  const double4 *__restrict__ xabs, const int32_t *__restrict__ cell,
                  const int32_t *__restrict__ start, uint32_t *__restrict__ nlist,
                  int32_t *__restrict__ ncount, int cap, DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    unsigned long long tot = 0;
    int overflow = 0, maxc = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Grid &g = grids[rep ? rep[i] : 0];
        const int c = cell[i] - g.cell0;
        // entry k of atom i: row[(k / 4) * 128 + k % 4]
        uint32_t *row = nlist + list_group(i, cap) + ((i & 31) << 2);
        BandNote band{0, 0, 0, 0};
        int cnt;
        if (!PREFILTER) {
            cnt = list_atom<LM_EXACT, WRITE, HALF>(i, g, lo, hi, rl2, xq, xabs, c, start, row, cap,
                                                   band);
        } else {
            cnt = list_atom<LM_DEFER, WRITE, HALF>(i, g, lo, hi, rl2, xq, xabs, c, start, row, cap,
                                                   band);
            if (band.count == 1 && WRITE && band.k >= cap) {
                overflow = 1;  // the entry was not stored: the row is regrown anyway
            } else if (band.count == 1) {
                // verify the one provisional entry; drop it if the float64
                // definition rejects it
                if (WRITE) {
                    const uint32_t ent = row[row_off(band.k)];
                    band.j = (int)(ent & kIndexMask);
                    band.s = (int)(ent >> kIndexBits);
                }
                const int cx = c % g.nx, cy = (c / g.nx) % g.ny, cz = c / (g.nx * g.ny);
                double shx, shy, shz;
                stencil_shift64(g, cx, cy, cz, band.s, shx, shy, shz);
                if (!exact_within_band(xabs, i, band.j, shx, shy, shz, rl2)) {
                    overflow |= (cnt > cap);  // a full row lost its tail: regrow
                    if (WRITE)
                        for (int k = band.k; k + 1 < min(cnt, cap); ++k)
                            row[row_off(k)] = row[row_off(k + 1)];
                    --cnt;
                }
            } else if (band.count > 1) {
                cnt = list_atom_band<WRITE, HALF>(i, g, lo, hi, rl2, xq, xabs, c, start, row, cap);
            }
        }
        if (WRITE && cnt <= cap) {
            // pad the last quad with self-entries that no cutoff accepts
            const uint32_t pad = (kPadStencil << kIndexBits) | (uint32_t)i;
            for (int k = cnt; k & 3; ++k) row[(size_t)(k >> 2) * 128 + (k & 3)] = pad;
        }
        ncount[i] = cnt;
        maxc = max(maxc, cnt);
        tot += (unsigned long long)cnt;
        overflow |= (cnt > cap);
    }
    // every lane of the block reaches this point (grid-stride loop, no early
    // exit); one atomic per warp instead of one per atom on the same address
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xffffffffu, tot, o);
    maxc = __reduce_max_sync(0xffffffffu, (unsigned)maxc);
    if ((threadIdx.x & 31) == 0) {
        if (tot) atomicAdd(&ds->list_entries, tot);
        if (maxc) atomicMax(&ds->max_count, maxc);
    }
    if (WRITE && overflow) atomicCAS(&ds->status, 0, (int)MD_ERR_LIST_OVERFLOW);
}

__global__ void reset_max_count_kernel(DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    ds->max_count = 0;
    ds->list_entries = 0;
}

__global__ void finish_rebuild_kernel(DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    ds->rebuild = 0;
    ds->since_build = 0;
    ds->builds += 1;
}

// ---- export (parity and inspection) -----------------------------------------

__global__ void export_rowcount_kernel(int n, int cap, int half, const int32_t *__restrict__ orig,
                                       const int32_t *__restrict__ ncount,
                                       const uint32_t *__restrict__ nlist,
                                       int32_t *__restrict__ rowcnt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int o = orig[i];
    int cnt = min(ncount[i], cap);
    int keep = cnt;
    if (half) {
        keep = 0;
        for (int k = 0; k < cnt; ++k) {
            int j = (int)(nlist[list_idx(i, k, cap)] & kIndexMask);
            keep += (orig[j] > o);
        }
    }
    rowcnt[o] = keep;
}

__global__ void export_fill_kernel(int n, int cap, int half, const int32_t *__restrict__ orig,
                                   const int32_t *__restrict__ ncount,
                                   const uint32_t *__restrict__ nlist,
                                   const int32_t *__restrict__ rowstart, int64_t *offsets,
                                   int32_t *__restrict__ ids) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int o = orig[i];
    int cnt = min(ncount[i], cap);
    int64_t p0 = rowstart[o];
    int64_t p = p0;
    for (int k = 0; k < cnt; ++k) {
        int j = (int)(nlist[list_idx(i, k, cap)] & kIndexMask);
        int oj = orig[j];
        if (!half || oj > o) ids[p++] = oj;
    }
    for (int64_t a = p0 + 1; a < p; ++a) {  // ascending original id
        int kv = ids[a];
        int64_t q = a - 1;
        while (q >= p0 && ids[q] > kv) {
            ids[q + 1] = ids[q];
            --q;
        }
        ids[q + 1] = kv;
    }
    offsets[o] = p0;
    if (o == n - 1) offsets[n] = rowstart[n];
}

}  // namespace

cudaError_t launch_build_list(md_system *h, bool write, bool gated, const float4 *positions) {
    int n = (int)h->n;
    cudaStream_t s = h->stream;
    const float4 *xq = positions ? positions : h->xq[h->cur];
    const bool prefilter = (h->p.precision == MD_MIXED);
    const bool half = half_variant(h->p.force_variant);
    reset_max_count_kernel<<<1, 1, 0, s>>>(h->ds, gated);
#define MDG_LIST(PF, WR, HF)                                                                    \
    build_list_kernel<PF, WR, HF><<<gs_blocks(n) * (kBlock / kListBlock), kListBlock, 0, s>>>(                                \
        n, h->grids, h->rep, h->list_lo, h->list_hi, h->rl2, xq, h->xabs, h->cell,           \
        h->cell_start,                                                                         \
        h->nlist, h->ncount, h->cap, h->ds, gated)
    if (prefilter) {
        if (write) { if (half) MDG_LIST(true, true, true); else MDG_LIST(true, true, false); }
        else { if (half) MDG_LIST(true, false, true); else MDG_LIST(true, false, false); }
    } else {
        if (write) { if (half) MDG_LIST(false, true, true); else MDG_LIST(false, true, false); }
        else { if (half) MDG_LIST(false, false, true); else MDG_LIST(false, false, false); }
    }
#undef MDG_LIST
    return cudaGetLastError();
}

cudaError_t launch_finish_rebuild(md_system *h, bool gated) {
    finish_rebuild_kernel<<<1, 1, 0, h->stream>>>(h->ds, gated);
    return cudaGetLastError();
}

cudaError_t launch_export_list(md_system *h, int half, int64_t *offsets, int32_t *ids,
                               int64_t *tmp) {
    // tmp: scratch of at least 2 * (n + 1) + 64 int32 words, provided by the caller
    int n = (int)h->n;
    int32_t *rowcnt = reinterpret_cast<int32_t *>(tmp);
    int32_t *rowstart = rowcnt + (n + 1);
    export_rowcount_kernel<<<nblocks(n), kBlock, 0, h->stream>>>(n, h->cap, half, h->orig,
                                                                  h->ncount, h->nlist, rowcnt);
    cudaError_t e = launch_scan_i32(rowcnt, rowstart, n, h->scan_bsum, h->ds, false, h->stream);
    if (e != cudaSuccess) return e;
    if (ids != nullptr)
        export_fill_kernel<<<nblocks(n), kBlock, 0, h->stream>>>(n, h->cap, half, h->orig,
                                                                  h->ncount, h->nlist, rowstart,
                                                                  offsets, ids);
    return cudaGetLastError();
}

}  // namespace mdg
