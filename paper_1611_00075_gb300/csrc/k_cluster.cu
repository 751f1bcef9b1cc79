// k_cluster.cu -- a cluster-pair list for the Lennard-Jones force pass: the
// clustering the paper compares its SIMD scheme with (Sec. 4.1: grouping
// atoms into clusters avoids gathers, which are costly for cheap potentials).
//
// Atoms of each cell (consecutive in the sorted order) form i-clusters of up
// to 8 and j-clusters of up to 4 atoms, balanced within the cell.  The list of
// an i-cluster holds every j-cluster of its 27 stencil cells whose bounding
// box comes within r_list of the i-cluster's box (so every pair within r_list
// is covered, as the half-skin rule requires).  One warp runs one i-cluster:
// lane (a, b) = (lane % 8, lane / 8) pairs i-atom a with j-atom b of the
// current j-cluster, so the four j positions of an entry are loaded once and
// broadcast to the eight lanes of each, and the entry itself is one word the
// warp shares.  Each lane sums its i-atom's force over its j-atoms in float32
// chunks added in float64 (as the per-atom kernel), the four lanes of an
// i-atom are then reduced, and the i-atom's lane of b = 0 finishes the atom.
//
// Entry: stencil cell s in bits 27-31, (j-cluster size - 1) in bits 25-26,
// first sorted atom of the j-cluster in bits 0-24.
#include "k_common.cuh"
#include "k_scan.cuh"

namespace mdg {

namespace {

constexpr int kIC = 8;  // atoms per i-cluster (at most)
constexpr int kJC = 4;  // atoms per j-cluster (at most)

__device__ __forceinline__ bool chain_off(const DevStatus *ds, bool gated) {
    return ds->status != 0 || (gated && ds->rebuild == 0);
}

// clusters per cell: ceil(m / 8) i-clusters, ceil(m / 4) j-clusters
__global__ void cluster_count_kernel(int ncells, const int32_t *__restrict__ start,
                                     int32_t *__restrict__ icnt, int32_t *__restrict__ jcnt,
                                     DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ds->cluster_pairs = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        const int m = start[c + 1] - start[c];
        icnt[c] = (m + kIC - 1) / kIC;
        jcnt[c] = (m + kJC - 1) / kJC;
    }
}

// k-th of K balanced pieces of m atoms: size and offset
__device__ __forceinline__ void piece(int m, int K, int k, int &off, int &size) {
    const int base = m / K, rem = m % K;
    size = base + (k < rem ? 1 : 0);
    off = k * base + min(k, rem);
}

// The cluster tables: icl[I] = first atom | (size - 1) << 27 and its cell;
// jcl boxes (lo, hi) in the cell's own frame (cell-relative float32).
__global__ void cluster_fill_kernel(int ncells, const int32_t *__restrict__ start,
                                    const int32_t *__restrict__ ioff,
                                    const int32_t *__restrict__ joff,
                                    const float4 *__restrict__ xq, uint32_t *__restrict__ icl,
                                    int32_t *__restrict__ icl_cell, float4 *__restrict__ jbox,
                                    int32_t *ntot, const DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ntot[0] = ioff[ncells];
        ntot[1] = joff[ncells];
    }
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += gridDim.x * blockDim.x) {
        const int b = start[c], m = start[c + 1] - b;
        const int ni = ioff[c + 1] - ioff[c], nj = joff[c + 1] - joff[c];
        for (int k = 0; k < ni; ++k) {
            int off, size;
            piece(m, ni, k, off, size);
            icl[ioff[c] + k] = (uint32_t)(b + off) | ((uint32_t)(size - 1) << 27);
            icl_cell[ioff[c] + k] = c;
        }
        for (int k = 0; k < nj; ++k) {
            int off, size;
            piece(m, nj, k, off, size);
            float4 lo = make_float4(3e38f, 3e38f, 3e38f, 0.f);
            float4 hi = make_float4(-3e38f, -3e38f, -3e38f, 0.f);
            for (int t = 0; t < size; ++t) {
                const float4 q = xq[b + off + t];
                lo.x = fminf(lo.x, q.x); lo.y = fminf(lo.y, q.y); lo.z = fminf(lo.z, q.z);
                hi.x = fmaxf(hi.x, q.x); hi.y = fmaxf(hi.y, q.y); hi.z = fmaxf(hi.z, q.z);
            }
            lo.w = __int_as_float(b + off);
            hi.w = __int_as_float(size);
            jbox[2 * (joff[c] + k)] = lo;
            jbox[2 * (joff[c] + k) + 1] = hi;
        }
    }
}

// Warp per i-cluster: the j-clusters of the 27 stencil cells whose boxes come
// within r_list (plus a float32 margin) of the i-cluster's box, in stencil
// order and then ascending atom index.
__global__ void __launch_bounds__(128)
cluster_list_kernel(const Grid g, const int32_t *__restrict__ joff, const uint32_t *__restrict__ icl,
                    const int32_t *__restrict__ icl_cell, const float4 *__restrict__ jbox,
                    const float4 *__restrict__ xq, const int32_t *ntot, float rl2m,
                    uint32_t *__restrict__ clist, int32_t *__restrict__ crow, int capc,
                    DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int nI = ntot[0];
    int overflow = 0;
    unsigned long long tot = 0;
    for (int I = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); I < nI; I += nw) {
        const uint32_t ic = icl[I];
        const int is = (int)(ic & ((1u << 27) - 1)), isz = (int)(ic >> 27) + 1;
        // the i-cluster's box (lanes 0..isz-1 hold its atoms)
        float3 lo = make_float3(3e38f, 3e38f, 3e38f), hi = make_float3(-3e38f, -3e38f, -3e38f);
        if (lane < isz) {
            const float4 q = xq[is + lane];
            lo = make_float3(q.x, q.y, q.z);
            hi = lo;
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo.x = fminf(lo.x, __shfl_xor_sync(0xffffffffu, lo.x, o));
            lo.y = fminf(lo.y, __shfl_xor_sync(0xffffffffu, lo.y, o));
            lo.z = fminf(lo.z, __shfl_xor_sync(0xffffffffu, lo.z, o));
            hi.x = fmaxf(hi.x, __shfl_xor_sync(0xffffffffu, hi.x, o));
            hi.y = fmaxf(hi.y, __shfl_xor_sync(0xffffffffu, hi.y, o));
            hi.z = fmaxf(hi.z, __shfl_xor_sync(0xffffffffu, hi.z, o));
        }
        const int c = icl_cell[I] - g.cell0;
        const int cx = c % g.nx, cy = (c / g.nx) % g.ny, cz = c / (g.nx * g.ny);
        uint32_t *row = clist + (size_t)I * capc;
        int cnt = 0;
        for (int s = 0; s < kStencil; ++s) {
            const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
            int xx = cx + dx, yy = cy + dy, zz = cz + dz;
            xx += (xx < 0) ? g.nx : (xx >= g.nx ? -g.nx : 0);
            yy += (yy < 0) ? g.ny : (yy >= g.ny ? -g.ny : 0);
            zz += (zz < 0) ? g.nz : (zz >= g.nz ? -g.nz : 0);
            const int cn = g.cell0 + (zz * g.ny + yy) * g.nx + xx;
            // the neighbour cell's frame seen from the home cell: + d * w
            const float sx = (float)(dx * g.w[0]), sy = (float)(dy * g.w[1]),
                        sz = (float)(dz * g.w[2]);
            const int j0 = joff[cn], j1 = joff[cn + 1];
            for (int jb = j0; jb < j1; jb += 32) {
                const int J = jb + lane;
                bool acc = false;
                uint32_t ent = 0;
                if (J < j1) {
                    const float4 blo = jbox[2 * J], bhi = jbox[2 * J + 1];
                    const float gx = fmaxf(0.f, fmaxf((blo.x + sx) - hi.x, lo.x - (bhi.x + sx)));
                    const float gy = fmaxf(0.f, fmaxf((blo.y + sy) - hi.y, lo.y - (bhi.y + sy)));
                    const float gz = fmaxf(0.f, fmaxf((blo.z + sz) - hi.z, lo.z - (bhi.z + sz)));
                    acc = gx * gx + gy * gy + gz * gz < rl2m;
                    ent = ((uint32_t)s << 27) | ((uint32_t)(__float_as_int(bhi.w) - 1) << 25) |
                          (uint32_t)__float_as_int(blo.w);
                }
                const unsigned m = __ballot_sync(0xffffffffu, acc);
                const int k = cnt + __popc(m & ((1u << lane) - 1u));
                if (acc && k < capc) row[k] = ent;
                cnt += __popc(m);
            }
        }
        if (lane == 0) crow[I] = min(cnt, capc);
        overflow |= cnt > capc;
        tot += (unsigned long long)cnt;
    }
    if (lane == 0 && tot) atomicAdd(&ds->cluster_pairs, tot);
    if (__any_sync(0xffffffffu, overflow) && lane == 0)
        atomicCAS(&ds->status, 0, (int)MD_ERR_LIST_OVERFLOW);
}

template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(128)
cluster_force_kernel(ForceArgs a, const uint32_t *__restrict__ icl,
                     const uint32_t *__restrict__ clist, const int32_t *__restrict__ crow,
                     const int32_t *ntot, int capc, int store_f) {
    __shared__ ShiftTab sh;
    load_shifts_f32(a.g, &sh);
    __syncthreads();
    if (a.ds->status != 0) return;
    step_bookkeeping<MODE>(a);
    const int lane = threadIdx.x & 31;
    const int ia = lane & (kIC - 1), jb = lane >> 3;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int nI = ntot[0];
    const float rc2 = a.fc.rc2f, sig2 = a.fc.sig2f, e48 = a.fc.eps48f;
    for (int I = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); I < nI; I += nw) {
        const uint32_t ic = icl[I];
        const int is = (int)(ic & ((1u << 27) - 1)), isz = (int)(ic >> 27) + 1;
        const bool ival = ia < isz;
        const int i = is + min(ia, isz - 1);
        const float4 qi = a.xq[i];
        const int len = crow[I];
        const uint32_t *row = clist + (size_t)I * capc;
        double Fx = 0.0, Fy = 0.0, Fz = 0.0, E = 0.0;
        unsigned npair = 0;
        for (int k0 = 0; k0 < len; k0 += 32) {
            const uint32_t mine = (k0 + lane < len) ? __ldcs(row + k0 + lane) : 0u;
            const int kend = min(32, len - k0);
            float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
            for (int t = 0; t < kend; ++t) {
                const uint32_t ent = __shfl_sync(0xffffffffu, mine, t);
                const int st = (int)(ent >> 27);
                const int jsz = (int)((ent >> 25) & 3u) + 1;
                const int j = (int)(ent & ((1u << 25) - 1)) + min(jb, jsz - 1);
                const float4 qj = __ldg(a.xq + j);
                const float ex = (qj.x - qi.x) + sh.x[st];
                const float ey = (qj.y - qi.y) + sh.y[st];
                const float ez = (qj.z - qi.z) + sh.z[st];
                const float r2 = ex * ex + ey * ey + ez * ez;
                if (ival && jb < jsz && j != i && r2 < rc2) {
                    const float r2i = __fdividef(1.0f, r2);
                    float s6 = sig2 * r2i;
                    s6 = s6 * s6 * s6;
                    const float fs = e48 * r2i * s6 * (s6 - 0.5f);
                    fx -= fs * ex;
                    fy -= fs * ey;
                    fz -= fs * ez;
                    if (ENERGY) {
                        e += a.fc.eps4f * s6 * (s6 - 1.0f) - a.fc.shiftf;
                        ++npair;
                    }
                }
            }
            Fx += (double)fx;
            Fy += (double)fy;
            Fz += (double)fz;
            if (ENERGY) E += (double)e;
        }
        // the four lanes of an i-atom (lane, lane + 8, + 16, + 24)
        for (int o = 8; o < 32; o <<= 1) {
            Fx += __shfl_xor_sync(0xffffffffu, Fx, o);
            Fy += __shfl_xor_sync(0xffffffffu, Fy, o);
            Fz += __shfl_xor_sync(0xffffffffu, Fz, o);
            if (ENERGY) E += __shfl_xor_sync(0xffffffffu, E, o);
        }
        if (ENERGY) {
            npair = __reduce_add_sync(0xffffffffu, npair);
            if (lane == 0 && npair) atomicAdd(&a.ds->pairs_cut, (unsigned long long)npair);
        }
        if (jb == 0 && ival) {
            const size_t n = (size_t)a.n;
            if (MODE == FM_STORE || store_f) {
                a.f[i] = Fx;
                a.f[n + i] = Fy;
                a.f[2 * n + i] = Fz;
            }
            if (ENERGY) a.e_atom[i] = 0.5 * E;
            if (MODE != FM_STORE) vv_epilogue<MODE>(a, i, Fx, Fy, Fz, qi.w);
        }
    }
}

}  // namespace

int cluster_cap(int max_cell) { return kStencil * ((max_cell + kJC - 1) / kJC); }
int64_t cluster_rows(int64_t n, int ncells) { return n / kIC + ncells + 1; }

cudaError_t launch_cluster_build(md_system *h, bool gated) {
    const int nc = h->g.ncells;
    cudaStream_t s = h->stream;
    cluster_count_kernel<<<gs_blocks(nc), kBlock, 0, s>>>(nc, h->cell_start, h->cl_icnt,
                                                          h->cl_jcnt, h->ds, gated);
    cudaError_t e = launch_scan<int32_t>(h->cl_icnt, h->cl_ioff, nc, h->cl_bsum, h->ds, gated, s);
    if (e == cudaSuccess) e = launch_scan<int32_t>(h->cl_jcnt, h->cl_joff, nc, h->cl_bsum, h->ds, gated, s);
    if (e != cudaSuccess) return e;
    cluster_fill_kernel<<<gs_blocks(nc), kBlock, 0, s>>>(nc, h->cell_start, h->cl_ioff, h->cl_joff,
                                                         h->xq[h->cur], h->cl_icl, h->cl_icell,
                                                         h->cl_jbox, h->cl_ntot, h->ds, gated);
    // r_list plus a float32 margin: a box test that rounds the other way only
    // adds a cluster pair (the force pass tests r_c itself)
    const float rl = (float)h->r_list * (1.0f + 1.0f / 4096.0f);
    cluster_list_kernel<<<152 * 16, 128, 0, s>>>(h->g, h->cl_joff, h->cl_icl, h->cl_icell,
                                                 h->cl_jbox, h->xq[h->cur], h->cl_ntot, rl * rl,
                                                 h->cl_list, h->cl_row, h->cl_cap, h->ds, gated);
    return cudaGetLastError();
}

cudaError_t launch_cluster_forces(md_system *h, int mode, bool energy, bool store_f) {
    ForceArgs a = make_force_args(h);
    const int sf = store_f ? 1 : 0;
    cudaStream_t s = h->stream;
    const int nb = 152 * 16;
#define MDG_CL(M, E)                                                                          \
    cluster_force_kernel<M, E><<<nb, 128, 0, s>>>(a, h->cl_icl, h->cl_list, h->cl_row,        \
                                                  h->cl_ntot, h->cl_cap, sf)
    switch (mode) {
        case FM_STORE: if (energy) MDG_CL(FM_STORE, true); else MDG_CL(FM_STORE, false); break;
        case FM_FUSED_FULL: MDG_CL(FM_FUSED_FULL, false); break;
        default: MDG_CL(FM_FUSED_HALF, false); break;
    }
#undef MDG_CL
    return cudaGetLastError();
}

}  // namespace mdg
