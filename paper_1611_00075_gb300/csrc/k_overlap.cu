// k_overlap.cu -- the inner/outer split of Sec. 2.1 on one GPU.
//
// The paper's domain decomposition splits the force calculation into an
// inner part (pairs inside a domain) and an outer part (pairs across a domain
// face), so that particle data can travel while the inner part runs:
//   1 assemble the coordinates of atoms near domain faces in send buffers,
//   2-3 start sending and receiving them,
//   4 compute the intra-domain forces,
//   5 wait for the receives,
//   6 compute the inter-domain forces,
//   7 wait for the sends.
// Here the box's cell grid is cut into px x py x pz virtual domains (blocks
// of cells).  A cell's 27-bit outer mask marks the stencil cells that lie in
// another domain; an atom whose cell has a non-zero mask is a boundary atom.
// Step 1 packs the boundary atoms' float32 positions into one continuous send
// buffer (the paper collapses its per-neighbour buffers into one, too); on
// one GPU the exchange of steps 2-3 is a copy kernel from that buffer into
// the receive buffer on a second stream, and the outer pass reads every
// foreign neighbour from the receive buffer.  Interior atoms finish their step
// (kick, drift) in the inner pass; boundary atoms keep the inner partial
// force in f and finish in the outer pass.
#include "k_common.cuh"
#include "k_scan.cuh"

namespace mdg {

namespace {

__device__ __forceinline__ bool chain_off(const DevStatus *ds, bool gated) {
    return ds->status != 0 || (gated && ds->rebuild == 0);
}

// boundary flag of every sorted atom
__global__ void boundary_flag_kernel(int n, const int32_t *__restrict__ cell,
                                     const uint32_t *__restrict__ cell_outer,
                                     int32_t *__restrict__ flag, const DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = cell_outer[cell[i]] != 0u ? 1 : 0;
}

// gidx[i]: slot of boundary atom i in the buffers (-1 otherwise); bidx: the
// boundary atoms in sorted order; nb_dev: their count
__global__ void boundary_index_kernel(int n, const int32_t *__restrict__ flag,
                                      const int32_t *__restrict__ pos, int32_t *__restrict__ gidx,
                                      int32_t *__restrict__ bidx, int32_t *nb_dev,
                                      const DevStatus *ds, bool gated) {
    if (chain_off(ds, gated)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) *nb_dev = pos[n];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (flag[i]) {
            gidx[i] = pos[i];
            bidx[pos[i]] = i;
        } else {
            gidx[i] = -1;
        }
    }
}

// Steps 2-3 on one GPU: the send buffer's first nb entries into the receive
// buffer (run on the second stream; on several GPUs this is the transfer).
__global__ void exchange_kernel(const int32_t *nb_dev, const float4 *__restrict__ send,
                                float4 *__restrict__ recv) {
    const int nb = *nb_dev;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x)
        recv[k] = send[k];
}

// Step 1: the boundary atoms' positions into the send buffer.
__global__ void assemble_kernel(const int32_t *nb_dev, const int32_t *__restrict__ bidx,
                                const float4 *__restrict__ xq, float4 *__restrict__ send,
                                const DevStatus *ds) {
    if (ds->status != 0) return;
    const int nb = *nb_dev;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x)
        send[k] = xq[bidx[k]];
}

struct OverlapArgs {
    const int32_t *cell;  // sorted slot -> global cell
    const uint32_t *cell_outer;
    const int32_t *gidx, *bidx, *nb_dev;
    const float4 *recv;
};

// The pair loop of one atom over the entries whose stencil cell's outer
// mask bit equals OUTER; neighbours come from xq in the inner pass and from
// the receive buffer (slot gidx[j]) in the outer pass.  Float32 pair terms summed per chunk into float64, as lj_mixed_atom.
template <bool OUTER, bool ENERGY>
__device__ __forceinline__ void split_pair_loop(const ForceArgs &a, const OverlapArgs &o,
                                                const ShiftTab *sh, int i, uint32_t omask,
                                                double &Fx, double &Fy, double &Fz, double &E,
                                                unsigned &npair) {
    const float4 qi = a.xq[i];
    const int nq = (min(a.ncount[i], a.cap) + 3) >> 2;
    const uint4 *lq = reinterpret_cast<const uint4 *>(a.nlist + list_group(i, a.cap)) + (i & 31);
    const float rc2 = a.fc.rc2f, sig2 = a.fc.sig2f, e48 = a.fc.eps48f;
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
    auto pair = [&](uint32_t ent) {
        const uint32_t st = ent >> kIndexBits;
        const bool mine = (((omask >> st) & 1u) != 0u) == OUTER;
        const int j = (int)(ent & kIndexMask);
        // foreign neighbours of the outer pass come from the receive buffer
        // (gidx of a foreign neighbour is >= 0: its cell faces ours across the
        // domain face, so it is a boundary atom too; the clamp keeps every
        // address in bounds regardless)
        const float4 qj =
            OUTER ? (mine ? __ldg(o.recv + max(o.gidx[j], 0)) : qi) : __ldg(a.xq + j);
        const float ex = (qj.x - qi.x) + sh->x[st];
        const float ey = (qj.y - qi.y) + sh->y[st];
        const float ez = (qj.z - qi.z) + sh->z[st];
        const float r2 = ex * ex + ey * ey + ez * ez;
        if (mine && r2 < rc2) {
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
    };
    uint4 nxt = nq > 0 ? __ldcs(lq) : make_uint4(0u, 0u, 0u, 0u);
    for (int q0 = 0; q0 < nq; q0 += kChunkQ) {
        const int q1 = min(q0 + kChunkQ, nq);
        for (int q = q0; q < q1; ++q) {
            const uint4 e4 = nxt;
            if (q + 1 < nq) nxt = __ldcs(lq + (size_t)(q + 1) * 32);
            pair(e4.x);
            pair(e4.y);
            pair(e4.z);
            pair(e4.w);
        }
        Fx += (double)fx;
        Fy += (double)fy;
        Fz += (double)fz;
        fx = fy = fz = 0.f;
        if (ENERGY) {
            E += (double)e;
            e = 0.f;
        }
    }
}

// Step 4: intra-domain forces of every atom.  Interior atoms finish here;
// boundary atoms leave their partial force (and energy) in f (and e_atom).
template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(128, 5) inner_force_kernel(ForceArgs a, OverlapArgs o,
                                                             int store_f) {
    __shared__ ShiftTab sh;
    load_shifts_f32(a.g, &sh);
    __syncthreads();
    if (a.ds->status != 0) return;
    step_bookkeeping<MODE>(a);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    // the outer mask of the atom's cell (cell[] holds global cell ids)
    const uint32_t omask = o.cell_outer[o.cell[i]];
    double Fx = 0.0, Fy = 0.0, Fz = 0.0, E = 0.0;
    unsigned npair = 0;
    split_pair_loop<false, ENERGY>(a, o, &sh, i, omask, Fx, Fy, Fz, E, npair);
    const size_t n = (size_t)a.n;
    if (ENERGY) {
        a.e_atom[i] = 0.5 * E;
        count_pairs(a.ds, npair);
    }
    if (omask != 0u || MODE == FM_STORE || store_f) {
        a.f[i] = Fx;
        a.f[n + i] = Fy;
        a.f[2 * n + i] = Fz;
    }
    if (omask == 0u && MODE != FM_STORE) vv_epilogue<MODE>(a, i, Fx, Fy, Fz, a.xq[i].w);
}

// Step 6: inter-domain forces of the boundary atoms, their neighbours read
// from the receive buffer; adds the inner partial force and finishes the atom.
template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(128, 5) outer_force_kernel(ForceArgs a, OverlapArgs o,
                                                             int store_f) {
    __shared__ ShiftTab sh;
    load_shifts_f32(a.g, &sh);
    __syncthreads();
    if (a.ds->status != 0) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *o.nb_dev) return;
    const int i = o.bidx[k];
    const uint32_t omask = o.cell_outer[o.cell[i]];
    const size_t n = (size_t)a.n;
    double Fx = a.f[i], Fy = a.f[n + i], Fz = a.f[2 * n + i], E = 0.0;
    unsigned npair = 0;
    split_pair_loop<true, ENERGY>(a, o, &sh, i, omask, Fx, Fy, Fz, E, npair);
    if (ENERGY) {
        a.e_atom[i] += 0.5 * E;
        count_pairs(a.ds, npair);
    }
    if (MODE == FM_STORE || store_f) {
        a.f[i] = Fx;
        a.f[n + i] = Fy;
        a.f[2 * n + i] = Fz;
    }
    if (MODE != FM_STORE) vv_epilogue<MODE>(a, i, Fx, Fy, Fz, a.xq[i].w);
}

}  // namespace

cudaError_t launch_overlap_index(md_system *h, bool gated) {
    const int n = (int)h->n;
    cudaStream_t s = h->stream;
    boundary_flag_kernel<<<gs_blocks(n), kBlock, 0, s>>>(n, h->cell, h->ov_cell_outer, h->ov_flag,
                                                         h->ds, gated);
    cudaError_t e = launch_scan<int32_t>(h->ov_flag, h->ov_pos, n, h->ov_bsum, h->ds, gated, s);
    if (e != cudaSuccess) return e;
    boundary_index_kernel<<<gs_blocks(n), kBlock, 0, s>>>(n, h->ov_flag, h->ov_pos, h->ov_gidx,
                                                          h->ov_bidx, h->ov_nb, h->ds, gated);
    return cudaGetLastError();
}

cudaError_t launch_overlap_forces(md_system *h, int mode, bool energy, bool store_f) {
    ForceArgs a = make_force_args(h);
    OverlapArgs o{h->cell, h->ov_cell_outer, h->ov_gidx, h->ov_bidx, h->ov_nb, h->ov_recv};
    const int n = (int)h->n;
    const int sf = store_f ? 1 : 0;
    cudaStream_t s = h->stream;
    // 1: assemble; 2-3: the exchange (a device copy on the second stream)
    assemble_kernel<<<gs_blocks(n), kBlock, 0, s>>>(h->ov_nb, h->ov_bidx, h->xq[h->cur],
                                                     h->ov_send, h->ds);
    cudaError_t e = cudaEventRecord(h->ov_ev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->ov_stream, h->ov_ev[0], 0);
    if (e == cudaSuccess) {
        exchange_kernel<<<gs_blocks(n), kBlock, 0, h->ov_stream>>>(h->ov_nb, h->ov_send,
                                                                   h->ov_recv);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(h->ov_ev[1], h->ov_stream);
    if (e != cudaSuccess) return e;
    // 4: intra-domain forces, while the copy runs
    const int nb = nblocks(n, 128);
#define MDG_OV(K, M, E) K<M, E><<<nb, 128, 0, s>>>(a, o, sf)
#define MDG_OV_MODE(K)                                                                   \
    switch (mode) {                                                                      \
        case FM_STORE: if (energy) MDG_OV(K, FM_STORE, true); else MDG_OV(K, FM_STORE, false); break; \
        case FM_FUSED_FULL: MDG_OV(K, FM_FUSED_FULL, false); break;                      \
        default: MDG_OV(K, FM_FUSED_HALF, false); break;                                 \
    }
    MDG_OV_MODE(inner_force_kernel);
    // 5 (and 7): wait for the exchange; 6: inter-domain forces
    e = cudaStreamWaitEvent(s, h->ov_ev[1], 0);
    if (e != cudaSuccess) return e;
    MDG_OV_MODE(outer_force_kernel);
#undef MDG_OV_MODE
#undef MDG_OV
    return cudaGetLastError();
}

}  // namespace mdg
