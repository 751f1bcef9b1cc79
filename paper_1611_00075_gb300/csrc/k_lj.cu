// k_lj.cu -- Lennard-Jones forces from a full neighbour list (Sec. 2.2).
//
// Pair force F = -(1/d) dPhi/dr R with R = r_i - r_j; for the truncated and
// energy-shifted Lennard-Jones pair potential
//     Phi(r) = 4 eps [(s/r)^12 - (s/r)^6] - Phi(r_c),   r < r_c,
// -(1/d) dPhi/dr = 48 eps / d^2 [(s/d)^12 - (s/d)^6 / 2].
//
// With a full list every atom sums its own force (f_j is never written by
// the thread of atom i), which is how this kernel avoids the Newton's-third-
// law race of Sec. 1 without atomics.  One thread per sorted atom walks its
// list; the lanes of a warp read their k-th entries from one 128-byte line.
//
// Precision:
//   MIXED  the pair vector, r^2, 1/r^2, (s/r)^6 and the force scalar are
//          float32, computed from cell-relative float32 coordinates plus the
//          float32 cell shift of the entry's stencil cell; each chunk of
//          kChunk entries is summed in float32 and the chunk sums are added
//          in float64 (the GPU form of the paper's blocked pair loop).
//   FP64   everything in float64 (the plain path).
//
// Modes (ForceMode): FM_STORE writes forces; FM_FUSED_FULL also applies the
// two merged half kicks of consecutive velocity-Verlet steps (v += dt f / m)
// and the drift (x += dt v) of the atom, writing its position into the other
// buffer of a double-buffered pair; FM_FUSED_HALF applies the closing half
// kick (v += dt f / 2m).  The drift also measures the displacement since the
// last list build and raises the rebuild flag past half the skin (Sec. 3.3).
#include "k_common.cuh"

namespace mdg {

template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(kBlock) lj_mixed_kernel(ForceArgs a, int store_f) {
    __shared__ float4 sh[kStencil];
    if (threadIdx.x < kStencil) {
        int s = threadIdx.x;
        int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        sh[s] = make_float4((float)(dx * a.g.w[0]), (float)(dy * a.g.w[1]),
                            (float)(dz * a.g.w[2]), 0.f);
    }
    __syncthreads();
    if (a.ds->status != 0) return;
    step_bookkeeping<MODE>(a);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const float4 qi = a.xq[i];
    const int cnt = min(a.ncount[i], a.cap);
    const uint32_t *lp = a.nlist + (size_t)(i >> 5) * (size_t)a.cap * 32 + (size_t)(i & 31);
    const float rc2 = a.fc.rc2f, sig2 = a.fc.sig2f, e48 = a.fc.eps48f;
    double Fx = 0.0, Fy = 0.0, Fz = 0.0, E = 0.0;
    unsigned npair = 0;
    for (int k0 = 0; k0 < cnt; k0 += kChunk) {
        const int k1 = min(k0 + kChunk, cnt);
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
        for (int k = k0; k < k1; ++k) {
            const uint32_t ent = __ldg(lp + (size_t)k * 32);
            const float4 qj = __ldg(a.xq + (ent & kIndexMask));
            const float4 sf = sh[ent >> kIndexBits];
            const float ex = (qj.x - qi.x) + sf.x;
            const float ey = (qj.y - qi.y) + sf.y;
            const float ez = (qj.z - qi.z) + sf.z;
            const float r2 = ex * ex + ey * ey + ez * ez;
            if (r2 < rc2) {
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
    const size_t n = (size_t)a.n;
    if (MODE == FM_STORE || store_f) {
        a.f[i] = Fx;
        a.f[n + i] = Fy;
        a.f[2 * n + i] = Fz;
    }
    if (ENERGY) {
        a.e_atom[i] = 0.5 * E;
        count_pairs(a.ds, npair);
    }
    if (MODE != FM_STORE) vv_epilogue<MODE>(a, i, Fx, Fy, Fz, qi.w);
}

template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(kBlock) lj_fp64_kernel(ForceArgs a, int store_f) {
    __shared__ double3 sh[kStencil];
    if (threadIdx.x < kStencil) {
        int s = threadIdx.x;
        int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        sh[s] = make_double3(dx * a.g.w[0], dy * a.g.w[1], dz * a.g.w[2]);
    }
    __syncthreads();
    if (a.ds->status != 0) return;
    step_bookkeeping<MODE>(a);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double4 ri = a.xr[i];
    const int cnt = min(a.ncount[i], a.cap);
    const uint32_t *lp = a.nlist + (size_t)(i >> 5) * (size_t)a.cap * 32 + (size_t)(i & 31);
    const double rc2 = a.fc.rc2, sig2 = a.fc.sig2, e48 = a.fc.eps48;
    double fx = 0.0, fy = 0.0, fz = 0.0, e = 0.0;
    unsigned npair = 0;
    for (int k = 0; k < cnt; ++k) {
        const uint32_t ent = __ldg(lp + (size_t)k * 32);
        const double4 rj = a.xr[ent & kIndexMask];
        const double3 sd = sh[ent >> kIndexBits];
        const double ex = (rj.x - ri.x) + sd.x;
        const double ey = (rj.y - ri.y) + sd.y;
        const double ez = (rj.z - ri.z) + sd.z;
        const double r2 = ex * ex + ey * ey + ez * ez;
        if (r2 < rc2) {
            const double r2i = 1.0 / r2;
            double s6 = sig2 * r2i;
            s6 = s6 * s6 * s6;
            const double fs = e48 * r2i * s6 * (s6 - 0.5);
            fx -= fs * ex;
            fy -= fs * ey;
            fz -= fs * ez;
            if (ENERGY) {
                e += a.fc.eps4 * s6 * (s6 - 1.0) - a.fc.shift;
                ++npair;
            }
        }
    }
    const size_t n = (size_t)a.n;
    if (MODE == FM_STORE || store_f) {
        a.f[i] = fx;
        a.f[n + i] = fy;
        a.f[2 * n + i] = fz;
    }
    if (ENERGY) {
        a.e_atom[i] = 0.5 * e;
        count_pairs(a.ds, npair);
    }
    if (MODE != FM_STORE) {
        const float4 qi = a.xq[i];
        vv_epilogue<MODE>(a, i, fx, fy, fz, qi.w);
    }
}

ForceArgs make_force_args(md_system *h) {
    ForceArgs a;
    a.n = (int)h->n;
    a.cap = h->cap;
    a.step = (int)h->steps_total;
    a.rebuild_every = h->p.rebuild_every;
    int cur = h->cur, nxt = cur ^ 1;
    a.xq = h->xq[cur];
    a.xq_out = h->xq[nxt];
    a.xr = h->xr64[cur];
    a.xr_out = h->xr64[nxt];
    a.xq_build = h->xq_build;
    a.v = h->v;
    a.f = h->f;
    a.e_atom = h->e_atom;
    a.nlist = h->nlist;
    a.ncount = h->ncount;
    a.rho = h->rho;
    a.dF32 = h->dF32;
    a.dF64 = h->dF64;
    a.ds = h->ds;
    a.g = h->g;
    a.fc = h->fc;
    return a;
}

cudaError_t launch_lj(md_system *h, int mode, bool energy, bool store_f) {
    ForceArgs a = make_force_args(h);
    const int nb = nblocks(a.n);
    const int sf = store_f ? 1 : 0;
    cudaStream_t s = h->stream;
#define MDG_LJ(K, M, E) K<M, E><<<nb, kBlock, 0, s>>>(a, sf)
    if (h->p.precision == MD_MIXED) {
        switch (mode) {
            case FM_STORE: if (energy) MDG_LJ(lj_mixed_kernel, FM_STORE, true); else MDG_LJ(lj_mixed_kernel, FM_STORE, false); break;
            case FM_FUSED_FULL: if (energy) MDG_LJ(lj_mixed_kernel, FM_FUSED_FULL, true); else MDG_LJ(lj_mixed_kernel, FM_FUSED_FULL, false); break;
            default: if (energy) MDG_LJ(lj_mixed_kernel, FM_FUSED_HALF, true); else MDG_LJ(lj_mixed_kernel, FM_FUSED_HALF, false); break;
        }
    } else {
        switch (mode) {
            case FM_STORE: if (energy) MDG_LJ(lj_fp64_kernel, FM_STORE, true); else MDG_LJ(lj_fp64_kernel, FM_STORE, false); break;
            case FM_FUSED_FULL: if (energy) MDG_LJ(lj_fp64_kernel, FM_FUSED_FULL, true); else MDG_LJ(lj_fp64_kernel, FM_FUSED_FULL, false); break;
            default: if (energy) MDG_LJ(lj_fp64_kernel, FM_FUSED_HALF, true); else MDG_LJ(lj_fp64_kernel, FM_FUSED_HALF, false); break;
        }
    }
#undef MDG_LJ
    return cudaGetLastError();
}

}  // namespace mdg
