// k_half.cu -- Lennard-Jones forces from a HALF list, i.e. with Newton's
// third law: each pair is evaluated once and its force F is added to f_i and
// subtracted from f_j (the pair loop of Sec. 2.2).  Two threads that update
// the same f_j at once is the race problem of Sec. 1; the paper's cell-task
// schedule (Sec. 2.1) avoids it by never running two tasks that touch the same
// particle.  Two GPU forms:
//
//   HALF_ATOMIC  one thread per owner atom; f_j updates are float64 atomic
//                adds; f_i is summed in registers and added atomically once.
//   HALF_COLOR   cells are coloured (color_1d) so that same-colour cells have
//                disjoint 27-cell neighbourhoods, and one launch per colour
//                runs one warp per cell.  The warp walks its cell's atoms one
//                at a time; its lanes take that atom's list entries, whose
//                targets j are distinct, so f_j is updated with plain loads
//                and stores -- no atomics, like the paper's lock-free tasks.
//
// A half list holds pair (i, j) at the atom with the lower original id.  On
// the mixed path the pair terms are float32 as in the full-list mixed kernel;
// on the float64 path (F64) they are float64 from the float64 cell-relative
// positions, as in the plain full-list kernel.  Every update of f and of the
// per-atom energy (split half and half between the two atoms) is float64.
// The velocity-Verlet update runs afterwards in integrate_kernel, because an
// atom's force is complete only when the whole pass has finished.
#include "k_common.cuh"

namespace mdg {

namespace {

__device__ __forceinline__ void shifts_f32(const Grid &g, float4 *sh) {
    if (threadIdx.x < kStencil) {
        int s = threadIdx.x;
        int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        sh[s] = make_float4((float)(dx * g.w[0]), (float)(dy * g.w[1]), (float)(dz * g.w[2]),
                            0.f);
    }
}

__device__ __forceinline__ void shifts_f64(const Grid &g, double3 *sh) {
    if (threadIdx.x < kStencil) {
        int s = threadIdx.x;
        int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        sh[s] = make_double3(dx * g.w[0], dy * g.w[1], dz * g.w[2]);
    }
}

// fp64 pair term for list entry `ent` of atom i at ri; returns false outside r_c.
__device__ __forceinline__ bool lj_pair_f64(const ForceArgs &a, const double3 *sh,
                                            const double4 &ri, uint32_t ent, double &Fx,
                                            double &Fy, double &Fz, double &phi) {
    const double4 rj = a.xr[ent & kIndexMask];
    const double3 sd = sh[ent >> kIndexBits];
    const double ex = (rj.x - ri.x) + sd.x;
    const double ey = (rj.y - ri.y) + sd.y;
    const double ez = (rj.z - ri.z) + sd.z;
    const double r2 = ex * ex + ey * ey + ez * ez;
    if (!(r2 < a.fc.rc2)) return false;
    const double r2i = 1.0 / r2;
    double s6 = a.fc.sig2 * r2i;
    s6 = s6 * s6 * s6;
    const double fs = a.fc.eps48 * r2i * s6 * (s6 - 0.5);
    Fx = -fs * ex;  // force on i: fs (r_i - r_j)
    Fy = -fs * ey;
    Fz = -fs * ez;
    phi = a.fc.eps4 * s6 * (s6 - 1.0) - a.fc.shift;
    return true;
}

// Shared-memory shift table and the pair term of one precision.
template <bool F64>
struct HalfPrec;
template <>
struct HalfPrec<false> {
    using Acc = float;
    using Pos = float4;
    struct Tab { float4 s[kStencil]; };
    static __device__ __forceinline__ void load(const Grid &g, Tab *t) { shifts_f32(g, t->s); }
    static __device__ __forceinline__ Pos pos(const ForceArgs &a, int i) { return a.xq[i]; }
    static __device__ __forceinline__ bool pair(const ForceArgs &a, const Tab *t, const Pos &p,
                                                uint32_t ent, Acc &x, Acc &y, Acc &z, Acc &e);
};
template <>
struct HalfPrec<true> {
    using Acc = double;
    using Pos = double4;
    struct Tab { double3 s[kStencil]; };
    static __device__ __forceinline__ void load(const Grid &g, Tab *t) { shifts_f64(g, t->s); }
    static __device__ __forceinline__ Pos pos(const ForceArgs &a, int i) { return a.xr[i]; }
    static __device__ __forceinline__ bool pair(const ForceArgs &a, const Tab *t, const Pos &p,
                                                uint32_t ent, Acc &x, Acc &y, Acc &z, Acc &e) {
        return lj_pair_f64(a, t->s, p, ent, x, y, z, e);
    }
};

// fp32 pair term for list entry `ent` of atom i at qi; returns false outside r_c.
__device__ __forceinline__ bool lj_pair_f32(const ForceArgs &a, const float4 *sh,
                                            const float4 &qi, uint32_t ent, float &Fx,
                                            float &Fy, float &Fz, float &phi) {
    const float4 qj = __ldg(a.xq + (ent & kIndexMask));
    const float4 sf = sh[ent >> kIndexBits];
    const float ex = (qj.x - qi.x) + sf.x;
    const float ey = (qj.y - qi.y) + sf.y;
    const float ez = (qj.z - qi.z) + sf.z;
    const float r2 = ex * ex + ey * ey + ez * ez;
    if (!(r2 < a.fc.rc2f)) return false;
    const float r2i = __fdividef(1.0f, r2);
    float s6 = a.fc.sig2f * r2i;
    s6 = s6 * s6 * s6;
    const float fs = a.fc.eps48f * r2i * s6 * (s6 - 0.5f);
    Fx = -fs * ex;  // force on i: fs (r_i - r_j)
    Fy = -fs * ey;
    Fz = -fs * ez;
    phi = a.fc.eps4f * s6 * (s6 - 1.0f) - a.fc.shiftf;
    return true;
}

__device__ __forceinline__ bool HalfPrec<false>::pair(const ForceArgs &a, const Tab *t,
                                                      const Pos &p, uint32_t ent, Acc &x,
                                                      Acc &y, Acc &z, Acc &e) {
    return lj_pair_f32(a, t->s, p, ent, x, y, z, e);
}

template <bool ENERGY, bool F64>
__global__ void __launch_bounds__(kBlock) lj_half_atomic_kernel(ForceArgs a) {
    using P = HalfPrec<F64>;
    using Acc = typename P::Acc;
    __shared__ typename P::Tab sh;
    P::load(a.g, &sh);
    __syncthreads();
    if (a.ds->status != 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const size_t n = (size_t)a.n;
    const typename P::Pos qi = P::pos(a, i);
    const int cnt = min(a.ncount[i], a.cap);
    double Fx = 0.0, Fy = 0.0, Fz = 0.0, E = 0.0;
    unsigned npair = 0;
    for (int k0 = 0; k0 < cnt; k0 += 4 * kChunkQ) {
        const int k1 = min(k0 + 4 * kChunkQ, cnt);
        Acc fx = 0, fy = 0, fz = 0, e = 0;
        for (int k = k0; k < k1; ++k) {
            const uint32_t ent = __ldg(a.nlist + list_idx(i, k, a.cap));
            Acc px, py, pz, phi;
            if (!P::pair(a, &sh, qi, ent, px, py, pz, phi)) continue;
            const size_t j = ent & kIndexMask;
            fx += px;
            fy += py;
            fz += pz;
            atomicAdd(a.f + j, -(double)px);
            atomicAdd(a.f + n + j, -(double)py);
            atomicAdd(a.f + 2 * n + j, -(double)pz);
            if (ENERGY) {
                e += Acc(0.5) * phi;
                atomicAdd(a.e_atom + j, 0.5 * (double)phi);
                ++npair;
            }
        }
        Fx += (double)fx;
        Fy += (double)fy;
        Fz += (double)fz;
        if (ENERGY) E += (double)e;
    }
    atomicAdd(a.f + i, Fx);
    atomicAdd(a.f + n + i, Fy);
    atomicAdd(a.f + 2 * n + i, Fz);
    if (ENERGY) {
        atomicAdd(a.e_atom + i, E);
        count_pairs(a.ds, npair);
    }
}

struct ColorArgs {
    const int32_t *cell_start;
    int kx, ky, kz;     // the colour of this launch
    int tx, ty, tz;     // cells of that colour per dimension
};

template <bool ENERGY, bool F64>
__global__ void __launch_bounds__(kBlock) lj_half_color_kernel(ForceArgs a, ColorArgs ca) {
    using P = HalfPrec<F64>;
    using Acc = typename P::Acc;
    __shared__ typename P::Tab sh;
    P::load(a.g, &sh);
    __syncthreads();
    if (a.ds->status != 0) return;
    const int lane = threadIdx.x & 31;
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // one warp per cell
    if (w >= ca.tx * ca.ty * ca.tz) return;                        // warp-uniform
    const int cx = color_cell_1d(ca.kx, w % ca.tx, a.g.nx);
    const int cy = color_cell_1d(ca.ky, (w / ca.tx) % ca.ty, a.g.ny);
    const int cz = color_cell_1d(ca.kz, w / (ca.tx * ca.ty), a.g.nz);
    const int c = (cz * a.g.ny + cy) * a.g.nx + cx;
    const size_t n = (size_t)a.n;
    unsigned npair = 0;
    for (int i = ca.cell_start[c]; i < ca.cell_start[c + 1]; ++i) {
        const typename P::Pos qi = P::pos(a, i);
        const int cnt = min(a.ncount[i], a.cap);
        Acc fx = 0, fy = 0, fz = 0, e = 0;
        for (int k = lane; k < cnt; k += 32) {
            const uint32_t ent = __ldg(a.nlist + list_idx(i, k, a.cap));
            Acc px, py, pz, phi;
            if (!P::pair(a, &sh, qi, ent, px, py, pz, phi)) continue;
            const size_t j = ent & kIndexMask;  // distinct across the lanes
            fx += px;
            fy += py;
            fz += pz;
            a.f[j] -= (double)px;
            a.f[n + j] -= (double)py;
            a.f[2 * n + j] -= (double)pz;
            if (ENERGY) {
                e += Acc(0.5) * phi;
                a.e_atom[j] += 0.5 * (double)phi;
                ++npair;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            fx += __shfl_down_sync(0xffffffffu, fx, o);
            fy += __shfl_down_sync(0xffffffffu, fy, o);
            fz += __shfl_down_sync(0xffffffffu, fz, o);
            if (ENERGY) e += __shfl_down_sync(0xffffffffu, e, o);
        }
        __syncwarp();  // the lanes' f_j stores are visible before lane 0 updates f_i
        if (lane == 0) {
            a.f[i] += (double)fx;
            a.f[n + i] += (double)fy;
            a.f[2 * n + i] += (double)fz;
            if (ENERGY) a.e_atom[i] += (double)e;
        }
        __syncwarp();
    }
    if (ENERGY) count_pairs(a.ds, npair);
}

// The velocity-Verlet update for a force pass that ended before it.
template <int MODE>
__global__ void integrate_kernel(ForceArgs a) {
    if (a.ds->status != 0) return;
    step_bookkeeping<MODE>(a);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const size_t n = (size_t)a.n;
    vv_epilogue<MODE>(a, i, a.f[i], a.f[n + i], a.f[2 * n + i], a.xq[i].w);
}

}  // namespace

cudaError_t launch_lj_half(md_system *h, int mode, bool energy, int *launches) {
    ForceArgs a = make_force_args(h);
    cudaStream_t s = h->stream;
    const size_t n = (size_t)h->n;
    cudaError_t e = cudaMemsetAsync(h->f, 0, 3 * n * sizeof(double), s);
    if (e == cudaSuccess && energy) e = cudaMemsetAsync(h->e_atom, 0, n * sizeof(double), s);
    if (e != cudaSuccess) return e;
    int nl = 0;
    const bool f64 = (h->p.precision == MD_FP64);
    if (h->p.force_variant == MD_FORCE_HALF_ATOMIC) {
        const int nb = nblocks(h->n);
        if (f64) {
            if (energy) lj_half_atomic_kernel<true, true><<<nb, kBlock, 0, s>>>(a);
            else lj_half_atomic_kernel<false, true><<<nb, kBlock, 0, s>>>(a);
        } else {
            if (energy) lj_half_atomic_kernel<true, false><<<nb, kBlock, 0, s>>>(a);
            else lj_half_atomic_kernel<false, false><<<nb, kBlock, 0, s>>>(a);
        }
        ++nl;
    } else {
        const Grid &g = h->g;
        ColorArgs ca;
        ca.cell_start = h->cell_start;
        for (int kz = 0; kz < colors_1d(g.nz); ++kz)
            for (int ky = 0; ky < colors_1d(g.ny); ++ky)
                for (int kx = 0; kx < colors_1d(g.nx); ++kx) {
                    ca.kx = kx; ca.ky = ky; ca.kz = kz;
                    ca.tx = color_count_1d(kx, g.nx);
                    ca.ty = color_count_1d(ky, g.ny);
                    ca.tz = color_count_1d(kz, g.nz);
                    const long long warps = (long long)ca.tx * ca.ty * ca.tz;
                    const int nb = (int)((warps * 32 + kBlock - 1) / kBlock);
                    if (f64) {
                        if (energy) lj_half_color_kernel<true, true><<<nb, kBlock, 0, s>>>(a, ca);
                        else lj_half_color_kernel<false, true><<<nb, kBlock, 0, s>>>(a, ca);
                    } else {
                        if (energy) lj_half_color_kernel<true, false><<<nb, kBlock, 0, s>>>(a, ca);
                        else lj_half_color_kernel<false, false><<<nb, kBlock, 0, s>>>(a, ca);
                    }
                    ++nl;
                }
    }
    if (mode == FM_FUSED_FULL) integrate_kernel<FM_FUSED_FULL><<<nblocks(h->n), kBlock, 0, s>>>(a);
    else if (mode == FM_FUSED_HALF) integrate_kernel<FM_FUSED_HALF><<<nblocks(h->n), kBlock, 0, s>>>(a);
    if (mode != FM_STORE) ++nl;
    if (launches) *launches = nl;
    return cudaGetLastError();
}

}  // namespace mdg

extern "C" md_status md_color_cells(const int32_t *ncell_host, int32_t *color_host,
                                    int32_t *ncolors_host) {
    if (!ncell_host) return MD_ERR_INVALID;
    const int nx = ncell_host[0], ny = ncell_host[1], nz = ncell_host[2];
    if (nx < 3 || ny < 3 || nz < 3) return MD_ERR_INVALID;
    const int kx = mdg::colors_1d(nx), ky = mdg::colors_1d(ny);
    if (ncolors_host) *ncolors_host = kx * ky * mdg::colors_1d(nz);
    if (color_host)
        for (int cz = 0; cz < nz; ++cz)
            for (int cy = 0; cy < ny; ++cy)
                for (int cx = 0; cx < nx; ++cx)
                    color_host[((size_t)cz * ny + cy) * nx + cx] =
                        (mdg::color_1d(cz, nz) * ky + mdg::color_1d(cy, ny)) * kx +
                        mdg::color_1d(cx, nx);
    return MD_OK;
}
