// k_integrate.cu -- velocity-Verlet pieces that are not fused into a force
// kernel (Sec. 3.3), state import/export, and deterministic energy sums.
//
// The first half kick and drift of a run (v += dt f / 2m, x += dt v) need the
// forces of the previous evaluation and run here; every later step merges
// its closing half kick with the next opening one inside the force kernel.
// Positions are float64 offsets from the atom's cell centre, so the drift is
// one multiply-add per component and the float32 copy read by the pair
// kernels is a single conversion.
#include "md_internal.cuh"

namespace mdg {

namespace {

// hk_t: the half kick dt / 2m of each species of a multi-element system
// (ntypes > 0), read from the species bits of the position word.
__global__ void kick_drift_kernel(int n, double hk0, double dt, float half_skin2,
                                  int rebuild_every, double4 *__restrict__ xr,
                                  float4 *__restrict__ xq, const float4 *__restrict__ xq_build,
                                  double *__restrict__ v, const double *__restrict__ f,
                                  DevStatus *ds, int ntypes, double4 hk_t) {
    if (ds->status != 0) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ds->abs_fresh = 0;
        int sb = ds->since_build + 1;
        ds->since_build = sb;
        if (rebuild_every > 0 && sb >= rebuild_every) ds->rebuild = 1;
    }
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t N = (size_t)n;
    float4 q = xq[i];
    double hk = hk0;
    if (ntypes > 0) {
        const int t = species_of(__float_as_uint(q.w));
        hk = t < 2 ? (t == 0 ? hk_t.x : hk_t.y) : (t == 2 ? hk_t.z : hk_t.w);
    }
    double vx = v[i] + hk * f[i];
    double vy = v[N + i] + hk * f[N + i];
    double vz = v[2 * N + i] + hk * f[2 * N + i];
    v[i] = vx;
    v[N + i] = vy;
    v[2 * N + i] = vz;
    double4 r = xr[i];
    r.x += dt * vx;
    r.y += dt * vy;
    r.z += dt * vz;
    xr[i] = r;
    q.x = (float)r.x;
    q.y = (float)r.y;
    q.z = (float)r.z;
    xq[i] = q;
    float4 b = xq_build[i];
    float ddx = q.x - b.x, ddy = q.y - b.y, ddz = q.z - b.z;
    float d2 = ddx * ddx + ddy * ddy + ddz * ddz;
    if (!(d2 <= 3.0e38f)) atomicCAS(&ds->status, 0, (int)MD_ERR_NONFINITE);
    if (rebuild_every <= 0 && d2 > half_skin2) ds->rebuild = 1;
}

// Original-order input: position i becomes slot i with absolute coordinates,
// wrapped into its box [0, L).
__global__ void load_state_kernel(int n, const Grid *__restrict__ grids,
                                  const double *__restrict__ pos,
                                  const double *__restrict__ vel, double4 *__restrict__ xr,
                                  float4 *__restrict__ xq, double4 *__restrict__ xabs,
                                  double *__restrict__ v, int32_t *__restrict__ orig,
                                  int32_t *__restrict__ cell, const int64_t *__restrict__ atom_off,
                                  int R, uint16_t *__restrict__ rep, DevStatus *ds,
                                  const int32_t *__restrict__ type_orig) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        ds->abs_fresh = 1;
        ds->rebuild = 1;
    }
    if (i >= n) return;
    const size_t N = (size_t)n;
    if (pos) {
        int r = 0;
        if (rep) {
            // replica of input row i: the last r with atom_off[r] <= i
            int lo = 0, hi = R - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (atom_off[mid] <= i) lo = mid;
                else hi = mid - 1;
            }
            rep[i] = (uint16_t)lo;
            r = lo;
        }
        const Grid &g = grids[r];
        const double4 a = make_double4(wrap_coord(pos[3 * (size_t)i], g.L[0]),
                                       wrap_coord(pos[3 * (size_t)i + 1], g.L[1]),
                                       wrap_coord(pos[3 * (size_t)i + 2], g.L[2]), 0.0);
        xr[i] = a;
        xabs[i] = a;
        const uint32_t w = (uint32_t)i | (type_orig ? (uint32_t)type_orig[i] << kIndexBits : 0u);
        xq[i] = make_float4((float)a.x, (float)a.y, (float)a.z, __uint_as_float(w));
        orig[i] = i;
        cell[i] = -1;
    }
    if (vel) {
        v[i] = vel[3 * (size_t)i];
        v[N + i] = vel[3 * (size_t)i + 1];
        v[2 * N + i] = vel[3 * (size_t)i + 2];
    }
}

// Velocities only, for an existing sorted order (orig maps slot -> input row).
__global__ void load_vel_kernel(int n, const double *__restrict__ vel,
                                const int32_t *__restrict__ orig, double *__restrict__ v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t N = (size_t)n, o = (size_t)orig[i];
    v[i] = vel[3 * o];
    v[N + i] = vel[3 * o + 1];
    v[2 * N + i] = vel[3 * o + 2];
}

__global__ void get_state_kernel(int n, const Grid *__restrict__ grids,
                                 const uint16_t *__restrict__ rep, const double4 *__restrict__ xr,
                                 const double4 *__restrict__ xabs, const int32_t *__restrict__ cell,
                                 const int32_t *__restrict__ orig, const double *__restrict__ v,
                                 const double *__restrict__ f, double *pos, double *vel,
                                 double *force, const DevStatus *ds) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t N = (size_t)n, o = (size_t)orig[i];
    if (pos) {
        const Grid &g = grids[rep ? rep[i] : 0];
        double x, y, z;
        if (ds->abs_fresh) {
            double4 a = xabs[i];
            x = a.x; y = a.y; z = a.z;
        } else {
            double4 r = xr[i];
            x = r.x; y = r.y; z = r.z;
            int c = cell[i];
            if (c >= 0) {
                c -= g.cell0;
                const double3 C =
                    cell_centre_of(c % g.nx, (c / g.nx) % g.ny, c / (g.nx * g.ny), g);
                x = C.x + x;
                y = C.y + y;
                z = C.z + z;
            }
            x = wrap_coord(x, g.L[0]);
            y = wrap_coord(y, g.L[1]);
            z = wrap_coord(z, g.L[2]);
        }
        pos[3 * o] = x;
        pos[3 * o + 1] = y;
        pos[3 * o + 2] = z;
    }
    if (vel) {
        vel[3 * o] = v[i];
        vel[3 * o + 1] = v[N + i];
        vel[3 * o + 2] = v[2 * N + i];
    }
    if (force) {
        force[3 * o] = f[i];
        force[3 * o + 1] = f[N + i];
        force[3 * o + 2] = f[2 * N + i];
    }
}

__global__ void scatter_orig_kernel(int n, const int32_t *__restrict__ orig,
                                    const double *__restrict__ src, double *__restrict__ dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[orig[i]] = src[i];
}

__global__ void scatter_orig_f32_kernel(int n, const int32_t *__restrict__ orig,
                                        const float *__restrict__ src, double *__restrict__ dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[orig[i]] = (double)src[i];
}

// Fixed-shape tree sums: per-block partials, then one block over partials.
__device__ double block_sum(double x) {
    __shared__ double ws[kBlock / 32];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = x;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = (lane < kBlock / 32) ? ws[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

__global__ void partial_pe_kernel(int n, const double *__restrict__ e, double *partials) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    double x = (i < n) ? e[i] : 0.0;
    double t = block_sum(x);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void partial_ke_kernel(int n, double half_m, const double *__restrict__ v,
                                  double *partials, const float4 *__restrict__ xq_typed,
                                  double4 half_m_t) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t N = (size_t)n;
    double x = 0.0;
    if (i < n) {
        double hm = half_m;
        if (xq_typed) {  // multi-element: the species' mass
            const int t = species_of(__float_as_uint(xq_typed[i].w));
            hm = t < 2 ? (t == 0 ? half_m_t.x : half_m_t.y) : (t == 2 ? half_m_t.z : half_m_t.w);
        }
        double a = v[i], b = v[N + i], c = v[2 * N + i];
        x = hm * (a * a + b * b + c * c);
    }
    double t = block_sum(x);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void final_sum_kernel(int nb, const double *__restrict__ partials, double *out) {
    double x = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) x += partials[b];
    double t = block_sum(x);
    if (threadIdx.x == 0) *out = t;
}

__global__ void set_rebuild_kernel(DevStatus *ds) { ds->rebuild = 1; }

// One block per replica: its atoms are one contiguous sorted range (its
// cells); fixed-order sums of potential and kinetic energy.
__global__ void replica_energy_kernel(const Grid *__restrict__ grids,
                                      const int32_t *__restrict__ start,
                                      const double *__restrict__ e, const double *__restrict__ v,
                                      int n, double half_m, double *__restrict__ pe,
                                      double *__restrict__ ke) {
    const Grid &g = grids[blockIdx.x];
    const int a = start[g.cell0], b = start[g.cell0 + g.ncells];
    const size_t N = (size_t)n;
    double sp = 0.0, sk = 0.0;
    for (int i = a + threadIdx.x; i < b; i += blockDim.x) {
        sp += e[i];
        const double x = v[i], y = v[N + i], z = v[2 * N + i];
        sk += half_m * (x * x + y * y + z * z);
    }
    const double tp = block_sum(sp);
    const double tk = block_sum(sk);
    if (threadIdx.x == 0) {
        pe[blockIdx.x] = tp;
        ke[blockIdx.x] = tk;
    }
}

}  // namespace

cudaError_t launch_kick_drift(md_system *h) {
    int n = (int)h->n;
    const double *im = h->fc.t_inv_m;
    const double hd = 0.5 * h->p.dt;
    kick_drift_kernel<<<nblocks(n), kBlock, 0, h->stream>>>(
        n, 0.5 * h->p.dt / h->p.mass, h->p.dt, h->fc.half_skin2f, h->p.rebuild_every,
        h->xr64[h->cur], h->xq[h->cur], h->xq_build, h->v, h->f, h->ds, h->fc.ntypes,
        make_double4(hd * im[0], hd * im[1], hd * im[2], hd * im[3]));
    return cudaGetLastError();
}

cudaError_t launch_load_state(md_system *h, const double *pos, const double *vel) {
    int n = (int)h->n;
    if (pos) {
        load_state_kernel<<<nblocks(n), kBlock, 0, h->stream>>>(
            n, h->grids, pos, vel, h->xr64[h->cur], h->xq[h->cur], h->xabs, h->v, h->orig, h->cell,
            h->atom_off, h->R, h->rep, h->ds, h->type_orig);
    } else if (vel) {
        load_vel_kernel<<<nblocks(n), kBlock, 0, h->stream>>>(n, vel, h->orig, h->v);
    }
    return cudaGetLastError();
}

cudaError_t launch_get_state(md_system *h, double *pos, double *vel, double *force) {
    int n = (int)h->n;
    get_state_kernel<<<nblocks(n), kBlock, 0, h->stream>>>(n, h->grids, h->rep, h->xr64[h->cur],
                                                           h->xabs, h->cell, h->orig, h->v, h->f,
                                                           pos, vel, force, h->ds);
    return cudaGetLastError();
}

cudaError_t launch_replica_energy(md_system *h) {
    replica_energy_kernel<<<h->R, kBlock, 0, h->stream>>>(h->grids, h->cell_start, h->e_atom, h->v,
                                                          (int)h->n, 0.5 * h->p.mass, h->rep_pe,
                                                          h->rep_ke);
    return cudaGetLastError();
}

cudaError_t launch_scatter_orig(md_system *h, const double *src_sorted, double *dst_orig) {
    int n = (int)h->n;
    scatter_orig_kernel<<<nblocks(n), kBlock, 0, h->stream>>>(n, h->orig, src_sorted, dst_orig);
    return cudaGetLastError();
}

cudaError_t launch_scatter_orig_f32(md_system *h, const float *src_sorted, double *dst_orig) {
    int n = (int)h->n;
    scatter_orig_f32_kernel<<<nblocks(n), kBlock, 0, h->stream>>>(n, h->orig, src_sorted, dst_orig);
    return cudaGetLastError();
}

cudaError_t launch_reduce_pe(md_system *h) {
    int n = (int)h->n, nb = nblocks(n);
    partial_pe_kernel<<<nb, kBlock, 0, h->stream>>>(n, h->e_atom, h->partials);
    final_sum_kernel<<<1, kBlock, 0, h->stream>>>(nb, h->partials, h->red_out + 0);
    return cudaGetLastError();
}

cudaError_t launch_reduce_ke(md_system *h) {
    int n = (int)h->n, nb = nblocks(n);
    const double *m = h->types_mass;
    partial_ke_kernel<<<nb, kBlock, 0, h->stream>>>(
        n, 0.5 * h->p.mass, h->v, h->partials, h->fc.ntypes > 0 ? h->xq[h->cur] : nullptr,
        make_double4(0.5 * m[0], 0.5 * m[1], 0.5 * m[2], 0.5 * m[3]));
    final_sum_kernel<<<1, kBlock, 0, h->stream>>>(nb, h->partials, h->red_out + 1);
    return cudaGetLastError();
}

cudaError_t launch_set_rebuild(md_system *h) {
    set_rebuild_kernel<<<1, 1, 0, h->stream>>>(h->ds);
    return cudaGetLastError();
}

}  // namespace mdg
