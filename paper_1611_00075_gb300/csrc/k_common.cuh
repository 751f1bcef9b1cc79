// k_common.cuh -- pieces shared by the force kernels: the argument block,
// the fused velocity-Verlet epilogue (Sec. 3.3) and per-step bookkeeping.
#pragma once

#include "md_internal.cuh"

namespace mdg {

// float32 partial sums cover kChunkQ quads (64 list entries) before they are
// added to the float64 accumulators
constexpr int kChunkQ = 16;

struct ForceArgs {
    int n, cap, step, rebuild_every;
    const float4 *__restrict__ xq;
    float4 *__restrict__ xq_out;
    const double4 *__restrict__ xr;
    double4 *__restrict__ xr_out;
    const float4 *__restrict__ xq_build;
    double *__restrict__ v;
    double *__restrict__ f;
    double *__restrict__ e_atom;
    const uint32_t *__restrict__ nlist;
    const int32_t *__restrict__ ncount;
    double *__restrict__ rho;     // many-body: rho_i (Eq. 2)
    float *__restrict__ dF32;     // many-body: F'(rho_i) in float32
    float4 *__restrict__ xqf;     // many-body, mixed: (x, y, z, F'(rho)) per atom
    double *__restrict__ dF64;    // many-body: F'(rho_i) in float64
    const uint16_t *__restrict__ rep;     // batches: replica of each sorted atom
    const float4 *__restrict__ shifts32;  // batches: R x 27 float32 cell shifts
    DevStatus *ds;
    Grid g;
    ForceConsts fc;
};

// Float32 cell shifts (dx, dy, dz) * w of the 27 stencil cells, in shared
// memory, one array per component: the lanes of a warp read up to 27
// distinct words of one array, which sit in 27 distinct banks, so each read
// is a single wavefront (a float4 table costs several).
struct ShiftTab {
    float x[32], y[32], z[32];
};

__device__ __forceinline__ void load_shifts_f32(const Grid &g, ShiftTab *sh) {
    if (threadIdx.x < kStencil) {
        int s = threadIdx.x;
        int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        sh->x[s] = (float)(dx * g.w[0]);
        sh->y[s] = (float)(dy * g.w[1]);
        sh->z[s] = (float)(dz * g.w[2]);
    }
}

// Fills a ForceArgs from the handle for the current double-buffer index.
ForceArgs make_force_args(md_system *h);

// Shared epilogue: kick (and drift) of atom i with its float64 force.
// SPECIES: a multi-element system, whose atom takes its species' mass (a
// compile-time switch: a run-time test here cost the persistent kernel 6 %).
template <int MODE, bool SPECIES = false>
__device__ __forceinline__ void vv_epilogue(const ForceArgs &a, int i, double Fx, double Fy,
                                            double Fz, float qw) {
    const size_t n = (size_t)a.n;
    double im = a.fc.inv_m;
    if (SPECIES) im = pick4(a.fc.t_inv_m, species_of(__float_as_uint(qw)));
    const double hk = (MODE == FM_FUSED_FULL) ? a.fc.dt * im : 0.5 * a.fc.dt * im;
    double vx = a.v[i] + hk * Fx;
    double vy = a.v[n + i] + hk * Fy;
    double vz = a.v[2 * n + i] + hk * Fz;
    a.v[i] = vx;
    a.v[n + i] = vy;
    a.v[2 * n + i] = vz;
    if (MODE == FM_FUSED_FULL) {
        double4 r = a.xr[i];
        r.x += a.fc.dt * vx;
        r.y += a.fc.dt * vy;
        r.z += a.fc.dt * vz;
        a.xr_out[i] = r;
        float4 q = make_float4((float)r.x, (float)r.y, (float)r.z, qw);
        a.xq_out[i] = q;
        float4 b = a.xq_build[i];
        float ddx = q.x - b.x, ddy = q.y - b.y, ddz = q.z - b.z;
        float d2 = ddx * ddx + ddy * ddy + ddz * ddz;
        if (!(d2 <= 3.0e38f)) atomicCAS(&a.ds->status, 0, (int)MD_ERR_NONFINITE);
        if (a.rebuild_every <= 0 && d2 > a.fc.half_skin2f) a.ds->rebuild = 1;
    }
}

// Adds v over the converged lanes of the warp to the in-cutoff pair counter
// (correct for any subset of lanes: each group's leader adds its own sum).
__device__ __forceinline__ void count_pairs(DevStatus *ds, unsigned v) {
    const unsigned m = __activemask();
    const unsigned t = __reduce_add_sync(m, v);
    if ((int)(threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(&ds->pairs_cut, (unsigned long long)t);
}

template <int MODE>
__device__ __forceinline__ void step_bookkeeping(const ForceArgs &a) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (MODE == FM_FUSED_FULL) {
            a.ds->abs_fresh = 0;
            int sb = a.ds->since_build + 1;
            a.ds->since_build = sb;
            if (a.rebuild_every > 0 && sb >= a.rebuild_every) a.ds->rebuild = 1;
        }
        // a device-side count, so that a step replayed from a CUDA graph counts too
        if (MODE != FM_STORE) a.ds->steps_done += 1;
    }
}

}  // namespace mdg
