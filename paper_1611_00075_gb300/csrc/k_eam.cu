// k_eam.cu -- embedded-atom forces with piecewise functions, the form of the
// paper's Fe potential (Sec. 3.1), in the paper's three steps: a pair pass for
// rho_i (Eq. 2), the embedding derivative as that pass's epilogue, and a pair
// pass for the pair term and the forces.
//
//   Phi(r) = sum_k a_k (r_k - r)^3 over the knots with r < r_k
//   psi(r) = sum_k b_k (s_k - r)^3 over the knots with r < s_k
//   F(rho) = -A sqrt(rho) + B rho^2
//   f_i = -sum_j [Phi'(r) + (F'(rho_i) + F'(rho_j)) psi'(r)] (r_i - r_j) / r
//
// A knot's term is written max(r_k - r, 0)^3: the same instructions for every
// pair whichever side of the knot it lies, so a warp never diverges on the
// pieces (the paper's SIMD loop had to mask them, Sec. 4.1 / Table 2).  The
// knot tables sit in the kernel's parameter space and are read with
// warp-uniform indices.
//
// Precision as for Sutton-Chen: MIXED evaluates r, the pieces and the pair
// force in float32 from cell-relative float32 coordinates and sums rho and the
// forces in float64 over float32 chunks; F'(rho) is float64 at the atom step
// and feeds the float32 pair terms as float32; energies are float64.
#include "k_common.cuh"
#include "k_pair.cuh"

namespace mdg {

namespace {

// sum_k c_k max(k_k - r, 0)^3 and its derivative -3 sum_k c_k max(k_k - r, 0)^2
// (float32); NK > 0 fixes the knot count at compile time.
template <int NK>
__device__ __forceinline__ float pieces_f32(const float *knot, const float *c, int nk, float r,
                                            float *deriv) {
    float v = 0.f, d = 0.f;
    const int m = NK > 0 ? NK : nk;
#pragma unroll
    for (int k = 0; k < (NK > 0 ? NK : kEamMaxKnots); ++k) {
        if (NK == 0 && k >= m) break;
        const float t = fmaxf(knot[k] - r, 0.f);
        const float t2 = t * t;
        v = fmaf(c[k] * t2, t, v);
        d = fmaf(c[k], t2, d);
    }
    if (deriv) *deriv = -3.f * d;
    return v;
}

__device__ __forceinline__ double pieces_f64(const double *knot, const double *c, int nk,
                                             double r, double *deriv) {
    double v = 0.0, d = 0.0;
    for (int k = 0; k < nk; ++k) {
        const double t = fmax(knot[k] - r, 0.0);
        v += c[k] * t * t * t;
        d += c[k] * t * t;
    }
    if (deriv) *deriv = -3.0 * d;
    return v;
}

// The atom step of Sec. 3.1: F'(rho) = -A / (2 sqrt(rho)) + 2 B rho (float64).
__device__ __forceinline__ double eam_dF(const EamTab &t, double rho) {
    double d = 2.0 * t.B * rho;
    if (rho > 0.0) d += -0.5 * t.A / sqrt(rho);
    return d;
}
__device__ __forceinline__ double eam_F(const EamTab &t, double rho) {
    return -t.A * sqrt(rho) + t.B * rho * rho;
}

// Both mixed passes: 256-thread blocks at up to 64 registers.
template <int NPSI>
__global__ void __launch_bounds__(kBlock, 4) eam_density_mixed(ForceArgs a, EamTab t) {
    __shared__ ShiftTab sh;
    load_shifts_f32(a.g, &sh);
    __syncthreads();
    if (a.ds->status != 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const float4 qi = a.xq[i];
    const int nq = (min(a.ncount[i], a.cap) + 3) >> 2;
    const uint4 *lq = reinterpret_cast<const uint4 *>(a.nlist + list_group(i, a.cap)) + (i & 31);
    const float rc2 = a.fc.rc2f;
    double R = 0.0;
    uint4 nxt = nq > 0 ? __ldcs(lq) : make_uint4(0u, 0u, 0u, 0u);
    for (int q0 = 0; q0 < nq; q0 += kChunkQ) {
        const int q1 = min(q0 + kChunkQ, nq);
        float r = 0.f;
        auto pair = [&](uint32_t ent) {
            const float4 qj = __ldg(a.xq + (ent & kIndexMask));
            const uint32_t st = ent >> kIndexBits;
            const float ex = (qj.x - qi.x) + sh.x[st];
            const float ey = (qj.y - qi.y) + sh.y[st];
            const float ez = (qj.z - qi.z) + sh.z[st];
            const float r2 = ex * ex + ey * ey + ez * ez;
            if (r2 < rc2) r += pieces_f32<NPSI>(t.qr, t.qa, t.npsi, r2 * rsqrtf(r2), nullptr);
        };
        for (int q = q0; q < q1; ++q) {
            const uint4 e4 = nxt;
            if (q + 1 < nq) nxt = __ldcs(lq + (size_t)(q + 1) * 32);
            pair(e4.x);
            pair(e4.y);
            pair(e4.z);
            pair(e4.w);
        }
        R += (double)r;
    }
    a.rho[i] = R;
    const float dF = (float)eam_dF(t, R);
    a.dF32[i] = dF;
    // the force pass gathers F'(rho_j) together with the position of j
    a.xqf[i] = make_float4(qi.x, qi.y, qi.z, dF);
}

__global__ void __launch_bounds__(kBlock) eam_density_fp64(ForceArgs a, EamTab t) {
    __shared__ double3 sh[kStencil];
    if (threadIdx.x < kStencil) {
        const int s = threadIdx.x;
        const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        sh[s] = make_double3(dx * a.g.w[0], dy * a.g.w[1], dz * a.g.w[2]);
    }
    __syncthreads();
    if (a.ds->status != 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double4 ri = a.xr[i];
    const int cnt = min(a.ncount[i], a.cap);
    const double rc2 = a.fc.rc2;
    double R = 0.0;
    for (int k = 0; k < cnt; ++k) {
        const uint32_t ent = __ldg(a.nlist + list_idx(i, k, a.cap));
        const double4 rj = a.xr[ent & kIndexMask];
        const double3 sd = sh[ent >> kIndexBits];
        const double ex = (rj.x - ri.x) + sd.x;
        const double ey = (rj.y - ri.y) + sd.y;
        const double ez = (rj.z - ri.z) + sd.z;
        const double r2 = ex * ex + ey * ey + ez * ez;
        if (r2 < rc2) R += pieces_f64(t.qrd, t.qad, t.npsi, sqrt(r2), nullptr);
    }
    a.rho[i] = R;
    const double d = eam_dF(t, R);
    a.dF64[i] = d;
    a.dF32[i] = (float)d;
}

template <int MODE, bool ENERGY, int NPHI, int NPSI>
__global__ void __launch_bounds__(kBlock, 4) eam_force_mixed(ForceArgs a, EamTab t, int store_f) {
    __shared__ ShiftTab sh;
    load_shifts_f32(a.g, &sh);
    __syncthreads();
    if (a.ds->status != 0) return;
    step_bookkeeping<MODE>(a);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const float4 qi = a.xqf[i];  // position, F'(rho_i)
    const float dFi = qi.w;
    const int nq = (min(a.ncount[i], a.cap) + 3) >> 2;
    const uint4 *lq = reinterpret_cast<const uint4 *>(a.nlist + list_group(i, a.cap)) + (i & 31);
    const float rc2 = a.fc.rc2f;
    double Fx = 0.0, Fy = 0.0, Fz = 0.0, E = 0.0;
    unsigned npair = 0;
    uint4 nxt = nq > 0 ? __ldcs(lq) : make_uint4(0u, 0u, 0u, 0u);
    for (int q0 = 0; q0 < nq; q0 += kChunkQ) {
        const int q1 = min(q0 + kChunkQ, nq);
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
        auto pair = [&](uint32_t ent) {
            const float4 qj = __ldg(a.xqf + (ent & kIndexMask));  // position, F'(rho_j)
            const uint32_t st = ent >> kIndexBits;
            const float ex = (qj.x - qi.x) + sh.x[st];
            const float ey = (qj.y - qi.y) + sh.y[st];
            const float ez = (qj.z - qi.z) + sh.z[st];
            const float r2 = ex * ex + ey * ey + ez * ez;
            if (r2 < rc2) {
                const float rinv = rsqrtf(r2);
                const float r = r2 * rinv;
                float dPhi, dpsi;
                const float Phi = pieces_f32<NPHI>(t.pr, t.pa, t.nphi, r, &dPhi);
                pieces_f32<NPSI>(t.qr, t.qa, t.npsi, r, &dpsi);
                // f_i += g (r_j - r_i) / r with g = Phi' + (F'_i + F'_j) psi'
                const float fs = (dPhi + (dFi + qj.w) * dpsi) * rinv;
                fx = fmaf(fs, ex, fx);
                fy = fmaf(fs, ey, fy);
                fz = fmaf(fs, ez, fz);
                if (ENERGY) {
                    e += Phi;
                    ++npair;
                }
            }
        };
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
        if (ENERGY) E += (double)e;
    }
    const size_t n = (size_t)a.n;
    if (MODE == FM_STORE || store_f) {
        a.f[i] = Fx;
        a.f[n + i] = Fy;
        a.f[2 * n + i] = Fz;
    }
    if (ENERGY) {
        a.e_atom[i] = 0.5 * E + eam_F(t, a.rho[i]);
        count_pairs(a.ds, npair);
    }
    // the float32 position's w word holds the original id
    if (MODE != FM_STORE)
        vv_epilogue<MODE>(a, i, Fx, Fy, Fz, reinterpret_cast<const float *>(a.xq)[4 * (size_t)i + 3]);
}

template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(kBlock) eam_force_fp64(ForceArgs a, EamTab t, int store_f) {
    __shared__ double3 sh[kStencil];
    if (threadIdx.x < kStencil) {
        const int s = threadIdx.x;
        const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        sh[s] = make_double3(dx * a.g.w[0], dy * a.g.w[1], dz * a.g.w[2]);
    }
    __syncthreads();
    if (a.ds->status != 0) return;
    step_bookkeeping<MODE>(a);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double4 ri = a.xr[i];
    const double dFi = a.dF64[i];
    const int cnt = min(a.ncount[i], a.cap);
    const double rc2 = a.fc.rc2;
    double fx = 0.0, fy = 0.0, fz = 0.0, e = 0.0;
    unsigned npair = 0;
    for (int k = 0; k < cnt; ++k) {
        const uint32_t ent = __ldg(a.nlist + list_idx(i, k, a.cap));
        const int j = (int)(ent & kIndexMask);
        const double4 rj = a.xr[j];
        const double3 sd = sh[ent >> kIndexBits];
        const double ex = (rj.x - ri.x) + sd.x;
        const double ey = (rj.y - ri.y) + sd.y;
        const double ez = (rj.z - ri.z) + sd.z;
        const double r2 = ex * ex + ey * ey + ez * ez;
        if (r2 < rc2) {
            const double r = sqrt(r2);
            double dPhi, dpsi;
            const double Phi = pieces_f64(t.prd, t.pad, t.nphi, r, &dPhi);
            pieces_f64(t.qrd, t.qad, t.npsi, r, &dpsi);
            const double fs = (dPhi + (dFi + a.dF64[j]) * dpsi) / r;
            fx += fs * ex;
            fy += fs * ey;
            fz += fs * ez;
            if (ENERGY) {
                e += Phi;
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
        a.e_atom[i] = 0.5 * e + eam_F(t, a.rho[i]);
        count_pairs(a.ds, npair);
    }
    if (MODE != FM_STORE) {
        const float4 qi = a.xq[i];
        vv_epilogue<MODE>(a, i, fx, fy, fz, qi.w);
    }
}

// ---- two atoms per thread (MD_FORCE_PAIRED) ---------------------------------
//
// The slot layout of k_pair.cu (two atoms of one cell, the union of their
// lists), as for Lennard-Jones and Sutton-Chen: the slot's own pair once,
// then both atoms against each entry with packed float32 pairs.  Every knot
// lies in (0, r_c], so each piece vanishes at r_c and beyond: entries past
// the cutoff, and the padding's far dummy, add exactly zero without a test.
// Sums: float32 over chunks of kChunkQ quads, float64 across chunks.
constexpr int kEamPairBlock = 128;

__device__ __forceinline__ float2 max2(float2 a, float b) {
    return make_float2(fmaxf(a.x, b), fmaxf(a.y, b));
}

// the two lanes' sum_k c_k max(k_k - r, 0)^3 and derivative -3 sum_k c_k max(k_k - r, 0)^2
template <int NK, bool DERIV>
__device__ __forceinline__ float2 pieces_pair(const float *knot, const float *c, int nk, float2 r,
                                              float2 *deriv) {
    float2 v = dup2(0.f), d = dup2(0.f);
    const int m = NK > 0 ? NK : nk;
#pragma unroll
    for (int k = 0; k < (NK > 0 ? NK : kEamMaxKnots); ++k) {
        if (NK == 0 && k >= m) break;
        const float2 tk = max2(add2(dup2(knot[k]), make_float2(-r.x, -r.y)), 0.f);
        const float2 t2 = mul2(tk, tk);
        v = fma2(mul2(dup2(c[k]), t2), tk, v);
        if (DERIV) d = fma2(dup2(c[k]), t2, d);
    }
    if (DERIV) *deriv = mul2(dup2(-3.f), d);
    return v;
}

template <int NPSI>
__global__ void __launch_bounds__(kEamPairBlock, 8) eam_density_pair(ForceArgs a, PairArgs p,
                                                                     EamTab t) {
    __shared__ ShiftTab sh;
    load_shifts_f32(a.g, &sh);
    __syncthreads();
    if (a.ds->status != 0) return;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.slot_start[p.ncells]) return;
    const uint32_t sa = p.slot_atom[s];
    const int i0 = (int)(sa & ~kSingle);
    const bool two = !(sa & kSingle);
    const float4 q0 = a.xq[i0];
    const float4 q1 = two ? a.xq[i0 + 1] : make_float4(3.0e18f, 3.0e18f, 3.0e18f, 0.f);
    const float rc2 = a.fc.rc2f;
    float2 r = dup2(0.f);
    {
        // the slot's own pair adds to both densities
        const float ex = q1.x - q0.x, ey = q1.y - q0.y, ez = q1.z - q0.z;
        const float r2 = ex * ex + ey * ey + ez * ez;
        if (r2 < rc2) r = dup2(pieces_f32<NPSI>(t.qr, t.qa, t.npsi, r2 * rsqrtf(r2), nullptr));
    }
    const float2 nqx = make_float2(-q0.x, -q1.x), nqy = make_float2(-q0.y, -q1.y),
                 nqz = make_float2(-q0.z, -q1.z);
    const int nq = (min(p.count[s], p.cap) + 3) >> 2;
    const uint4 *lq = reinterpret_cast<const uint4 *>(p.list + list_group(s, p.cap)) + (s & 31);
    auto pair = [&](uint32_t ent) {
        const float4 qj = __ldg(a.xq + (ent & kIndexMask));
        const uint32_t st = ent >> kIndexBits;
        const float tx = qj.x + sh.x[st], ty = qj.y + sh.y[st], tz = qj.z + sh.z[st];
        const float2 dx = add2(dup2(tx), nqx), dy = add2(dup2(ty), nqy), dz = add2(dup2(tz), nqz);
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float2 rr = mul2(r2, make_float2(rsqrtf(r2.x), rsqrtf(r2.y)));
        r = add2(r, pieces_pair<NPSI, false>(t.qr, t.qa, t.npsi, rr, nullptr));
    };
    double R0 = 0.0, R1 = 0.0;
    uint4 nxt = nq > 0 ? __ldcs(lq) : make_uint4(0u, 0u, 0u, 0u);
    for (int c0 = 0; c0 < nq; c0 += kChunkQ) {
        const int c1 = min(c0 + kChunkQ, nq);
        for (int q = c0; q < c1; ++q) {
            const uint4 e4 = nxt;
            if (q + 1 < nq) nxt = __ldcs(lq + (size_t)(q + 1) * 32);
            pair(e4.x);
            pair(e4.y);
            pair(e4.z);
            pair(e4.w);
        }
        R0 += (double)r.x;
        R1 += (double)r.y;
        r = dup2(0.f);
    }
    R0 += (double)r.x;
    R1 += (double)r.y;
    // the atom step (embedding derivative) and the gather record of the force pass
    const float d0 = (float)eam_dF(t, R0);
    a.rho[i0] = R0;
    a.dF32[i0] = d0;
    a.xqf[i0] = make_float4(q0.x, q0.y, q0.z, d0);
    if (two) {
        const float d1 = (float)eam_dF(t, R1);
        a.rho[i0 + 1] = R1;
        a.dF32[i0 + 1] = d1;
        a.xqf[i0 + 1] = make_float4(q1.x, q1.y, q1.z, d1);
    }
}

template <int MODE, bool ENERGY>
__device__ __forceinline__ void eam_pair_atom_out(const ForceArgs &a, const EamTab &t, int i,
                                                  double Fx, double Fy, double Fz, double E,
                                                  unsigned np, int store_f) {
    const size_t n = (size_t)a.n;
    if (MODE == FM_STORE || store_f) {
        a.f[i] = Fx;
        a.f[n + i] = Fy;
        a.f[2 * n + i] = Fz;
    }
    if (ENERGY) {
        a.e_atom[i] = 0.5 * E + eam_F(t, a.rho[i]);
        count_pairs(a.ds, np);
    }
    // the float32 position's w word holds the original id
    if (MODE != FM_STORE)
        vv_epilogue<MODE>(a, i, Fx, Fy, Fz, reinterpret_cast<const float *>(a.xq)[4 * (size_t)i + 3]);
}

template <int MODE, bool ENERGY, int NPHI, int NPSI>
__global__ void __launch_bounds__(kEamPairBlock, 8) eam_force_pair(ForceArgs a, PairArgs p,
                                                                   EamTab t, int store_f) {
    __shared__ ShiftTab sh;
    load_shifts_f32(a.g, &sh);
    __syncthreads();
    if (a.ds->status != 0) return;
    step_bookkeeping<MODE>(a);
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.slot_start[p.ncells]) return;
    const uint32_t sa = p.slot_atom[s];
    const int i0 = (int)(sa & ~kSingle);
    const bool two = !(sa & kSingle);
    const float4 q0 = a.xqf[i0];  // position, F'(rho)
    const float4 q1 = two ? a.xqf[i0 + 1] : make_float4(3.0e18f, 3.0e18f, 3.0e18f, 0.f);
    const float2 dFi = make_float2(q0.w, q1.w);
    const float rc2 = a.fc.rc2f;
    float2 fx = dup2(0.f), fy = dup2(0.f), fz = dup2(0.f), en = dup2(0.f);
    unsigned np0 = 0, np1 = 0;
    {
        // the slot's own pair once: e = x_1 - x_0, f_0 += g e / r, f_1 -= g e / r
        const float ex = q1.x - q0.x, ey = q1.y - q0.y, ez = q1.z - q0.z;
        const float r2 = ex * ex + ey * ey + ez * ez;
        if (r2 < rc2) {
            const float rinv = rsqrtf(r2);
            const float rr = r2 * rinv;
            float dPhi, dpsi;
            const float Phi = pieces_f32<NPHI>(t.pr, t.pa, t.nphi, rr, &dPhi);
            pieces_f32<NPSI>(t.qr, t.qa, t.npsi, rr, &dpsi);
            const float fs = (dPhi + (q0.w + q1.w) * dpsi) * rinv;
            fx = make_float2(fs * ex, -fs * ex);
            fy = make_float2(fs * ey, -fs * ey);
            fz = make_float2(fs * ez, -fs * ez);
            if (ENERGY) {
                en = dup2(Phi);
                np0 = np1 = 1;
            }
        }
    }
    const float2 nqx = make_float2(-q0.x, -q1.x), nqy = make_float2(-q0.y, -q1.y),
                 nqz = make_float2(-q0.z, -q1.z);
    const int nq = (min(p.count[s], p.cap) + 3) >> 2;
    const uint4 *lq = reinterpret_cast<const uint4 *>(p.list + list_group(s, p.cap)) + (s & 31);
    // f_i += g (x_j - x_i) / r with g = Phi' + (F'_i + F'_j) psi'
    auto pair = [&](uint32_t ent) {
        const float4 qj = __ldg(a.xqf + (ent & kIndexMask));  // position, F'(rho_j)
        const uint32_t st = ent >> kIndexBits;
        const float tx = qj.x + sh.x[st], ty = qj.y + sh.y[st], tz = qj.z + sh.z[st];
        const float2 dx = add2(dup2(tx), nqx), dy = add2(dup2(ty), nqy), dz = add2(dup2(tz), nqz);
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float2 rinv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        const float2 rr = mul2(r2, rinv);
        float2 dPhi, dpsi;
        const float2 Phi = pieces_pair<NPHI, true>(t.pr, t.pa, t.nphi, rr, &dPhi);
        pieces_pair<NPSI, true>(t.qr, t.qa, t.npsi, rr, &dpsi);
        const float2 fs = mul2(fma2(add2(dFi, dup2(qj.w)), dpsi, dPhi), rinv);
        fx = fma2(fs, dx, fx);
        fy = fma2(fs, dy, fy);
        fz = fma2(fs, dz, fz);
        if (ENERGY) {
            en = add2(en, Phi);
            np0 += r2.x < rc2 ? 1u : 0u;
            np1 += r2.y < rc2 ? 1u : 0u;
        }
    };
    double F0x = 0.0, F0y = 0.0, F0z = 0.0, F1x = 0.0, F1y = 0.0, F1z = 0.0, E0 = 0.0, E1 = 0.0;
    auto flush = [&]() {
        F0x += (double)fx.x; F0y += (double)fy.x; F0z += (double)fz.x;
        F1x += (double)fx.y; F1y += (double)fy.y; F1z += (double)fz.y;
        fx = fy = fz = dup2(0.f);
        if (ENERGY) {
            E0 += (double)en.x;
            E1 += (double)en.y;
            en = dup2(0.f);
        }
    };
    uint4 nxt = nq > 0 ? __ldcs(lq) : make_uint4(0u, 0u, 0u, 0u);
    for (int c0 = 0; c0 < nq; c0 += kChunkQ) {
        const int c1 = min(c0 + kChunkQ, nq);
        for (int q = c0; q < c1; ++q) {
            const uint4 e4 = nxt;
            if (q + 1 < nq) nxt = __ldcs(lq + (size_t)(q + 1) * 32);
            pair(e4.x);
            pair(e4.y);
            pair(e4.z);
            pair(e4.w);
        }
        flush();
    }
    flush();
    eam_pair_atom_out<MODE, ENERGY>(a, t, i0, F0x, F0y, F0z, E0, np0, store_f);
    if (two) eam_pair_atom_out<MODE, ENERGY>(a, t, i0 + 1, F1x, F1y, F1z, E1, np1, store_f);
}

}  // namespace

cudaError_t launch_eam_density(md_system *h) {
    ForceArgs a = make_force_args(h);
    const int nb = nblocks(a.n);
    const EamTab &t = h->eam;
    if (h->p.force_variant == MD_FORCE_PAIRED) {
        const PairArgs p = make_pair_args(h);
        const int pb = pair_grid_blocks(h, kEamPairBlock);
        if (t.npsi == 1) eam_density_pair<1><<<pb, kEamPairBlock, 0, h->stream>>>(a, p, t);
        else eam_density_pair<0><<<pb, kEamPairBlock, 0, h->stream>>>(a, p, t);
        return cudaGetLastError();
    }
    if (h->p.precision == MD_MIXED) {
        if (t.npsi == 1) eam_density_mixed<1><<<nb, kBlock, 0, h->stream>>>(a, t);
        else eam_density_mixed<0><<<nb, kBlock, 0, h->stream>>>(a, t);
    } else {
        eam_density_fp64<<<nb, kBlock, 0, h->stream>>>(a, t);
    }
    return cudaGetLastError();
}

cudaError_t launch_eam_force(md_system *h, int mode, bool energy, bool store_f) {
    ForceArgs a = make_force_args(h);
    const int nb = nblocks(a.n);
    const int sf = store_f ? 1 : 0;
    const EamTab &t = h->eam;
    cudaStream_t s = h->stream;
    if (h->p.force_variant == MD_FORCE_PAIRED) {
        const PairArgs p = make_pair_args(h);
        const int pb = pair_grid_blocks(h, kEamPairBlock);
        const bool fe = (t.nphi == 7 && t.npsi == 1);
#define MDG_EAMP(M, E)                                                                  \
    do {                                                                                \
        if (fe) eam_force_pair<M, E, 7, 1><<<pb, kEamPairBlock, 0, s>>>(a, p, t, sf);   \
        else eam_force_pair<M, E, 0, 0><<<pb, kEamPairBlock, 0, s>>>(a, p, t, sf);      \
    } while (0)
        switch (mode) {
            case FM_STORE: if (energy) MDG_EAMP(FM_STORE, true); else MDG_EAMP(FM_STORE, false); break;
            case FM_FUSED_FULL: if (energy) MDG_EAMP(FM_FUSED_FULL, true); else MDG_EAMP(FM_FUSED_FULL, false); break;
            default: if (energy) MDG_EAMP(FM_FUSED_HALF, true); else MDG_EAMP(FM_FUSED_HALF, false); break;
        }
#undef MDG_EAMP
        return cudaGetLastError();
    }
    if (h->p.precision == MD_MIXED) {
        // the knot counts of the Fe-like table get compile-time loops
        const bool fe = (t.nphi == 7 && t.npsi == 1);
#define MDG_EAM(M, E)                                                                   \
    do {                                                                                \
        if (fe) eam_force_mixed<M, E, 7, 1><<<nb, kBlock, 0, s>>>(a, t, sf);            \
        else eam_force_mixed<M, E, 0, 0><<<nb, kBlock, 0, s>>>(a, t, sf);               \
    } while (0)
        switch (mode) {
            case FM_STORE: if (energy) MDG_EAM(FM_STORE, true); else MDG_EAM(FM_STORE, false); break;
            case FM_FUSED_FULL: if (energy) MDG_EAM(FM_FUSED_FULL, true); else MDG_EAM(FM_FUSED_FULL, false); break;
            default: if (energy) MDG_EAM(FM_FUSED_HALF, true); else MDG_EAM(FM_FUSED_HALF, false); break;
        }
#undef MDG_EAM
    } else {
        switch (mode) {
            case FM_STORE: if (energy) eam_force_fp64<FM_STORE, true><<<nb, kBlock, 0, s>>>(a, t, sf); else eam_force_fp64<FM_STORE, false><<<nb, kBlock, 0, s>>>(a, t, sf); break;
            case FM_FUSED_FULL: if (energy) eam_force_fp64<FM_FUSED_FULL, true><<<nb, kBlock, 0, s>>>(a, t, sf); else eam_force_fp64<FM_FUSED_FULL, false><<<nb, kBlock, 0, s>>>(a, t, sf); break;
            default: if (energy) eam_force_fp64<FM_FUSED_HALF, true><<<nb, kBlock, 0, s>>>(a, t, sf); else eam_force_fp64<FM_FUSED_HALF, false><<<nb, kBlock, 0, s>>>(a, t, sf); break;
        }
    }
    return cudaGetLastError();
}

}  // namespace mdg
