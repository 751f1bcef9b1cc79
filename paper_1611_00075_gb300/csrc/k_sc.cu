// k_sc.cu -- Sutton-Chen many-body forces in the paper's three steps
// (Sec. 3.1): a pair pass for the localization function rho_i (Eq. 2), an
// atom pass for the embedding function, and a pair pass for the pair term
// and the forces.
//
// Sutton-Chen instance of Eq. 1:
//   Phi(r) = eps (a/r)^n,  psi(r) = (a/r)^m,  F(rho) = -eps c sqrt(rho),
//   truncated (no shift) at r_c.  Differentiating U gives the force on i
//   f_i = -sum_j [Phi'(r) + (F'(rho_i) + F'(rho_j)) psi'(r)] (r_i - r_j) / r
//       = -sum_j (n Phi + m (F'_i + F'_j) psi) / r^2 * d,   d = r_j - r_i
//   since Phi' = -n Phi / r and psi' = -m psi / r.
//
// The second step (atom loop: F(rho_i), F'(rho_i)) only needs rho_i, so it
// runs as the epilogue of the density pass in the thread that owns atom i;
// sc_embed_deriv_*() below is that step.  The third step needs F'_j per pair:
// the mixed path's density epilogue writes (x, y, z, F'(rho)) of each atom
// into one float4, so the force pass gathers position and F'_j in one load.
//
// Precision as for Lennard-Jones: MIXED computes pair terms in float32 and
// sums rho and the forces in float64 over float32 chunks; F'(rho) feeds the
// float32 pair terms as float32.  The embedding energy is float64.
#include "k_common.cuh"
#include "k_pair.cuh"

namespace mdg {

namespace {

template <int K>
__device__ __forceinline__ float cpow(float x) {
    float r = 1.f, b = x;
    int k = K;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        if (k & 1) r *= b;
        k >>= 1;
        if (k) b *= b;
    }
    return r;
}
__device__ __forceinline__ float rpow(float x, int k) {
    float r = 1.f;
    while (k) {
        if (k & 1) r *= x;
        k >>= 1;
        x *= x;
    }
    return r;
}
__device__ __forceinline__ double rpowd(double x, int k) {
    double r = 1.0;
    while (k) {
        if (k & 1) r *= x;
        k >>= 1;
        x *= x;
    }
    return r;
}

// (a/r)^K from s = (a/r)^2 and ar = a/r (ar only used for odd K).
template <int K>
__device__ __forceinline__ float ar_pow(float s, float ar) {
    if (K % 2 == 0) return cpow<K / 2>(s);
    return cpow<K / 2>(s) * ar;
}

// The atom step of Sec. 3.1 for Sutton-Chen: F'(rho) = -eps c / (2 sqrt(rho)).
__device__ __forceinline__ float sc_embed_deriv_f32(double rho, float ec) {
    return rho > 0.0 ? -0.5f * ec * rsqrtf((float)rho) : 0.f;
}
__device__ __forceinline__ double sc_embed_deriv_f64(double rho, double ec) {
    return rho > 0.0 ? -0.5 * ec / sqrt(rho) : 0.0;
}

// Both mixed passes run 256-thread blocks at up to 64 registers (4 per SM),
// measured 2 % faster than at 48.
template <int ME>
__global__ void __launch_bounds__(kBlock, 4) sc_density_mixed(ForceArgs a) {
    __shared__ ShiftTab sh;
    load_shifts_f32(a.g, &sh);
    __syncthreads();
    if (a.ds->status != 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const float4 qi = a.xq[i];
    const int nq = (min(a.ncount[i], a.cap) + 3) >> 2;
    const uint4 *lq = reinterpret_cast<const uint4 *>(a.nlist + list_group(i, a.cap)) + (i & 31);
    const float rc2 = a.fc.rc2f, af = a.fc.sc_af, a2 = af * af;
    const int m = a.fc.sc_m;
    double R = 0.0;
    // list quads stream through once (evict-first), one quad loaded ahead
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
            if (r2 < rc2) {
                const float s = a2 * __fdividef(1.0f, r2);
                float psi;
                if (ME > 0) psi = ar_pow<ME>(s, (ME & 1) ? af * rsqrtf(r2) : 0.f);
                else psi = (m & 1) ? rpow(s, m / 2) * af * rsqrtf(r2) : rpow(s, m / 2);
                r += psi;
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
        R += (double)r;
    }
    a.rho[i] = R;
    const float dF = sc_embed_deriv_f32(R, a.fc.sc_ecf);
    a.dF32[i] = dF;
    // the force pass gathers F'(rho_j) together with the position of j
    a.xqf[i] = make_float4(qi.x, qi.y, qi.z, dF);
}

__global__ void __launch_bounds__(kBlock) sc_density_fp64(ForceArgs a) {
    __shared__ double3 sh[kStencil];
    if (threadIdx.x < kStencil) {
        int s = threadIdx.x;
        int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        sh[s] = make_double3(dx * a.g.w[0], dy * a.g.w[1], dz * a.g.w[2]);
    }
    __syncthreads();
    if (a.ds->status != 0) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double4 ri = a.xr[i];
    const int cnt = min(a.ncount[i], a.cap);
    const double rc2 = a.fc.rc2, A = a.fc.sc_a;
    const int m = a.fc.sc_m;
    double R = 0.0;
    for (int k = 0; k < cnt; ++k) {
        const uint32_t ent = __ldg(a.nlist + list_idx(i, k, a.cap));
        const double4 rj = a.xr[ent & kIndexMask];
        const double3 sd = sh[ent >> kIndexBits];
        const double ex = (rj.x - ri.x) + sd.x;
        const double ey = (rj.y - ri.y) + sd.y;
        const double ez = (rj.z - ri.z) + sd.z;
        const double r2 = ex * ex + ey * ey + ez * ez;
        if (r2 < rc2) R += rpowd(A / sqrt(r2), m);
    }
    a.rho[i] = R;
    const double d = sc_embed_deriv_f64(R, a.fc.sc_ec);
    a.dF64[i] = d;
    a.dF32[i] = (float)d;
}

template <int MODE, bool ENERGY, int NE, int ME>
__global__ void __launch_bounds__(kBlock, 4) sc_force_mixed(ForceArgs a, int store_f) {
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
    const float rc2 = a.fc.rc2f, af = a.fc.sc_af, a2 = af * af, epsf = a.fc.sc_epsf;
    const float inv_a2 = 1.0f / a2;
    const int nexp = a.fc.sc_n, mexp = a.fc.sc_m;
    const float nf = (float)(NE > 0 ? NE : nexp), mf = (float)(ME > 0 ? ME : mexp);
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
                // with an odd exponent a/r comes from one reciprocal square
                // root, and (a/r)^2 and 1/r^2 from it without a reciprocal
                const bool odd = (NE > 0) ? ((NE | ME) & 1) : ((nexp | mexp) & 1);
                const float ar = odd ? af * rsqrtf(r2) : 0.f;
                const float r2i = odd ? ar * ar * inv_a2 : __fdividef(1.0f, r2);
                const float s = odd ? ar * ar : a2 * r2i;
                float Phi, psi;
                if (NE > 0) {
                    Phi = epsf * ar_pow<NE>(s, ar);
                    psi = ar_pow<ME>(s, ar);
                } else {
                    Phi = epsf * ((nexp & 1) ? rpow(s, nexp / 2) * ar : rpow(s, nexp / 2));
                    psi = (mexp & 1) ? rpow(s, mexp / 2) * ar : rpow(s, mexp / 2);
                }
                const float fs = (nf * Phi + mf * (dFi + qj.w) * psi) * r2i;
                fx -= fs * ex;
                fy -= fs * ey;
                fz -= fs * ez;
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
        a.e_atom[i] = 0.5 * E - a.fc.sc_ec * sqrt(a.rho[i]);
        count_pairs(a.ds, npair);
    }
    // the float32 position's w word holds the original id
    if (MODE != FM_STORE)
        vv_epilogue<MODE>(a, i, Fx, Fy, Fz, reinterpret_cast<const float *>(a.xq)[4 * (size_t)i + 3]);
}

template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(kBlock) sc_force_fp64(ForceArgs a, int store_f) {
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
    const double dFi = a.dF64[i];
    const int cnt = min(a.ncount[i], a.cap);
    const double rc2 = a.fc.rc2, A = a.fc.sc_a, eps = a.fc.sc_eps;
    const int nexp = a.fc.sc_n, mexp = a.fc.sc_m;
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
            const double ar = A / sqrt(r2);
            const double Phi = eps * rpowd(ar, nexp);
            const double psi = rpowd(ar, mexp);
            const double fs = (nexp * Phi + mexp * (dFi + a.dF64[j]) * psi) / r2;
            fx -= fs * ex;
            fy -= fs * ey;
            fz -= fs * ez;
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
        a.e_atom[i] = 0.5 * e - a.fc.sc_ec * sqrt(a.rho[i]);
        count_pairs(a.ds, npair);
    }
    if (MODE != FM_STORE) {
        const float4 qi = a.xq[i];
        vv_epilogue<MODE>(a, i, fx, fy, fz, qi.w);
    }
}

// ---- two atoms per thread (MD_FORCE_PAIRED) ---------------------------------
//
// The slot layout of k_pair.cu: slot s holds sorted atoms i0 and i0 + 1 of
// one cell (one atom when bit 31 of its entry is set) and the union of their
// lists.  Both passes evaluate the slot's own pair once, then both atoms
// against each list entry with packed float32 pairs (lane x: i0, lane y:
// i1), so that one gathered neighbour serves two pair evaluations.  Sums run
// in float32 over chunks of kChunkQ quads and in float64 across chunks, as in
// the per-atom passes: a crystal's many-body forces cancel strongly.
constexpr int kScPairBlock = 128;

// (a/r)^K lane by lane for run-time exponents (s = (a/r)^2, ar = a/r)
__device__ __forceinline__ float2 ar_pow_rt(float2 s, float2 ar, int k) {
    float2 r = make_float2(rpow(s.x, k / 2), rpow(s.y, k / 2));
    if (k & 1) r = mul2(r, ar);
    return r;
}

template <int ME>
__global__ void __launch_bounds__(kScPairBlock, 8) sc_density_pair(ForceArgs a, PairArgs p) {
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
    const float rc2 = a.fc.rc2f, af = a.fc.sc_af, a2 = af * af;
    const int m = a.fc.sc_m;
    float2 r = dup2(0.f);
    {
        // the slot's own pair adds to both densities
        const float ex = q1.x - q0.x, ey = q1.y - q0.y, ez = q1.z - q0.z;
        const float r2 = ex * ex + ey * ey + ez * ez;
        if (r2 < rc2) {
            const float sp = a2 * __fdividef(1.0f, r2);
            const float psi = ME > 0 ? ar_pow<ME>(sp, (ME & 1) ? af * rsqrtf(r2) : 0.f)
                                     : ((m & 1) ? rpow(sp, m / 2) * af * rsqrtf(r2)
                                                : rpow(sp, m / 2));
            r = dup2(psi);
        }
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
        const float2 sp = mul2(dup2(a2), make_float2(__fdividef(1.0f, r2.x), __fdividef(1.0f, r2.y)));
        float2 psi;
        if (ME == 6) {
            psi = mul2(mul2(sp, sp), sp);
        } else {
            const float2 ar = (m & 1) ? make_float2(af * rsqrtf(r2.x), af * rsqrtf(r2.y)) : dup2(0.f);
            psi = ar_pow_rt(sp, ar, m);
        }
        psi.x = r2.x < rc2 ? psi.x : 0.f;
        psi.y = r2.y < rc2 ? psi.y : 0.f;
        r = add2(r, psi);
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
    const float d0 = sc_embed_deriv_f32(R0, a.fc.sc_ecf);
    a.rho[i0] = R0;
    a.dF32[i0] = d0;
    a.xqf[i0] = make_float4(q0.x, q0.y, q0.z, d0);
    if (two) {
        const float d1 = sc_embed_deriv_f32(R1, a.fc.sc_ecf);
        a.rho[i0 + 1] = R1;
        a.dF32[i0 + 1] = d1;
        a.xqf[i0 + 1] = make_float4(q1.x, q1.y, q1.z, d1);
    }
}

template <int MODE, bool ENERGY>
__device__ __forceinline__ void sc_pair_atom_out(const ForceArgs &a, int i, double Fx, double Fy,
                                                 double Fz, double E, unsigned np, int store_f) {
    const size_t n = (size_t)a.n;
    if (MODE == FM_STORE || store_f) {
        a.f[i] = Fx;
        a.f[n + i] = Fy;
        a.f[2 * n + i] = Fz;
    }
    if (ENERGY) {
        a.e_atom[i] = 0.5 * E - a.fc.sc_ec * sqrt(a.rho[i]);
        count_pairs(a.ds, np);
    }
    // the float32 position's w word holds the original id
    if (MODE != FM_STORE)
        vv_epilogue<MODE>(a, i, Fx, Fy, Fz, reinterpret_cast<const float *>(a.xq)[4 * (size_t)i + 3]);
}

template <int MODE, bool ENERGY, int NE, int ME>
__global__ void __launch_bounds__(kScPairBlock, 7) sc_force_pair(ForceArgs a, PairArgs p,
                                                                 int store_f) {
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
    const float rc2 = a.fc.rc2f, af = a.fc.sc_af, a2 = af * af, epsf = a.fc.sc_epsf;
    const float inv_a2 = 1.0f / a2;
    const int nexp = a.fc.sc_n, mexp = a.fc.sc_m;
    const float nf = (float)(NE > 0 ? NE : nexp), mf = (float)(ME > 0 ? ME : mexp);
    const bool odd = (NE > 0) ? ((NE | ME) & 1) : ((nexp | mexp) & 1);
    float2 fx = dup2(0.f), fy = dup2(0.f), fz = dup2(0.f), en = dup2(0.f);
    unsigned np0 = 0, np1 = 0;
    {
        // the slot's own pair once: e = x_1 - x_0, f_0 -= fs e, f_1 += fs e
        const float ex = q1.x - q0.x, ey = q1.y - q0.y, ez = q1.z - q0.z;
        const float r2 = ex * ex + ey * ey + ez * ez;
        if (r2 < rc2) {
            const float r2i = __fdividef(1.0f, r2);
            const float sp = a2 * r2i;
            const float ar = odd ? af * rsqrtf(r2) : 0.f;
            float Phi, psi;
            if (NE > 0) {
                Phi = epsf * ar_pow<NE>(sp, ar);
                psi = ar_pow<ME>(sp, ar);
            } else {
                Phi = epsf * ((nexp & 1) ? rpow(sp, nexp / 2) * ar : rpow(sp, nexp / 2));
                psi = (mexp & 1) ? rpow(sp, mexp / 2) * ar : rpow(sp, mexp / 2);
            }
            const float fs = (nf * Phi + mf * (q0.w + q1.w) * psi) * r2i;
            fx = make_float2(-fs * ex, fs * ex);
            fy = make_float2(-fs * ey, fs * ey);
            fz = make_float2(-fs * ez, fs * ez);
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
    // d = x_j - x_i per atom; f_i -= fs d with fs = (n Phi + m (F'_i + F'_j) psi) / r^2
    auto pair = [&](uint32_t ent) {
        const float4 qj = __ldg(a.xqf + (ent & kIndexMask));  // position, F'(rho_j)
        const uint32_t st = ent >> kIndexBits;
        const float tx = qj.x + sh.x[st], ty = qj.y + sh.y[st], tz = qj.z + sh.z[st];
        const float2 dx = add2(dup2(tx), nqx), dy = add2(dup2(ty), nqy), dz = add2(dup2(tz), nqz);
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        // with an odd exponent a/r comes from one reciprocal square root,
        // and (a/r)^2 and 1/r^2 from it without a reciprocal
        float2 ar, sp, r2i;
        if (odd) {
            ar = mul2(dup2(af), make_float2(rsqrtf(r2.x), rsqrtf(r2.y)));
            sp = mul2(ar, ar);
            r2i = mul2(sp, dup2(inv_a2));
        } else {
            ar = dup2(0.f);
            r2i = make_float2(__fdividef(1.0f, r2.x), __fdividef(1.0f, r2.y));
            sp = mul2(dup2(a2), r2i);
        }
        float2 Phi, psi;
        if (NE == 9 && ME == 6) {
            const float2 s2 = mul2(sp, sp);
            psi = mul2(s2, sp);
            Phi = mul2(mul2(mul2(s2, s2), ar), dup2(epsf));
        } else {
            Phi = mul2(dup2(epsf), ar_pow_rt(sp, ar, NE > 0 ? NE : nexp));
            psi = ar_pow_rt(sp, ar, ME > 0 ? ME : mexp);
        }
        const float2 t = add2(dFi, dup2(qj.w));
        float2 nfs = mul2(fma2(mul2(dup2(-mf), t), psi, mul2(dup2(-nf), Phi)), r2i);
        const bool in0 = r2.x < rc2, in1 = r2.y < rc2;
        nfs.x = in0 ? nfs.x : 0.f;
        nfs.y = in1 ? nfs.y : 0.f;
        fx = fma2(nfs, dx, fx);
        fy = fma2(nfs, dy, fy);
        fz = fma2(nfs, dz, fz);
        if (ENERGY) {
            en.x += in0 ? Phi.x : 0.f;
            en.y += in1 ? Phi.y : 0.f;
            np0 += in0 ? 1u : 0u;
            np1 += in1 ? 1u : 0u;
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
    sc_pair_atom_out<MODE, ENERGY>(a, i0, F0x, F0y, F0z, E0, np0, store_f);
    if (two) sc_pair_atom_out<MODE, ENERGY>(a, i0 + 1, F1x, F1y, F1z, E1, np1, store_f);
}

}  // namespace

cudaError_t launch_sc_density(md_system *h) {
    ForceArgs a = make_force_args(h);
    const int nb = nblocks(a.n);
    if (h->p.force_variant == MD_FORCE_PAIRED) {
        const PairArgs p = make_pair_args(h);
        if (a.fc.sc_m == 6) sc_density_pair<6><<<pair_grid_blocks(h, kScPairBlock), kScPairBlock, 0, h->stream>>>(a, p);
        else sc_density_pair<0><<<pair_grid_blocks(h, kScPairBlock), kScPairBlock, 0, h->stream>>>(a, p);
        return cudaGetLastError();
    }
    if (h->p.precision == MD_MIXED) {
        if (a.fc.sc_m == 6) sc_density_mixed<6><<<nb, kBlock, 0, h->stream>>>(a);
        else sc_density_mixed<0><<<nb, kBlock, 0, h->stream>>>(a);
    } else {
        sc_density_fp64<<<nb, kBlock, 0, h->stream>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_sc_force(md_system *h, int mode, bool energy, bool store_f) {
    ForceArgs a = make_force_args(h);
    const int nb = nblocks(a.n);
    const int sf = store_f ? 1 : 0;
    cudaStream_t s = h->stream;
    if (h->p.force_variant == MD_FORCE_PAIRED) {
        const PairArgs p = make_pair_args(h);
        const int pb = pair_grid_blocks(h, kScPairBlock);
        const bool cu = (a.fc.sc_n == 9 && a.fc.sc_m == 6);
#define MDG_SCP(M, E)                                                                   \
    do {                                                                                \
        if (cu) sc_force_pair<M, E, 9, 6><<<pb, kScPairBlock, 0, s>>>(a, p, sf);        \
        else sc_force_pair<M, E, 0, 0><<<pb, kScPairBlock, 0, s>>>(a, p, sf);           \
    } while (0)
        switch (mode) {
            case FM_STORE: if (energy) MDG_SCP(FM_STORE, true); else MDG_SCP(FM_STORE, false); break;
            case FM_FUSED_FULL: if (energy) MDG_SCP(FM_FUSED_FULL, true); else MDG_SCP(FM_FUSED_FULL, false); break;
            default: if (energy) MDG_SCP(FM_FUSED_HALF, true); else MDG_SCP(FM_FUSED_HALF, false); break;
        }
#undef MDG_SCP
        return cudaGetLastError();
    }
    if (h->p.precision == MD_MIXED) {
        const bool cu = (a.fc.sc_n == 9 && a.fc.sc_m == 6);
#define MDG_SC(M, E)                                                                    \
    do {                                                                                \
        if (cu) sc_force_mixed<M, E, 9, 6><<<nb, kBlock, 0, s>>>(a, sf);                \
        else sc_force_mixed<M, E, 0, 0><<<nb, kBlock, 0, s>>>(a, sf);                   \
    } while (0)
        switch (mode) {
            case FM_STORE: if (energy) MDG_SC(FM_STORE, true); else MDG_SC(FM_STORE, false); break;
            case FM_FUSED_FULL: if (energy) MDG_SC(FM_FUSED_FULL, true); else MDG_SC(FM_FUSED_FULL, false); break;
            default: if (energy) MDG_SC(FM_FUSED_HALF, true); else MDG_SC(FM_FUSED_HALF, false); break;
        }
#undef MDG_SC
    } else {
        switch (mode) {
            case FM_STORE: if (energy) sc_force_fp64<FM_STORE, true><<<nb, kBlock, 0, s>>>(a, sf); else sc_force_fp64<FM_STORE, false><<<nb, kBlock, 0, s>>>(a, sf); break;
            case FM_FUSED_FULL: if (energy) sc_force_fp64<FM_FUSED_FULL, true><<<nb, kBlock, 0, s>>>(a, sf); else sc_force_fp64<FM_FUSED_FULL, false><<<nb, kBlock, 0, s>>>(a, sf); break;
            default: if (energy) sc_force_fp64<FM_FUSED_HALF, true><<<nb, kBlock, 0, s>>>(a, sf); else sc_force_fp64<FM_FUSED_HALF, false><<<nb, kBlock, 0, s>>>(a, sf); break;
        }
    }
    return cudaGetLastError();
}

}  // namespace mdg
