// k_pair_typed.cu -- two home atoms per thread (MD_FORCE_PAIRED) for the
// multi-element Lennard-Jones systems (Sec. 2.2's parameter reload, the
// Alloy and Layer configurations of Sec. 3.1).
//
// The slots and union lists of k_pair.cu, unchanged: a slot's two atoms may
// be of different species.  Each thread keeps the parameter rows of both of
// its atoms' species in registers (sigma^2 and 48 eps, with the energy 4 eps
// and the shift at r_c for energies); per list entry it reads the
// neighbour's species from the position word it gathers anyway and picks
// the two atoms' parameters from their rows, so each lane of the packed
// float32 pair arithmetic carries its own pair's parameters.  Sums: float32
// over the whole list, as for the one-species slot kernel; the
// velocity-Verlet epilogue uses each atom's species mass.
#include "k_pair.cuh"

namespace mdg {

namespace {

constexpr int kTypedPairBlock = 128;

// element t of a row of NT values held in registers
template <int NT>
__device__ __forceinline__ float row_at(const float *row, int t) {
    if (NT == 1) return row[0];
    if (NT == 2) return t ? row[1] : row[0];
    if (NT == 3) return t == 0 ? row[0] : (t == 1 ? row[1] : row[2]);
    return t < 2 ? (t == 0 ? row[0] : row[1]) : (t == 2 ? row[2] : row[3]);
}

// row ti of an NT x NT parameter table into registers
template <int NT>
__device__ __forceinline__ void row_of(const float *tab, int ti, float *row) {
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        float v = tab[k];
#pragma unroll
        for (int r = 1; r < NT; ++r) v = (ti == r) ? tab[r * NT + k] : v;
        row[k] = v;
    }
}

template <int MODE, bool ENERGY>
__device__ __forceinline__ void typed_atom_out(const ForceArgs &a, int i, double Fx, double Fy,
                                               double Fz, double E, unsigned np, float qw,
                                               int store_f) {
    const size_t n = (size_t)a.n;
    if (MODE == FM_STORE || store_f) {
        a.f[i] = Fx;
        a.f[n + i] = Fy;
        a.f[2 * n + i] = Fz;
    }
    if (ENERGY) {
        a.e_atom[i] = 0.5 * E;
        count_pairs(a.ds, np);
    }
    if (MODE != FM_STORE) vv_epilogue<MODE, true>(a, i, Fx, Fy, Fz, qw);
}

template <int MODE, bool ENERGY, int NT>
__global__ void __launch_bounds__(kTypedPairBlock, 8)
lj_typed_pair_kernel(ForceArgs a, PairArgs p, TypeTab tt, int store_f) {
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
    const float4 q0 = a.xq[i0];
    // a one-atom slot puts its second atom at the dummy's distance
    const float4 q1 = two ? a.xq[i0 + 1] : make_float4(3.0e18f, 3.0e18f, 3.0e18f, 0.f);
    const int t0 = species_of(__float_as_uint(q0.w));
    const int t1 = two ? species_of(__float_as_uint(q1.w)) : t0;
    float s2a[NT], s2b[NT], e48a[NT], e48b[NT];
    row_of<NT>(tt.s2, t0, s2a);
    row_of<NT>(tt.s2, t1, s2b);
    row_of<NT>(tt.e48, t0, e48a);
    row_of<NT>(tt.e48, t1, e48b);
    float e4a[ENERGY ? NT : 1], e4b[ENERGY ? NT : 1], sha[ENERGY ? NT : 1], shb[ENERGY ? NT : 1];
    if (ENERGY) {
        row_of<NT>(tt.e4, t0, e4a);
        row_of<NT>(tt.e4, t1, e4b);
        row_of<NT>(tt.sh, t0, sha);
        row_of<NT>(tt.sh, t1, shb);
    }
    const float rc2 = a.fc.rc2f;
    float2 fx = dup2(0.f), fy = dup2(0.f), fz = dup2(0.f), en = dup2(0.f);
    unsigned np0 = 0, np1 = 0;
    {
        // the slot's own pair once: f_0 -= fs e, f_1 += fs e with e = x_1 - x_0
        const float ex = q1.x - q0.x, ey = q1.y - q0.y, ez = q1.z - q0.z;
        const float r2 = ex * ex + ey * ey + ez * ez;
        if (r2 < rc2) {
            const float r2i = __fdividef(1.0f, r2);
            float s6 = row_at<NT>(s2a, t1) * r2i;
            s6 = s6 * s6 * s6;
            const float fs = row_at<NT>(e48a, t1) * r2i * s6 * (s6 - 0.5f);
            fx = make_float2(-fs * ex, fs * ex);
            fy = make_float2(-fs * ey, fs * ey);
            fz = make_float2(-fs * ez, fs * ez);
            if (ENERGY) {
                en = dup2(row_at<NT>(e4a, t1) * s6 * (s6 - 1.0f) - row_at<NT>(sha, t1));
                np0 = np1 = 1;
            }
        }
    }
    const float2 nqx = make_float2(-q0.x, -q1.x), nqy = make_float2(-q0.y, -q1.y),
                 nqz = make_float2(-q0.z, -q1.z);
    const int nq = (min(p.count[s], p.cap) + 3) >> 2;
    const uint4 *lq = reinterpret_cast<const uint4 *>(p.list + list_group(s, p.cap)) + (s & 31);
    // -fs = 48 eps r2i s6 (1/2 - s6), s6 = (sigma^2 r2i)^3, each lane with its
    // own pair's sigma and eps
    auto pair = [&](uint32_t ent) {
        const float4 qj = __ldg(a.xq + (ent & kIndexMask));
        const uint32_t st = ent >> kIndexBits;
        const int tj = species_of(__float_as_uint(qj.w));
        const float tx = qj.x + sh.x[st], ty = qj.y + sh.y[st], tz = qj.z + sh.z[st];
        const float2 dx = add2(dup2(tx), nqx), dy = add2(dup2(ty), nqy), dz = add2(dup2(tz), nqz);
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float2 r2i = make_float2(__fdividef(1.0f, r2.x), __fdividef(1.0f, r2.y));
        const float2 s2 = mul2(make_float2(row_at<NT>(s2a, tj), row_at<NT>(s2b, tj)), r2i);
        const float2 s6 = mul2(mul2(s2, s2), s2);
        const float2 e48 = make_float2(row_at<NT>(e48a, tj), row_at<NT>(e48b, tj));
        float2 nfs = mul2(mul2(mul2(e48, fma2(s6, dup2(-1.0f), dup2(0.5f))), s6), r2i);
        const bool in0 = r2.x < rc2, in1 = r2.y < rc2;
        nfs.x = in0 ? nfs.x : 0.f;
        nfs.y = in1 ? nfs.y : 0.f;
        fx = fma2(nfs, dx, fx);
        fy = fma2(nfs, dy, fy);
        fz = fma2(nfs, dz, fz);
        if (ENERGY) {
            float2 u = add2(mul2(mul2(make_float2(row_at<NT>(e4a, tj), row_at<NT>(e4b, tj)),
                                      add2(s6, dup2(-1.0f))), s6),
                            make_float2(-row_at<NT>(sha, tj), -row_at<NT>(shb, tj)));
            u.x = in0 ? u.x : 0.f;
            u.y = in1 ? u.y : 0.f;
            en = add2(en, u);
            np0 += in0 ? 1u : 0u;
            np1 += in1 ? 1u : 0u;
        }
    };
    uint4 nxt = nq > 0 ? __ldcs(lq) : make_uint4(0u, 0u, 0u, 0u);
    for (int q = 0; q < nq; ++q) {
        const uint4 e4 = nxt;
        if (q + 1 < nq) nxt = __ldcs(lq + (size_t)(q + 1) * 32);
        pair(e4.x);
        pair(e4.y);
        pair(e4.z);
        pair(e4.w);
    }
    // the position words (id and species bits) are read again here rather
    // than held through the loop
    typed_atom_out<MODE, ENERGY>(a, i0, fx.x, fy.x, fz.x, en.x, np0, a.xq[i0].w, store_f);
    if (two)
        typed_atom_out<MODE, ENERGY>(a, i0 + 1, fx.y, fy.y, fz.y, en.y, np1, a.xq[i0 + 1].w,
                                     store_f);
}

template <int NT>
cudaError_t launch_nt(md_system *h, int mode, bool energy, bool store_f) {
    const ForceArgs a = make_force_args(h);
    const PairArgs p = make_pair_args(h);
    const TypeTab &tt = h->types;
    const int blocks = pair_grid_blocks(h, kTypedPairBlock);
    const int sf = store_f ? 1 : 0;
    cudaStream_t s = h->stream;
#define MDG_TP(M)                                                                         \
    do {                                                                                  \
        if (energy) lj_typed_pair_kernel<M, true, NT><<<blocks, kTypedPairBlock, 0, s>>>(a, p, tt, sf); \
        else lj_typed_pair_kernel<M, false, NT><<<blocks, kTypedPairBlock, 0, s>>>(a, p, tt, sf);      \
    } while (0)
    switch (mode) {
        case FM_STORE: MDG_TP(FM_STORE); break;
        case FM_FUSED_FULL: MDG_TP(FM_FUSED_FULL); break;
        default: MDG_TP(FM_FUSED_HALF); break;
    }
#undef MDG_TP
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pair_typed_forces(md_system *h, int mode, bool energy, bool store_f) {
    switch (h->fc.ntypes) {
        case 1: return launch_nt<1>(h, mode, energy, store_f);
        case 2: return launch_nt<2>(h, mode, energy, store_f);
        case 3: return launch_nt<3>(h, mode, energy, store_f);
        default: return launch_nt<4>(h, mode, energy, store_f);
    }
}

}  // namespace mdg
