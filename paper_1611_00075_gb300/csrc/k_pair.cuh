// k_pair.cuh -- the per-slot job of the two-atoms-per-thread force pass
// (MD_FORCE_PAIRED), shared by its grid kernel (k_pair.cu) and the
// persistent kernel of the schedulers (k_lj.cu).  The layout, the list and
// the arithmetic are described at the top of k_pair.cu.
#pragma once

#include "k_common.cuh"

namespace mdg {

constexpr uint32_t kSingle = 0x80000000u;  // slot_atom: a one-atom slot

struct PairArgs {
    const int32_t *slot_start;   // ncells + 1 (slot_start[ncells] = slots)
    const uint32_t *slot_atom;
    const uint32_t *list;
    const int32_t *count;
    int cap, ncells;
};

// The slot tables and union lists of a handle, for the kernels.
inline PairArgs make_pair_args(const md_system *h) {
    PairArgs p;
    p.slot_start = h->ps_start;
    p.slot_atom = h->ps_atom;
    p.list = h->ps_list;
    p.count = h->ps_count;
    p.cap = h->ps_cap;
    p.ncells = h->g.ncells;
    return p;
}

// Blocks of `block` threads that cover every slot a binning can make.
inline int pair_grid_blocks(const md_system *h, int block) {
    return (int)((pair_slots_max(h->n, h->g.ncells) + block - 1) / block);
}

// Lennard-Jones pair term in float32 for the pair vector e = x_j - x_i:
// f_i -= fs * e; with ENERGY the shifted pair energy is added to `en`.
template <bool ENERGY>
__device__ __forceinline__ void lj_term(const ForceConsts &fc, float ex, float ey, float ez,
                                        float r2, float &fx, float &fy, float &fz, float &en,
                                        unsigned &np) {
    const float r2i = __fdividef(1.0f, r2);
    float s6 = fc.sig2f * r2i;
    s6 = s6 * s6 * s6;
    const float fs = fc.eps48f * r2i * s6 * (s6 - 0.5f);
    fx -= fs * ex;
    fy -= fs * ey;
    fz -= fs * ez;
    if (ENERGY) {
        en += fc.eps4f * s6 * (s6 - 1.0f) - fc.shiftf;
        ++np;
    }
}

// Stores, energies and the velocity-Verlet epilogue of one atom of a slot.
template <int MODE, bool ENERGY>
__device__ __forceinline__ void pair_atom_out(const ForceArgs &a, int i, double Fx, double Fy,
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
    if (MODE != FM_STORE) vv_epilogue<MODE>(a, i, Fx, Fy, Fz, qw);
}

// Packed float32 pairs (add/mul/fma.rn.f32x2, sm_100 and later): lane .x
// carries the slot's first atom, .y its second, so each instruction of the
// pair arithmetic serves both atoms.
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// MULTI (a batch of boxes, the block's boxes not all in shared memory): the
// stencil shifts come from the slot's box's row of the global R x 27 table.
template <int MODE, bool ENERGY, bool MULTI = false>
__device__ __forceinline__ void lj_pair_slot(const ForceArgs &a, const PairArgs &p,
                                             const ShiftTab *sh, int s, int store_f) {
    const uint32_t sa = p.slot_atom[s];
    const int i0 = (int)(sa & ~kSingle);
    const float4 *shr = MULTI ? a.shifts32 + kStencil * (int)a.rep[i0] : nullptr;
    const bool two = !(sa & kSingle);
    const float4 q0 = a.xq[i0];
    // a one-atom slot puts its second atom at the dummy's distance
    const float4 q1 = two ? a.xq[i0 + 1] : make_float4(3.0e18f, 3.0e18f, 3.0e18f, 0.f);
    const float rc2 = a.fc.rc2f;
    float2 fx = dup2(0.f), fy = dup2(0.f), fz = dup2(0.f), en = dup2(0.f);
    unsigned np0 = 0, np1 = 0;
    {
        // the slot's own pair, once: f_i0 -= fs e, f_i1 += fs e
        const float ex = q1.x - q0.x, ey = q1.y - q0.y, ez = q1.z - q0.z;
        const float r2 = ex * ex + ey * ey + ez * ez;
        if (r2 < rc2) {
            float gx = 0.f, gy = 0.f, gz = 0.f, e = 0.f;
            unsigned k = 0;
            lj_term<ENERGY>(a.fc, ex, ey, ez, r2, gx, gy, gz, e, k);
            fx = make_float2(gx, -gx);
            fy = make_float2(gy, -gy);
            fz = make_float2(gz, -gz);
            if (ENERGY) {
                en = dup2(e);
                np0 = np1 = 1;
            }
        }
    }
    // the slot's atoms negated, in the two lanes of each pair
    const float2 nqx = make_float2(-q0.x, -q1.x), nqy = make_float2(-q0.y, -q1.y),
                 nqz = make_float2(-q0.z, -q1.z);
    const int nq = (min(p.count[s], p.cap) + 3) >> 2;
    const uint4 *lq = reinterpret_cast<const uint4 *>(p.list + list_group(s, p.cap)) + (s & 31);
    // one gather and one stencil shift per entry, both atoms' pair terms in
    // packed instructions; -fs = r2i s6 (e48 / 2 - e48 s6) is added with one fma
    auto pair = [&](uint32_t ent) {
        const float4 qj = __ldg(a.xq + (ent & kIndexMask));
        const uint32_t st = ent >> kIndexBits;
        const float4 sf = MULTI ? __ldg(shr + st) : make_float4(sh->x[st], sh->y[st], sh->z[st], 0.f);
        const float tx = qj.x + sf.x, ty = qj.y + sf.y, tz = qj.z + sf.z;
        const float2 dx = add2(dup2(tx), nqx), dy = add2(dup2(ty), nqy), dz = add2(dup2(tz), nqz);
        const float2 r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
        const float2 r2i = make_float2(__fdividef(1.0f, r2.x), __fdividef(1.0f, r2.y));
        const float2 s2 = mul2(dup2(a.fc.sig2f), r2i);
        const float2 s6 = mul2(mul2(s2, s2), s2);
        float2 nfs = mul2(mul2(fma2(s6, dup2(-a.fc.eps48f), dup2(0.5f * a.fc.eps48f)), s6), r2i);
        const bool in0 = r2.x < rc2, in1 = r2.y < rc2;
        nfs.x = in0 ? nfs.x : 0.f;
        nfs.y = in1 ? nfs.y : 0.f;
        fx = fma2(nfs, dx, fx);
        fy = fma2(nfs, dy, fy);
        fz = fma2(nfs, dz, fz);
        if (ENERGY) {
            float2 u = add2(mul2(fma2(s6, dup2(a.fc.eps4f), dup2(-a.fc.eps4f)), s6),
                            dup2(-a.fc.shiftf));
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
    // than held through the loop: registers are the kernel's limit
    pair_atom_out<MODE, ENERGY>(a, i0, fx.x, fy.x, fz.x, en.x, np0, a.xq[i0].w, store_f);
    if (two)
        pair_atom_out<MODE, ENERGY>(a, i0 + 1, fx.y, fy.y, fz.y, en.y, np1, a.xq[i0 + 1].w, store_f);
}

}  // namespace mdg
