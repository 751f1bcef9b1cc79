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
//          64 entries is summed in float32 and the chunk sums are added in
//          float64 (the GPU form of the paper's blocked pair loop).  Entries
//          arrive four at a time (one 16-byte load), so four gathers are in
//          flight before the arithmetic that needs them.
//   FP64   everything in float64 (the plain path).
//
// Modes (ForceMode): FM_STORE writes forces; FM_FUSED_FULL also applies the
// two merged half kicks of consecutive velocity-Verlet steps (v += dt f / m)
// and the drift (x += dt v) of the atom, writing its position into the other
// buffer of a double-buffered pair; FM_FUSED_HALF applies the closing half
// kick (v += dt f / 2m).  The drift also measures the displacement since the
// last list build and raises the rebuild flag past half the skin (Sec. 3.3).
#include "k_pair.cuh"

namespace mdg {

// The whole per-atom job of the mixed path for sorted atom i: pair loop over
// its list, stores, and the velocity-Verlet epilogue.  MULTI (systems of
// several boxes) reads the cell shifts of the atom's own box from a global
// R x 27 table instead of the block's shared table.
template <int MODE, bool ENERGY, bool MULTI = false>
__device__ __forceinline__ void lj_mixed_atom(const ForceArgs &a, const ShiftTab *sh, int i,
                                              int store_f) {
    const float4 *shr = MULTI ? a.shifts32 + 27 * (int)a.rep[i] : nullptr;
    const float4 qi = a.xq[i];
    const int nq = (min(a.ncount[i], a.cap) + 3) >> 2;
    const uint4 *lq = reinterpret_cast<const uint4 *>(a.nlist + list_group(i, a.cap)) + (i & 31);
    const float rc2 = a.fc.rc2f, sig2 = a.fc.sig2f, e48 = a.fc.eps48f;
    double Fx = 0.0, Fy = 0.0, Fz = 0.0, E = 0.0;
    unsigned npair = 0;
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
    auto pair = [&](uint32_t ent) {
        const float4 qj = __ldg(a.xq + (ent & kIndexMask));
        const uint32_t st = ent >> kIndexBits;
        const float4 sf = MULTI ? __ldg(shr + st) : make_float4(sh->x[st], sh->y[st], sh->z[st], 0.f);
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
    };
    // list quads stream through once (evict-first), one quad loaded ahead;
    // the float64 sums run once per chunk, outside the inner loop
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

// Float64 cell shifts (dx, dy, dz) * w of the 27 stencil cells.
__device__ __forceinline__ void load_shifts_f64(const Grid &g, double3 *sh) {
    if (threadIdx.x < kStencil) {
        const int s = threadIdx.x;
        const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
        sh[s] = make_double3(dx * g.w[0], dy * g.w[1], dz * g.w[2]);
    }
}

// The whole per-atom job of the plain float64 path for sorted atom i.
template <int MODE, bool ENERGY>
__device__ __forceinline__ void lj_fp64_atom(const ForceArgs &a, const double3 *sh, int i,
                                             int store_f) {
    const double4 ri = a.xr[i];
    const int cnt = min(a.ncount[i], a.cap);
    const double rc2 = a.fc.rc2, sig2 = a.fc.sig2, e48 = a.fc.eps48;
    double fx = 0.0, fy = 0.0, fz = 0.0, e = 0.0;
    unsigned npair = 0;
    for (int k = 0; k < cnt; ++k) {
        const uint32_t ent = __ldg(a.nlist + list_idx(i, k, a.cap));
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

// One thread per sorted atom; the hardware block scheduler spreads the work.
// MULTI: a block's atoms are consecutive, so they belong to one or two boxes
// (more only when a box holds fewer atoms than a block); the shift tables of
// those boxes go to shared memory like a single box's, and a block that
// spans more boxes reads the global R x 27 table.
// Block shape of the grid kernel, measured on GB300: 128 threads for one
// box and 256 for batches, each at up to 56 registers (4-9 % faster than
// 256 threads at 48 registers).
template <bool MULTI>
constexpr int grid_block() { return MULTI ? 256 : 128; }

template <int MODE, bool ENERGY, bool MULTI = false>
__global__ void __launch_bounds__(grid_block<MULTI>(), MULTI ? 4 : 5)
lj_mixed_kernel(ForceArgs a, int store_f) {
    __shared__ ShiftTab sh[MULTI ? 2 : 1];
    __shared__ int s_r0, s_span;
    if (!MULTI) {
        load_shifts_f32(a.g, &sh[0]);
    } else {
        const int i0 = blockIdx.x * blockDim.x;
        const int r0 = a.rep[i0], r1 = a.rep[min(a.n, i0 + (int)blockDim.x) - 1];
        if (threadIdx.x < 2 * kStencil) {
            const int t = threadIdx.x / kStencil, st = threadIdx.x % kStencil;
            if (t <= r1 - r0) {
                const float4 v = a.shifts32[kStencil * (r0 + t) + st];
                sh[t].x[st] = v.x;
                sh[t].y[st] = v.y;
                sh[t].z[st] = v.z;
            }
        }
        if (threadIdx.x == 0) {
            s_r0 = r0;
            s_span = r1 - r0;
        }
    }
    __syncthreads();
    if (a.ds->status != 0) return;
    step_bookkeeping<MODE>(a);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    if (MULTI && s_span <= 1)
        lj_mixed_atom<MODE, ENERGY, false>(a, &sh[(int)a.rep[i] - s_r0], i, store_f);
    else
        lj_mixed_atom<MODE, ENERGY, MULTI>(a, &sh[0], i, store_f);
}

// Persistent variant: gridDim.x CTAs stay resident; each warp processes tiles
// of 32 consecutive sorted atoms (tile t = atoms 32t .. 32t+31, aligned with
// the list layout).
//   STATIC:  the cells are cut into rounds * G contiguous ranges of equal
//            (predicted) cost; CTA b owns ranges b, b + G, b + 2G, ... and its
//            warps claim their tiles from a shared counter.  A range starts at
//            the first whole tile of its first cell, so no tile is split
//            between two ranges (and no lane idles at a range boundary).  Each CTA gets the
//            same predicted total, while at any moment all CTAs work in the
//            same window of the sorted atoms, which keeps neighbour gathers
//            in L2.
//            The cells after the static ranges (the partition's last parts,
//            a fifth of the predicted cost) form a tail that warps
//            claim from a global counter, one tile at a time, once their
//            CTA's ranges are done: whichever CTA is early absorbs the error
//            of the prediction.
//   DYNAMIC: warps claim tiles from a global counter until none are left.
//   Either way the last CTA to finish resets the counter for the next launch.
// TIMING adds clock64 per tile: the tile's cycles are shared equally by its
// active atoms and added to their cells (cell_cycles), and each CTA's busy
// cycles go to cta_cycles -- the training data of the cost model.
constexpr int kClaim = 8;      // tiles claimed per atomic by the dynamic queue
constexpr int kClaimTail = 1;  // tiles claimed per atomic from the static mode's tail

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// F64: the same scheduling of the plain float64 per-atom job (the baseline
// the mixed path is measured against).  PAIRED: the items are the two-atom
// slots of MD_FORCE_PAIRED (tiles of 32 slots; sa.cell_start then holds the
// first slot of every cell) and each runs the slot job of k_pair.cuh.
// CTAs of 128 threads at up to 56 registers (9 per SM) were measured fastest:
// 1.359 ms against 1.395 ms for 256 threads at 48 registers on the 9.8 M-atom
// porous system.
constexpr int kPersistBlock = 128;
// The slot job holds twice the accumulators: its persistent kernel gets up to
// 64 registers (8 CTAs per SM) instead of spilling at 56.
constexpr int kPersistPairedCtas = 9;

template <int MODE, bool ENERGY, bool DYNAMIC, bool TIMING, bool MULTI = false, bool F64 = false,
          bool PAIRED = false>
__global__ void __launch_bounds__(kPersistBlock, F64 ? 8 : (PAIRED ? kPersistPairedCtas : 9))
lj_mixed_persist(ForceArgs a, int store_f, SchedArgs sa, PairArgs pa) {

    static_assert(!(F64 && MULTI), "batches run the mixed path");
    static_assert(!(PAIRED && (F64 || MULTI || ENERGY)), "slots: one box, mixed path, forces");
    __shared__ ShiftTab sh;
    __shared__ double3 sh64[F64 ? kStencil : 1];
    __shared__ int s_first[kSchedRounds], s_pre[kSchedRounds + 1], s_next;  // this CTA's ranges
    __shared__ int s_stop;
    if (F64) load_shifts_f64(a.g, sh64);
    else if (!MULTI) load_shifts_f32(a.g, &sh);
    // one read of the status word for the whole CTA: every thread must take the
    // same branch, since the CTA meets barriers below
    if (threadIdx.x == 0) s_stop = a.ds->status;
    __syncthreads();
    if (s_stop != 0) return;
    step_bookkeeping<MODE>(a);
    const int lane = threadIdx.x & 31;
    const int nitems = PAIRED ? pa.slot_start[pa.ncells] : a.n;
    const int ntiles = (nitems + 31) >> 5;
    long long cta_t0 = 0;
    if (TIMING) cta_t0 = clock64();
    // The claim state lives in shared memory (the CTA's ranges, and each
    // warp's queue cursor), so that no register is held through the work of
    // a tile: the slot job needs all of them.
    __shared__ int s_nlocal, s_tail0;
    __shared__ int s_wq[kPersistBlock / 32][4];  // per warp: claim end, next, range, local done
    if (threadIdx.x == 0) {
        s_nlocal = 0;
        s_tail0 = ntiles;
    }
    if (lane < 4) s_wq[threadIdx.x >> 5][lane] = (lane == 3) ? (DYNAMIC ? 1 : 0) : 0;
    if (!DYNAMIC) {
        // cyclic static partition: this CTA owns ranges b, b + G, b + 2G, ...
        // so that at any time all CTAs work in one window of the sorted atoms
        // (neighbour gathers then hit in L2).  Its warps claim the ranges'
        // tiles one at a time from a shared counter, so they finish together.
        if (threadIdx.x == 0) {
            const long long qt = (long long)sa.rounds * gridDim.x;
            s_tail0 = (sa.cell_start[sa.bounds[qt]] + 31) >> 5;
            int acc = 0;
            for (int r = 0; r < sa.rounds; ++r) {
                const long long q = (long long)r * gridDim.x + blockIdx.x;
                const int tf = (sa.cell_start[sa.bounds[q]] + 31) >> 5;
                const int te = (sa.cell_start[sa.bounds[q + 1]] + 31) >> 5;
                s_first[r] = tf;
                s_pre[r] = acc;
                acc += te - tf;
            }
            s_pre[sa.rounds] = acc;
            s_nlocal = acc;
            s_next = 0;
        }
    }
    __syncthreads();
    // next tile of this warp, or -1 when none is left; every lane computes the
    // same values, so the lanes' identical stores to the warp's cursor agree
    auto claim = [&]() -> int {
        int *wq = s_wq[threadIdx.x >> 5];
        int res = -1;
        bool done = wq[3] != 0;
        if (!done) {
            int k = 0;
            if (lane == 0) k = atomicAdd(&s_next, 1);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k < s_nlocal) {
                int r = wq[2];  // this warp's claims only grow: its range only advances
                while (k >= s_pre[r + 1]) ++r;
                res = s_first[r] + (k - s_pre[r]);
                __syncwarp();
                wq[2] = r;
            } else {
                done = true;
                __syncwarp();
                wq[3] = 1;
            }
        }
        if (done) {
            // the global queue: all tiles (dynamic mode) or the tail (static mode)
            const int base = DYNAMIC ? 0 : s_tail0;
            const int step = DYNAMIC ? kClaim : kClaimTail;
            int tnext = wq[1], cend = wq[0];
            if (tnext >= cend) {
                int c = 0;
                if (lane == 0) c = atomicAdd(&a.ds->tile_counter, step);
                tnext = base + __shfl_sync(0xffffffffu, c, 0);
                cend = tnext + step;
            }
            if (tnext < ntiles) res = tnext++;
            __syncwarp();
            wq[1] = tnext;
            wq[0] = cend;
        }
        __syncwarp();
        return res;
    };
    int t = claim();
    while (t >= 0) {
        // claim the next tile now and bring its list head, position and count
        // into L2 while this tile runs (a grid launch gets this overlap from
        // its next CTAs)
        const int tn = claim();
        if (tn >= 0) {
            const int in = (tn << 5) + lane;
            if (in < nitems) {
                if (PAIRED) {
                    prefetch_l2(pa.list + list_group(in, pa.cap) + ((in & 31) << 2));
                    prefetch_l2(pa.slot_atom + in);
                    prefetch_l2(pa.count + in);
                } else {
                    prefetch_l2(a.nlist + list_group(in, a.cap) + ((in & 31) << 2));
                    if (F64) prefetch_l2(a.xr + in);
                    else prefetch_l2(a.xq + in);
                    prefetch_l2(a.ncount + in);
                }
            }
        }
        const int i = (t << 5) + lane;
        const bool active = i < nitems;
        long long t0 = 0;
        if (TIMING) {
            __syncwarp();
            t0 = clock64();
        }
        if (active) {
            if (PAIRED) lj_pair_slot<MODE, false>(a, pa, &sh, i, store_f);
            else if (F64) lj_fp64_atom<MODE, ENERGY>(a, sh64, i, store_f);
            else lj_mixed_atom<MODE, ENERGY, MULTI>(a, &sh, i, store_f);
        }
        if (TIMING) {
            __syncwarp();
            const long long dt = clock64() - t0;
            const unsigned act = __ballot_sync(0xffffffffu, active);
            if (active) {
                const int c = PAIRED ? sa.cell[pa.slot_atom[i] & ~kSingle] : sa.cell[i];
                atomicAdd(&sa.cell_cycles[c], (float)dt / (float)__popc(act));
            }
        }
        t = tn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (TIMING) sa.cta_cycles[blockIdx.x] += (float)(clock64() - cta_t0);
        {
            __threadfence();
            const unsigned prev = atomicAdd(&a.ds->done_ctas, 1u);
            if (prev == gridDim.x - 1) {
                a.ds->tile_counter = 0;
                a.ds->done_ctas = 0;
                __threadfence();
            }
        }
    }
}

template <int MODE, bool ENERGY>
__global__ void __launch_bounds__(kBlock) lj_fp64_kernel(ForceArgs a, int store_f) {
    __shared__ double3 sh[kStencil];
    load_shifts_f64(a.g, sh);
    __syncthreads();
    if (a.ds->status != 0) return;
    step_bookkeeping<MODE>(a);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.n) lj_fp64_atom<MODE, ENERGY>(a, sh, i, store_f);
}

// ---- multi-element Lennard-Jones (Sec. 2.2 pair loop, Sec. 3.1 Cu-Au) ------
//
// The paper's SIMD loop reloads the parameters of each pair with masks.  Here
// the lane keeps the row of its own species (NT values of each parameter) in
// registers and picks the pair's entry with the species of j, which sits in
// the position word it loads anyway: selects instead of loads.

template <int NT>
__device__ __forceinline__ float pick_row(const float *row, int t) {
    if (NT == 1) return row[0];
    if (NT == 2) return t ? row[1] : row[0];
    if (NT == 3) return t == 0 ? row[0] : (t == 1 ? row[1] : row[2]);
    return t < 2 ? (t == 0 ? row[0] : row[1]) : (t == 2 ? row[2] : row[3]);
}
template <int NT>
__device__ __forceinline__ double pick_row(const double *row, int t) {
    if (NT == 1) return row[0];
    if (NT == 2) return t ? row[1] : row[0];
    if (NT == 3) return t == 0 ? row[0] : (t == 1 ? row[1] : row[2]);
    return t < 2 ? (t == 0 ? row[0] : row[1]) : (t == 2 ? row[2] : row[3]);
}
// row ti of an NT x NT table, into registers (constant indices only)
template <int NT, class T>
__device__ __forceinline__ void load_row(const T *tab, int ti, T *row) {
#pragma unroll
    for (int k = 0; k < NT; ++k) {
        T v = tab[k];
#pragma unroll
        for (int r = 1; r < NT; ++r) v = (ti == r) ? tab[r * NT + k] : v;
        row[k] = v;
    }
}

template <int MODE, bool ENERGY, int NT>
__device__ __forceinline__ void lj_typed_mixed_atom(const ForceArgs &a, const TypeTab &tt,
                                                    const ShiftTab *sh, int i, int store_f) {
    const float4 qi = a.xq[i];
    const int ti = species_of(__float_as_uint(qi.w));
    float e48[NT], e4[NT], s2[NT], shf[NT];
    load_row<NT>(tt.e48, ti, e48);
    load_row<NT>(tt.e4, ti, e4);
    load_row<NT>(tt.s2, ti, s2);
    load_row<NT>(tt.sh, ti, shf);
    const int nq = (min(a.ncount[i], a.cap) + 3) >> 2;
    const uint4 *lq = reinterpret_cast<const uint4 *>(a.nlist + list_group(i, a.cap)) + (i & 31);
    const float rc2 = a.fc.rc2f;
    double Fx = 0.0, Fy = 0.0, Fz = 0.0, E = 0.0;
    unsigned npair = 0;
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
    auto pair = [&](uint32_t ent) {
        const float4 qj = __ldg(a.xq + (ent & kIndexMask));
        const uint32_t st = ent >> kIndexBits;
        const float ex = (qj.x - qi.x) + sh->x[st];
        const float ey = (qj.y - qi.y) + sh->y[st];
        const float ez = (qj.z - qi.z) + sh->z[st];
        const float r2 = ex * ex + ey * ey + ez * ez;
        if (r2 < rc2) {
            const int tj = species_of(__float_as_uint(qj.w));
            const float r2i = __fdividef(1.0f, r2);
            float s6 = pick_row<NT>(s2, tj) * r2i;
            s6 = s6 * s6 * s6;
            const float fs = pick_row<NT>(e48, tj) * r2i * s6 * (s6 - 0.5f);
            fx -= fs * ex;
            fy -= fs * ey;
            fz -= fs * ez;
            if (ENERGY) {
                e += pick_row<NT>(e4, tj) * s6 * (s6 - 1.0f) - pick_row<NT>(shf, tj);
                ++npair;
            }
        }
    };
    uint4 nxt = nq > 0 ? __ldcs(lq) : make_uint4(0u, 0u, 0u, 0u);
    for (int q0 = 0; q0 < nq; q0 += kChunkQ) {
        const int q1 = min(q0 + kChunkQ, nq);
        for (int q = q0; q < q1; ++q) {
            const uint4 e4q = nxt;
            if (q + 1 < nq) nxt = __ldcs(lq + (size_t)(q + 1) * 32);
            pair(e4q.x);
            pair(e4q.y);
            pair(e4q.z);
            pair(e4q.w);
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
    if (MODE != FM_STORE) vv_epilogue<MODE, true>(a, i, Fx, Fy, Fz, qi.w);
}

template <int MODE, bool ENERGY, int NT>
__device__ __forceinline__ void lj_typed_fp64_atom(const ForceArgs &a, const TypeTab &tt,
                                                   const double3 *sh, int i, int store_f) {
    const double4 ri = a.xr[i];
    const float4 qi = a.xq[i];
    const int ti = species_of(__float_as_uint(qi.w));
    double e48[NT], e4[NT], s2[NT], shd[NT];
    load_row<NT>(tt.e48d, ti, e48);
    load_row<NT>(tt.e4d, ti, e4);
    load_row<NT>(tt.s2d, ti, s2);
    load_row<NT>(tt.shd, ti, shd);
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
            const int tj = species_of(__float_as_uint(__ldg(&a.xq[j].w)));
            const double r2i = 1.0 / r2;
            double s6 = pick_row<NT>(s2, tj) * r2i;
            s6 = s6 * s6 * s6;
            const double fs = pick_row<NT>(e48, tj) * r2i * s6 * (s6 - 0.5);
            fx -= fs * ex;
            fy -= fs * ey;
            fz -= fs * ez;
            if (ENERGY) {
                e += pick_row<NT>(e4, tj) * s6 * (s6 - 1.0) - pick_row<NT>(shd, tj);
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
    if (MODE != FM_STORE) vv_epilogue<MODE, true>(a, i, fx, fy, fz, qi.w);
}

template <int MODE, bool ENERGY, int NT, bool F64>
__global__ void __launch_bounds__(128) lj_typed_kernel(ForceArgs a, TypeTab tt, int store_f) {
    __shared__ ShiftTab sh;
    __shared__ double3 sh64[F64 ? kStencil : 1];
    if (F64) load_shifts_f64(a.g, sh64);
    else load_shifts_f32(a.g, &sh);
    __syncthreads();
    if (a.ds->status != 0) return;
    step_bookkeeping<MODE>(a);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    if (F64) lj_typed_fp64_atom<MODE, ENERGY, NT>(a, tt, sh64, i, store_f);
    else lj_typed_mixed_atom<MODE, ENERGY, NT>(a, tt, &sh, i, store_f);
}

template <int NT, bool F64>
cudaError_t launch_lj_typed_nt(md_system *h, const ForceArgs &a, int mode, bool energy, int sf) {
    const int nb = nblocks(a.n, 128);
    cudaStream_t s = h->stream;
    const TypeTab &tt = h->types;
    switch (mode) {
        case FM_STORE:
            if (energy) lj_typed_kernel<FM_STORE, true, NT, F64><<<nb, 128, 0, s>>>(a, tt, sf);
            else lj_typed_kernel<FM_STORE, false, NT, F64><<<nb, 128, 0, s>>>(a, tt, sf);
            break;
        case FM_FUSED_FULL:
            if (energy) lj_typed_kernel<FM_FUSED_FULL, true, NT, F64><<<nb, 128, 0, s>>>(a, tt, sf);
            else lj_typed_kernel<FM_FUSED_FULL, false, NT, F64><<<nb, 128, 0, s>>>(a, tt, sf);
            break;
        default:
            if (energy) lj_typed_kernel<FM_FUSED_HALF, true, NT, F64><<<nb, 128, 0, s>>>(a, tt, sf);
            else lj_typed_kernel<FM_FUSED_HALF, false, NT, F64><<<nb, 128, 0, s>>>(a, tt, sf);
            break;
    }
    return cudaGetLastError();
}

template <bool F64>
cudaError_t launch_lj_typed_p(md_system *h, const ForceArgs &a, int mode, bool energy, int sf) {
    switch (h->fc.ntypes) {
        case 1: return launch_lj_typed_nt<1, F64>(h, a, mode, energy, sf);
        case 2: return launch_lj_typed_nt<2, F64>(h, a, mode, energy, sf);
        case 3: return launch_lj_typed_nt<3, F64>(h, a, mode, energy, sf);
        default: return launch_lj_typed_nt<4, F64>(h, a, mode, energy, sf);
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
    a.xqf = h->xqf;
    a.dF64 = h->dF64;
    a.rep = h->rep;
    a.shifts32 = h->shifts32;
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
    if (h->fc.ntypes > 0) {
        return h->p.precision == MD_MIXED ? launch_lj_typed_p<false>(h, a, mode, energy, sf)
                                          : launch_lj_typed_p<true>(h, a, mode, energy, sf);
    }
#define MDG_LJ(K, M, E) K<M, E><<<nb, kBlock, 0, s>>>(a, sf)
    if (h->R > 1) {
        // several boxes: mixed precision only (checked at creation)
        constexpr int tb = grid_block<true>();
        const int nbm = nblocks(a.n, tb);
        switch (mode) {
            case FM_STORE:
                if (energy) lj_mixed_kernel<FM_STORE, true, true><<<nbm, tb, 0, s>>>(a, sf);
                else lj_mixed_kernel<FM_STORE, false, true><<<nbm, tb, 0, s>>>(a, sf);
                break;
            case FM_FUSED_FULL:
                lj_mixed_kernel<FM_FUSED_FULL, false, true><<<nbm, tb, 0, s>>>(a, sf);
                break;
            default:
                lj_mixed_kernel<FM_FUSED_HALF, false, true><<<nbm, tb, 0, s>>>(a, sf);
                break;
        }
    } else if (h->p.precision == MD_MIXED) {
        constexpr int tb = grid_block<false>();
        const int nbs = nblocks(a.n, tb);
#define MDG_LJM(M, E) lj_mixed_kernel<M, E><<<nbs, tb, 0, s>>>(a, sf)
        switch (mode) {
            case FM_STORE: if (energy) MDG_LJM(FM_STORE, true); else MDG_LJM(FM_STORE, false); break;
            case FM_FUSED_FULL: if (energy) MDG_LJM(FM_FUSED_FULL, true); else MDG_LJM(FM_FUSED_FULL, false); break;
            default: if (energy) MDG_LJM(FM_FUSED_HALF, true); else MDG_LJM(FM_FUSED_HALF, false); break;
        }
#undef MDG_LJM
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

namespace mdg {

int persist_ctas_per_sm(bool f64, bool paired) {
    int nb = 0;
    const cudaError_t e =
        f64 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                  &nb, lj_mixed_persist<FM_FUSED_FULL, false, false, false, false, true>, kPersistBlock, 0)
        : paired ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                  &nb, lj_mixed_persist<FM_FUSED_FULL, false, false, false, false, false, true>,
                  kPersistBlock, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                  &nb, lj_mixed_persist<FM_FUSED_FULL, false, false, false>, kPersistBlock, 0);
    if (e != cudaSuccess) nb = 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_lj_persist(md_system *h, int mode, bool store_f, bool dynamic, bool timing) {
    ForceArgs a = make_force_args(h);
    const bool paired = (h->p.force_variant == MD_FORCE_PAIRED);
    SchedArgs sa;
    sa.cell_start = paired ? h->ps_start : h->cell_start;
    sa.bounds = h->part_bounds;
    sa.cell = h->cell;
    sa.cell_cycles = h->cell_cycles;
    sa.cta_cycles = h->cta_cycles;
    sa.rounds = h->sched_rounds;
    const PairArgs pa = paired ? make_pair_args(h) : PairArgs{};
    const int G = h->sched_ctas;
    const int sf = store_f ? 1 : 0;
    cudaStream_t s = h->stream;
    if (h->R > 1) {
        // several boxes: the tile queue (the static partitions are single-box)
        switch (mode) {
            case FM_STORE:
                lj_mixed_persist<FM_STORE, false, true, false, true><<<G, kPersistBlock, 0, s>>>(a, sf, sa, pa);
                break;
            case FM_FUSED_FULL:
                lj_mixed_persist<FM_FUSED_FULL, false, true, false, true><<<G, kPersistBlock, 0, s>>>(a, sf, sa, pa);
                break;
            default:
                lj_mixed_persist<FM_FUSED_HALF, false, true, false, true><<<G, kPersistBlock, 0, s>>>(a, sf, sa, pa);
                break;
        }
        return cudaGetLastError();
    }
    if (timing) {
        if (paired) {
            if (dynamic) lj_mixed_persist<FM_STORE, false, true, true, false, false, true><<<G, kPersistBlock, 0, s>>>(a, 1, sa, pa);
            else lj_mixed_persist<FM_STORE, false, false, true, false, false, true><<<G, kPersistBlock, 0, s>>>(a, 1, sa, pa);
        } else {
            if (dynamic) lj_mixed_persist<FM_STORE, false, true, true><<<G, kPersistBlock, 0, s>>>(a, 1, sa, pa);
            else lj_mixed_persist<FM_STORE, false, false, true><<<G, kPersistBlock, 0, s>>>(a, 1, sa, pa);
        }
        return cudaGetLastError();
    }
    const bool f64 = (h->p.precision == MD_FP64);
#define MDG_P(M)                                                                               \
    do {                                                                                       \
        if (paired) {                                                                          \
            if (dynamic)                                                                       \
                lj_mixed_persist<M, false, true, false, false, false, true><<<G, kPersistBlock, 0, s>>>(a, sf, sa, pa);  \
            else                                                                               \
                lj_mixed_persist<M, false, false, false, false, false, true><<<G, kPersistBlock, 0, s>>>(a, sf, sa, pa); \
        } else if (f64) {                                                                      \
            if (dynamic)                                                                       \
                lj_mixed_persist<M, false, true, false, false, true><<<G, kPersistBlock, 0, s>>>(a, sf, sa, pa);  \
            else                                                                               \
                lj_mixed_persist<M, false, false, false, false, true><<<G, kPersistBlock, 0, s>>>(a, sf, sa, pa); \
        } else if (dynamic) {                                                                  \
            lj_mixed_persist<M, false, true, false><<<G, kPersistBlock, 0, s>>>(a, sf, sa, pa);            \
        } else {                                                                               \
            lj_mixed_persist<M, false, false, false><<<G, kPersistBlock, 0, s>>>(a, sf, sa, pa);           \
        }                                                                                      \
    } while (0)
    switch (mode) {
        case FM_STORE: MDG_P(FM_STORE); break;
        case FM_FUSED_FULL: MDG_P(FM_FUSED_FULL); break;
        default: MDG_P(FM_FUSED_HALF); break;
    }
#undef MDG_P
    return cudaGetLastError();
}

}  // namespace mdg
