// k_scan.cuh -- exclusive prefix sum over a device array (three passes:
// per-tile scan, scan of tile sums, add tile offsets).  out[n] = total.
#pragma once

#include "md_internal.cuh"

namespace mdg {

constexpr int kScanItems = 8;
constexpr int kScanTile = kBlock * kScanItems;

template <class T>
__device__ T block_exclusive(T v, T *total) {
    __shared__ T warp_sums[kBlock / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T ws = (lane < kBlock / 32) ? warp_sums[lane] : T(0);
        T wi = ws;
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < kBlock / 32) warp_sums[lane] = wi - ws;  // exclusive warp offsets
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    T r = warp_sums[wid] + inc - v;
    __syncthreads();
    return r;
}

__device__ __forceinline__ bool scan_off(const DevStatus *ds, bool gated) {
    return ds != nullptr && (ds->status != 0 || (gated && ds->rebuild == 0));
}

template <class T>
__global__ void scan_block_kernel(const T *__restrict__ in, T *__restrict__ out, int n,
                                  T *__restrict__ bsum, const DevStatus *ds, bool gated) {
    if (scan_off(ds, gated)) return;
    __shared__ T tot;
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    T vals[kScanItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long idx = base + k;
        vals[k] = (idx < n) ? in[idx] : T(0);
        s += vals[k];
    }
    T off = block_exclusive<T>(s, &tot);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        long long idx = base + k;
        if (idx < n) out[idx] = off;
        off += vals[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <class T>
__global__ void scan_bsum_kernel(T *bsum, int nb, const DevStatus *ds, bool gated) {
    if (scan_off(ds, gated)) return;
    __shared__ T tot;
    T carry = 0;
    for (int c0 = 0; c0 < nb; c0 += kBlock) {
        int idx = c0 + threadIdx.x;
        T v = (idx < nb) ? bsum[idx] : T(0);
        T ex = block_exclusive<T>(v, &tot);
        if (idx < nb) bsum[idx] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) bsum[nb] = carry;
}

template <class T>
__global__ void scan_add_kernel(T *out, int n, const T *__restrict__ bsum, int nb,
                                const DevStatus *ds, bool gated) {
    if (scan_off(ds, gated)) return;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += gridDim.x * blockDim.x)
        out[idx] += bsum[idx / kScanTile];
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = bsum[nb];
}

// bsum must hold at least n / kScanTile + 2 elements.
template <class T>
inline cudaError_t launch_scan(const T *in, T *out, int n, T *bsum, const DevStatus *ds,
                               bool gated, cudaStream_t s) {
    int nb = (n + kScanTile - 1) / kScanTile;
    if (nb < 1) nb = 1;
    scan_block_kernel<T><<<nb, kBlock, 0, s>>>(in, out, n, bsum, ds, gated);
    scan_bsum_kernel<T><<<1, kBlock, 0, s>>>(bsum, nb, ds, gated);
    scan_add_kernel<T><<<gs_blocks(n), kBlock, 0, s>>>(out, n, bsum, nb, ds, gated);
    return cudaGetLastError();
}

}  // namespace mdg
