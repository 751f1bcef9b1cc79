// k_mlp.cu -- the learned per-cell cost model: a 3 -> 32 -> 32 -> 1
// multilayer perceptron with ReLU, trained with mean-squared error and Adam
// (Kingma & Ba) on per-cell timings, and the contiguous equal-cost partition
// of cells over persistent CTAs that its predictions feed.  The paper
// balances uneven work with its cell-task schedule (Sec. 2.1) and reports the
// imbalance of inhomogeneous systems (Sec. 1); this model predicts that
// unevenness ahead of the force pass.
//
// Parameter layout (1217 float32): W1[32][3], b1[32], W2[32][32], b2[32],
// W3[32], b3[1].
#include <cmath>
#include <mutex>
#include <string>

#include "k_scan.cuh"

namespace mdg {

constexpr int kH = 32;
constexpr int kNP = kH * 3 + kH + kH * kH + kH + kH + 1;  // 1217
constexpr int kOffB1 = kH * 3, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH;
constexpr int kMS = 64;        // samples per block in the gradient kernel
constexpr int kGradThreads = 128;

namespace {

__global__ void mlp_forward_kernel(const float *__restrict__ X, long long ns,
                                   const float *__restrict__ P, float *__restrict__ y,
                                   const DevStatus *ds, bool gated) {
    if (scan_off(ds, gated)) return;
    __shared__ float sP[kNP];
    for (int k = threadIdx.x; k < kNP; k += blockDim.x) sP[k] = P[k];
    __syncthreads();
    const float *W1 = sP, *b1 = sP + kOffB1, *W2 = sP + kOffW2, *b2 = sP + kOffB2,
                *W3 = sP + kOffW3;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < ns;
         s += (long long)gridDim.x * blockDim.x) {
        const float x0 = X[3 * s], x1 = X[3 * s + 1], x2 = X[3 * s + 2];
        float a1[kH];
#pragma unroll
        for (int u = 0; u < kH; ++u) {
            float z = b1[u] + W1[3 * u] * x0 + W1[3 * u + 1] * x1 + W1[3 * u + 2] * x2;
            a1[u] = z > 0.f ? z : 0.f;
        }
        float out = sP[kOffB3];
        for (int u = 0; u < kH; ++u) {
            float z = b2[u];
#pragma unroll
            for (int k = 0; k < kH; ++k) z += W2[kH * u + k] * a1[k];
            out += W3[u] * (z > 0.f ? z : 0.f);
        }
        y[s] = out;
    }
}

// Stage 1: each block back-propagates kMS samples and writes its partial
// gradient (sum over its samples) and partial squared-error sum.
__global__ void __launch_bounds__(kGradThreads)
mlp_grad_partial_kernel(const float *__restrict__ X, const float *__restrict__ Y, long long ns,
                        const float *__restrict__ P, float *__restrict__ partial,
                        float *__restrict__ lossp) {
    __shared__ float sP[kNP];
    __shared__ float sx[kMS][3];
    __shared__ float sa1[kMS][kH + 1], sd1[kMS][kH + 1], sa2[kMS][kH + 1], sd2[kMS][kH + 1];
    __shared__ float sdy[kMS], sl[kMS];
    for (int k = threadIdx.x; k < kNP; k += blockDim.x) sP[k] = P[k];
    __syncthreads();
    const float *W1 = sP, *b1 = sP + kOffB1, *W2 = sP + kOffW2, *b2 = sP + kOffB2,
                *W3 = sP + kOffW3;
    const int t = threadIdx.x;
    if (t < kMS) {
        const long long s = (long long)blockIdx.x * kMS + t;
        const bool ok = s < ns;
        const float x0 = ok ? X[3 * s] : 0.f, x1 = ok ? X[3 * s + 1] : 0.f,
                    x2 = ok ? X[3 * s + 2] : 0.f;
        sx[t][0] = x0; sx[t][1] = x1; sx[t][2] = x2;
        float z1[kH], a1[kH];
#pragma unroll
        for (int u = 0; u < kH; ++u) {
            float z = b1[u] + W1[3 * u] * x0 + W1[3 * u + 1] * x1 + W1[3 * u + 2] * x2;
            z1[u] = z;
            a1[u] = z > 0.f ? z : 0.f;
            sa1[t][u] = ok ? a1[u] : 0.f;
        }
        float yh = sP[kOffB3];
        for (int u = 0; u < kH; ++u) {
            float z = b2[u];
#pragma unroll
            for (int k = 0; k < kH; ++k) z += W2[kH * u + k] * a1[k];
            const float a2 = z > 0.f ? z : 0.f;
            sa2[t][u] = ok ? a2 : 0.f;
            sd2[t][u] = z > 0.f ? 1.f : 0.f;  // ReLU mask for now
            yh += W3[u] * a2;
        }
        const float e = ok ? yh - Y[s] : 0.f;
        const float dy = ok ? 2.f * e / (float)ns : 0.f;
        sdy[t] = dy;
        sl[t] = e * e;
        float d2[kH];
#pragma unroll
        for (int u = 0; u < kH; ++u) {
            d2[u] = sd2[t][u] * dy * W3[u];
            sd2[t][u] = d2[u];
        }
#pragma unroll
        for (int k = 0; k < kH; ++k) {
            float acc = 0.f;
            for (int u = 0; u < kH; ++u) acc += W2[kH * u + k] * d2[u];
            sd1[t][k] = z1[k] > 0.f ? acc : 0.f;
        }
    }
    __syncthreads();
    float *out = partial + (size_t)blockIdx.x * kNP;
    for (int p = t; p < kNP; p += blockDim.x) {
        float acc = 0.f;
        if (p < kOffB1) {
            const int u = p / 3, c = p % 3;
            for (int s = 0; s < kMS; ++s) acc += sd1[s][u] * sx[s][c];
        } else if (p < kOffW2) {
            const int u = p - kOffB1;
            for (int s = 0; s < kMS; ++s) acc += sd1[s][u];
        } else if (p < kOffB2) {
            const int u = (p - kOffW2) / kH, k = (p - kOffW2) % kH;
            for (int s = 0; s < kMS; ++s) acc += sd2[s][u] * sa1[s][k];
        } else if (p < kOffW3) {
            const int u = p - kOffB2;
            for (int s = 0; s < kMS; ++s) acc += sd2[s][u];
        } else if (p < kOffB3) {
            const int k = p - kOffW3;
            for (int s = 0; s < kMS; ++s) acc += sdy[s] * sa2[s][k];
        } else {
            for (int s = 0; s < kMS; ++s) acc += sdy[s];
        }
        out[p] = acc;
    }
    if (t == 0) {
        float l = 0.f;
        for (int s = 0; s < kMS; ++s) l += sl[s];
        lossp[blockIdx.x] = l;
    }
}

// Stage 2: fixed-order sums over blocks.
__global__ void mlp_grad_reduce_kernel(const float *__restrict__ partial,
                                       const float *__restrict__ lossp, int nblk, long long ns,
                                       float *__restrict__ G, float *__restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kNP) {
        float acc = 0.f;
        for (int b = 0; b < nblk; ++b) acc += partial[(size_t)b * kNP + p];
        G[p] = acc;
    } else if (p == kNP && loss) {
        double l = 0.0;
        for (int b = 0; b < nblk; ++b) l += lossp[b];
        *loss = (float)(l / (double)ns);
    }
}

__global__ void adam_kernel(float *__restrict__ P, const float *__restrict__ G,
                            float *__restrict__ m, float *__restrict__ v, long long np, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= np) return;
    const float g = G[k];
    const float mk = b1 * m[k] + (1.f - b1) * g;
    const float vk = b2 * v[k] + (1.f - b2) * g * g;
    m[k] = mk;
    v[k] = vk;
    P[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// bounds[b] = first k with inclusive_prefix[k] * nparts > b * total.
__global__ void partition_kernel(const long long *__restrict__ excl, long long ncells, int nparts,
                                 long long *__restrict__ bounds, const DevStatus *ds,
                                 bool gated) {
    if (scan_off(ds, gated)) return;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nparts) return;
    if (b == 0) { bounds[0] = 0; return; }
    if (b == nparts) { bounds[nparts] = ncells; return; }
    const long long total = excl[ncells];
    const long long target = (long long)b * total;
    long long lo = 0, hi = ncells;  // search in [lo, hi)
    while (lo < hi) {
        const long long mid = lo + (hi - lo) / 2;
        if (excl[mid + 1] * (long long)nparts > target) hi = mid;
        else lo = mid + 1;
    }
    bounds[b] = lo;
}

// He-uniform initial weights (bound sqrt(6 / fan_in)), zero biases.  The
// uniform deviates come from splitmix64 of (seed, parameter index).
__global__ void mlp_init_kernel(float *P, unsigned long long seed) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kNP) return;
    int fan_in = 0;
    if (k < kOffB1) fan_in = 3;
    else if (k >= kOffW2 && k < kOffB2) fan_in = kH;
    else if (k >= kOffW3 && k < kOffB3) fan_in = kH;
    if (fan_in == 0) {
        P[k] = 0.f;
        return;
    }
    unsigned long long z = seed + (unsigned long long)(k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double u = ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double b = sqrt(6.0 / fan_in);
    P[k] = (float)((2.0 * u - 1.0) * b);
}

}  // namespace

cudaError_t launch_mlp_init(float *P, unsigned long long seed, cudaStream_t s) {
    mlp_init_kernel<<<(kNP + kBlock - 1) / kBlock, kBlock, 0, s>>>(P, seed);
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float *X, long long ns, const float *P, float *y,
                               cudaStream_t s, const DevStatus *ds, bool gated) {
    if (ns <= 0) return cudaSuccess;
    long long nb = (ns + kBlock - 1) / kBlock;
    int grid = (int)(nb < 152 * 16 ? nb : 152 * 16);
    mlp_forward_kernel<<<grid, kBlock, 0, s>>>(X, ns, P, y, ds, gated);
    return cudaGetLastError();
}

// scratch: at least mlp_grad_scratch_floats(ns) floats
size_t mlp_grad_scratch_floats(long long ns) {
    const long long nblk = (ns + kMS - 1) / kMS;
    return (size_t)nblk * (kNP + 1) + 1;
}

cudaError_t launch_mlp_loss_grad(const float *X, const float *Y, long long ns, const float *P,
                                 float *G, float *loss, float *scratch, cudaStream_t s) {
    const int nblk = (int)((ns + kMS - 1) / kMS);
    float *partial = scratch;
    float *lossp = scratch + (size_t)nblk * kNP;
    mlp_grad_partial_kernel<<<nblk, kGradThreads, 0, s>>>(X, Y, ns, P, partial, lossp);
    mlp_grad_reduce_kernel<<<(kNP + 1 + kBlock - 1) / kBlock, kBlock, 0, s>>>(partial, lossp, nblk,
                                                                            ns, G, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *P, const float *G, float *m, float *v, long long np, long long t,
                        float lr, float b1, float b2, float eps, cudaStream_t s) {
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)t));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)t));
    adam_kernel<<<(int)((np + kBlock - 1) / kBlock), kBlock, 0, s>>>(P, G, m, v, np, lr, b1, b2,
                                                                    eps, c1, c2);
    return cudaGetLastError();
}

// scratch: at least ncells + 1 + ncells / kScanTile + 4 int64
cudaError_t launch_partition(const long long *cost, long long ncells, int nparts,
                             long long *bounds, long long *scratch, cudaStream_t s,
                             const DevStatus *ds, bool gated) {
    long long *excl = scratch;
    long long *bsum = scratch + ncells + 1;
    cudaError_t e = launch_scan<long long>(cost, excl, (int)ncells, bsum, ds, gated, s);
    if (e != cudaSuccess) return e;
    partition_kernel<<<(nparts + 1 + kBlock - 1) / kBlock, kBlock, 0, s>>>(excl, ncells, nparts,
                                                                          bounds, ds, gated);
    return cudaGetLastError();
}

}  // namespace mdg

// ---- C ABI of the cost-model building blocks --------------------------------

namespace {
thread_local std::string g_mlp_error;
}

extern "C" {

md_status md_mlp_forward(const float *X_dev, int64_t ns, const float *P_dev, float *y_dev,
                         void *cuda_stream) {
    if (ns < 0 || (ns > 0 && (!X_dev || !P_dev || !y_dev))) return MD_ERR_INVALID;
    return mdg::launch_mlp_forward(X_dev, ns, P_dev, y_dev, (cudaStream_t)cuda_stream) ==
                   cudaSuccess
               ? MD_OK
               : MD_ERR_CUDA;
}

md_status md_mlp_loss_grad(const float *X_dev, const float *y_dev, int64_t ns,
                           const float *P_dev, float *G_dev, float *loss_dev,
                           void *cuda_stream) {
    if (ns <= 0 || !X_dev || !y_dev || !P_dev || !G_dev) return MD_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    float *scratch = nullptr;
    const size_t bytes = mdg::mlp_grad_scratch_floats(ns) * sizeof(float);
    if (cudaMallocAsync((void **)&scratch, bytes, s) != cudaSuccess) return MD_ERR_OOM;
    cudaError_t e = mdg::launch_mlp_loss_grad(X_dev, y_dev, ns, P_dev, G_dev, loss_dev, scratch, s);
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    return (e == cudaSuccess && e2 == cudaSuccess) ? MD_OK : MD_ERR_CUDA;
}

md_status md_mlp_adam(float *P_dev, const float *G_dev, float *m_dev, float *v_dev, int64_t np,
                      int64_t t, float lr, float beta1, float beta2, float epsilon,
                      void *cuda_stream) {
    if (np <= 0 || t < 1 || !P_dev || !G_dev || !m_dev || !v_dev) return MD_ERR_INVALID;
    return mdg::launch_adam(P_dev, G_dev, m_dev, v_dev, np, t, lr, beta1, beta2, epsilon,
                            (cudaStream_t)cuda_stream) == cudaSuccess
               ? MD_OK
               : MD_ERR_CUDA;
}

md_status md_partition(const int64_t *cost_dev, int64_t ncells, int32_t nparts,
                       int64_t *bounds_dev, void *cuda_stream) {
    if (ncells < 1 || ncells >= ((int64_t)1 << 31) || nparts < 1 || !cost_dev || !bounds_dev)
        return MD_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    long long *scratch = nullptr;
    const size_t words = (size_t)ncells + 1 + (size_t)ncells / mdg::kScanTile + 8;
    if (cudaMallocAsync((void **)&scratch, words * sizeof(long long), s) != cudaSuccess)
        return MD_ERR_OOM;
    cudaError_t e = mdg::launch_partition((const long long *)cost_dev, ncells, nparts,
                                          (long long *)bounds_dev, scratch, s);
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    return (e == cudaSuccess && e2 == cudaSuccess) ? MD_OK : MD_ERR_CUDA;
}

}  // extern "C"

// ---- md_partition without device allocation ----------------------------------
//
// Some callers cannot allocate device memory while they run: a simulation loop
// that fixed its memory budget at start-up, a host framework whose own
// allocator owns the device heap, or a driver setup without stream-ordered
// allocation (cudaMallocAsync unsupported).  md_partition takes its scan
// scratch from cudaMallocAsync; this variant uses a fixed array that lives in
// the library's device image instead.  Every GPU that loads the library holds
// the array (about 8.4 MB) until the process exits.

namespace mdg {
namespace {

constexpr long long kNoAllocMaxCells = 1ll << 20;  // largest ncells accepted
constexpr long long kNoAllocWords = kNoAllocMaxCells + 1 + kNoAllocMaxCells / kScanTile + 8;

// prefix sums of the costs (ncells + 1) followed by the scan's tile sums
static __device__ __align__(256) long long g_partition_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
long long *g_scratch_addr[kMaxDevices] = {};

// Device address of g_partition_scratch on the current device.  In host code
// the array's name is only a stand-in, so the address is looked up once per
// device (with that device current) and cached.
cudaError_t scratch_address(long long **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        long long *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_partition_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace mdg

extern "C" md_status md_partition_noalloc(const int64_t *cost_dev, int64_t ncells, int32_t nparts,
                                          int64_t *bounds_dev, void *cuda_stream) {
    if (ncells < 1 || nparts < 1 || !cost_dev || !bounds_dev) {
        mdg::set_thread_error("md_partition_noalloc: bad argument");
        return MD_ERR_INVALID;
    }
    if (ncells > mdg::kNoAllocMaxCells) {
        mdg::set_thread_error("md_partition_noalloc: ncells = " + std::to_string(ncells) +
                              " exceeds the fixed scratch limit of " +
                              std::to_string(mdg::kNoAllocMaxCells) +
                              " cells (use md_partition, which allocates)");
        return MD_ERR_INVALID;
    }
    long long *scratch = nullptr;
    cudaError_t e = mdg::scratch_address(&scratch);
    if (e != cudaSuccess) {
        mdg::set_thread_error(std::string("md_partition_noalloc: cudaGetSymbolAddress: ") +
                              cudaGetErrorString(e));
        return MD_ERR_CUDA;
    }
    // The scan overwrites every scratch word it reads, so nothing needs clearing.
    e = mdg::launch_partition((const long long *)cost_dev, ncells, nparts, (long long *)bounds_dev,
                              scratch, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        mdg::set_thread_error(std::string("md_partition_noalloc: ") + cudaGetErrorString(e));
        return MD_ERR_CUDA;
    }
    return MD_OK;
}
