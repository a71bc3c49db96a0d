// k_batched.cu -- kernels of the batched engine (many independent CP fits).
//
//  * k_pad_problem: copy one problem's Y into a zero-padded layout whose
//    dimensions are multiples of 4 (the TMA stride rule) and pack its mask into
//    bits; padded entries are unobserved.
//  * k_mirror_batched: the canonical copies of every unit's starting factors.
//  * k_loss_batched: sum over observed entries of D_{alpha,beta}(y, yhat) for
//    every restart of one problem, reading Y once per entry (App. B, Eq. 3.1).
#include "nef_batched.h"
#include "nef_device.cuh"

namespace nef {

namespace {

constexpr int kThreads = 256;

__global__ void k_pad_problem(const float* __restrict__ y, const uint8_t* __restrict__ mask, int64_t I,
                              int64_t J, int64_t K, int64_t Ip, int64_t Jp, int64_t Kp,
                              float* __restrict__ yp, uint32_t* __restrict__ bits) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t np = Ip * Jp * Kp;
    const int64_t nw = (np + 31) >> 5;
    if (w >= nw) return;
    uint32_t word = 0;
    for (int b = 0; b < 32; ++b) {
        const int64_t e = (w << 5) + b;
        if (e >= np) break;
        const int64_t k = e % Kp, ij = e / Kp;
        const int64_t j = ij % Jp, i = ij / Jp;
        float v = 0.f;
        int obs = 0;
        if (i < I && j < J && k < K) {
            const int64_t src = (i * J + j) * K + k;
            v = y[src];
            obs = mask ? (mask[src] != 0) : 1;
        }
        yp[e] = v;
        word |= (uint32_t)obs << b;
    }
    bits[w] = word;
}

__device__ __forceinline__ uint16_t bf16_bits_b(float x) {
    uint32_t u = __float_as_uint(x);
    uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(r >> 16);
}

// Element g of the concatenated factor space -> unit by binary search in prefix[].
__global__ void k_mirror_batched(const BatchFinish* __restrict__ fin, const int64_t* __restrict__ prefix,
                                 int n_units) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= prefix[n_units]) return;
    int lo = 0, hi = n_units - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const BatchFinish& f = fin[lo];
    const int64_t e = g - prefix[lo];
    const int64_t row = e / f.rank, r = e % f.rank;
    const int64_t so = row * f.bp + r;
    const float v = f.theta[e];
    f.canon32[so] = v;
    f.canon16[so] = bf16_bits_b(v);
}

// One problem, all restarts: thread per entry of the unpadded tensor.
template <bool SMEM>
__global__ void k_loss_batched(const float* __restrict__ y, const uint8_t* __restrict__ mask, int64_t I,
                               int64_t J, int64_t K, int rank, int restarts, const __grid_constant__ BatchFactors fac,
                               const __grid_constant__ LossSpec L, double* __restrict__ part) {
    // One restart at a time: C of that restart in shared memory as [rank][K] (lanes read
    // consecutive k; SMEM = false for a C too large for it: read from global memory),
    // each warp takes (i, j) pairs and its lanes the k of that row of Y; lane r holds
    // A[i,r] B[j,r] and the rank-sum runs over shuffles of it (rank <= 32).
    extern __shared__ float c_sh[];
    __shared__ double sh[kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t n_ij = I * J;
    const int64_t warps_total = (int64_t)gridDim.x * (kThreads / 32);
    for (int q = 0; q < restarts; ++q) {
        const float* A = fac.f[q][0];
        const float* B = fac.f[q][1];
        const float* C = fac.f[q][2];
        if constexpr (SMEM) {
            __syncthreads();  // c_sh free from the previous restart
            for (int64_t t = threadIdx.x; t < K * rank; t += kThreads) {
                const int64_t k = t / rank, r = t - k * rank;
                c_sh[r * K + k] = C[t];
            }
            __syncthreads();
        }
        double acc = 0.0;
        for (int64_t ij = (int64_t)blockIdx.x * (kThreads / 32) + warp; ij < n_ij; ij += warps_total) {
            const int64_t i = ij / J, j = ij - i * J;
            const float ab = lane < rank ? A[i * rank + lane] * B[j * rank + lane] : 0.f;
            for (int64_t k0 = 0; k0 < K; k0 += 32) {
                const int64_t k = k0 + lane;
                const int64_t kc = k < K ? k : K - 1;
                float yh = 0.f;
                for (int r = 0; r < rank; ++r)
                    yh = fmaf(__shfl_sync(0xffffffffu, ab, r), SMEM ? c_sh[r * K + kc] : C[kc * rank + r], yh);
                const int64_t e = ij * K + k;
                if (k < K && (!mask || mask[e])) acc += (double)divergence(y[e], yh, L);
            }
        }
        acc = warp_sum(acc);
        if (lane == 0) sh[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tsum = 0.0;
            for (int w = 0; w < kThreads / 32; ++w) tsum += sh[w];
            part[(int64_t)blockIdx.x * restarts + q] = tsum;
        }
        __syncthreads();  // sh read before the next restart writes it
    }
}

__global__ void k_loss_reduce(const double* __restrict__ part, int n_blocks, int restarts, double* out) {
    const int q = threadIdx.x;
    if (q >= restarts) return;
    double t = 0.0;
    for (int b = 0; b < n_blocks; ++b) t += part[(int64_t)b * restarts + q];
    out[q] = t;
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t launch_pad_problem(const float* y, const uint8_t* mask, const int64_t* dims, const int64_t* pdims,
                               float* yp, uint32_t* bits, cudaStream_t st) {
    const int64_t nw = (pdims[0] * pdims[1] * pdims[2] + 31) >> 5;
    k_pad_problem<<<blocks_for(nw), kThreads, 0, st>>>(y, mask, dims[0], dims[1], dims[2], pdims[0], pdims[1],
                                                        pdims[2], yp, bits);
    return cudaGetLastError();
}

cudaError_t launch_mirror_batched(const BatchFinish* fin, const int64_t* prefix, int n_units, int64_t total,
                                  cudaStream_t st) {
    k_mirror_batched<<<blocks_for(total), kThreads, 0, st>>>(fin, prefix, n_units);
    return cudaGetLastError();
}

cudaError_t launch_loss_batched(const float* y, const uint8_t* mask, const int64_t* dims, int rank, int restarts,
                                const BatchFactors& fac, const LossSpec& L, double* part, int n_blocks,
                                double* out, cudaStream_t st) {
    if (rank > 32) return cudaErrorInvalidValue;
    const size_t smem = (size_t)dims[2] * rank * sizeof(float);  // C of one restart, [rank][K]
    if (smem <= 96 * 1024) {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_loss_batched<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        k_loss_batched<true><<<n_blocks, kThreads, smem, st>>>(y, mask, dims[0], dims[1], dims[2], rank, restarts,
                                                               fac, L, part);
    } else {
        k_loss_batched<false><<<n_blocks, kThreads, 0, st>>>(y, mask, dims[0], dims[1], dims[2], rank, restarts, fac,
                                                             L, part);
    }
    k_loss_reduce<<<1, 32, 0, st>>>(part, n_blocks, restarts, out);
    return cudaGetLastError();
}

}  // namespace nef
