// k_foldin.cu -- elementwise kernels of the fold-in encoder (training and
// inference of the MLP that maps a slice Y[i, :, :] to its mode-0 loading row):
//   x = log1p(slice) in BF16 (row-major and transposed copies),
//   z = acc + b, h = relu(z) (BF16 copies for the next products), out = softplus(z),
//   the loss L = mean (log1p(out) - log1p(t))^2 and dL/dz at the output,
//   relu backward, bias gradients (column sums), Adam, and the BF16 weight copies.
// The products themselves run on the tensor cores (k_gemm_tc.cu).
#include <cuda_bf16.h>

#include "nef_device.cuh"
#include "nef_internal.h"
#include "nef_launch.cuh"

namespace nef {

namespace {

constexpr int kT = 256;

__device__ __forceinline__ uint16_t to_bf16(float x) {
    const __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<const uint16_t*>(&b);
}

__device__ __forceinline__ float softplus_f(float z) { return z > 30.f ? z : log1pf(__expf(z)); }
__device__ __forceinline__ float sigmoid_f(float z) { return 1.f / (1.f + __expf(-z)); }

// 32 x 32 tiles: row-major write of f(src) and a transposed write through shared memory.
// src [n x d] FP32 (ld d); dst [n x d] BF16 (ld d); dst_t [d x ldt] BF16.
template <int OP>
__global__ void k_fi_convert_t(const float* __restrict__ src, int n, int d, uint16_t* __restrict__ dst,
                               uint16_t* __restrict__ dst_t, int ldt) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint16_t tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    for (int k = ty; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + tx;
        uint16_t b = 0;
        if (r < n && c < d) {
            const float v = src[(int64_t)r * d + c];
            b = to_bf16(OP == 1 ? log1pf(v) : v);
            if (dst) dst[(int64_t)r * d + c] = b;
        }
        tile[k][tx] = b;
    }
    __syncthreads();
    if (!dst_t) return;
    for (int k = ty; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + tx;
        if (c < d && r < n) dst_t[(int64_t)c * ldt + r] = tile[tx][k];
    }
}

// z += b (per column); act 1: h = relu(z) -> BF16 (row-major, and transposed if ht);
// act 2: out = softplus(z) (FP32).
__global__ void k_fi_bias_act(float* __restrict__ z, const float* __restrict__ b, int n, int h, int act,
                              uint16_t* __restrict__ hb, uint16_t* __restrict__ ht, int ldt, float* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint16_t tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k = ty; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + tx;
        uint16_t v16 = 0;
        if (r < n && c < h) {
            const int64_t e = (int64_t)r * h + c;
            const float zz = z[e] + b[c];
            z[e] = zz;
            if (act == 1) {
                v16 = to_bf16(fmaxf(zz, 0.f));
                hb[e] = v16;
            } else {
                out[e] = softplus_f(zz);
            }
        }
        tile[k][tx] = v16;
    }
    if (act != 1 || !ht) return;
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + tx;
        if (c < h && r < n) ht[(int64_t)c * ldt + r] = tile[tx][k];
    }
}

// Output layer: d = log1p(out) - log1p(t); g = 2 d / (1 + out) * inv_count * sigmoid(z);
// per-block sums of d^2 into part[block].
__global__ void k_fi_out_grad(const float* __restrict__ out, const float* __restrict__ t, const float* __restrict__ z,
                              int64_t n_el, float inv_count, float* __restrict__ g, double* __restrict__ part) {
    pdl_wait();
    pdl_trigger();
    __shared__ double sh[kT / 32];
    double acc = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += (int64_t)gridDim.x * blockDim.x) {
        const float o = out[e];
        const float d = log1pf(o) - log1pf(t[e]);
        acc += (double)d * d;
        if (g) g[e] = 2.f * d / (1.f + o) * inv_count * sigmoid_f(z[e]);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < kT / 32; ++k) s += sh[k];
        part[blockIdx.x] = s;
    }
}

// g *= (z > 0) (relu backward), in place; BF16 copies row-major (gb) and transposed (gt).
__global__ void k_fi_relu_grad(float* __restrict__ g, const float* __restrict__ z, int n, int h,
                               uint16_t* __restrict__ gb, uint16_t* __restrict__ gt, int ldt) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint16_t tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k = ty; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + tx;
        uint16_t v16 = 0;
        if (r < n && c < h) {
            const int64_t e = (int64_t)r * h + c;
            const float v = z[e] > 0.f ? g[e] : 0.f;
            g[e] = v;
            v16 = to_bf16(v);
            if (gb) gb[e] = v16;
        }
        tile[k][tx] = v16;
    }
    if (!gt) return;
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + tx;
        if (c < h && r < n) gt[(int64_t)c * ldt + r] = tile[tx][k];
    }
}

// out[c] = sum over rows of g[r][c] (fixed order), one thread per column.
// Column sums of g [n x h]: a block per 32 columns; its 32 warps take rows
// w, w + 32, ... of their column (lane), then warp 0 adds the 32 partial sums in
// warp order (a fixed order: the result does not depend on scheduling).
constexpr int kColsumWarps = 32;
__global__ void __launch_bounds__(32 * kColsumWarps) k_fi_colsum(const float* __restrict__ g, int n, int h,
                                                                 float* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    __shared__ float part[kColsumWarps][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (c < h)
        for (int r = w; r < n; r += kColsumWarps) s += g[(int64_t)r * h + c];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && c < h) {
        float t = 0.f;
        for (int k = 0; k < kColsumWarps; ++k) t += part[k][lane];
        out[c] = t;
    }
}

// Adam (Kingma & Ba) on the packed parameters; bc1 = 1 - b1^t, bc2 = 1 - b2^t.
__global__ void k_fi_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                          float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float bc1,
                          float bc2) {
    pdl_wait();
    pdl_trigger();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
}

// Adam on a row-major [rows x cols] weight block, in 32 x 32 tiles, that also writes
// the BF16 transposed copy of the updated weights (dst_t [cols x rows]) through
// shared memory, so the copy costs no second read of the weights.
__global__ void k_fi_adam_t(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int rows, int cols, float lr, float b1, float b2, float eps,
                            float bc1, float bc2, uint16_t* __restrict__ dst_t) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint16_t tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k = ty; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + tx;
        uint16_t b = 0;
        if (r < rows && c < cols) {
            const int64_t e = (int64_t)r * cols + c;
            const float gg = g[e];
            const float mm = b1 * m[e] + (1.f - b1) * gg;
            const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
            m[e] = mm;
            v[e] = vv;
            const float np = p[e] - lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
            p[e] = np;
            b = to_bf16(np);
        }
        tile[k][tx] = b;
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + tx;
        if (c < cols && r < rows) dst_t[(int64_t)c * rows + r] = tile[tx][k];
    }
}

// BF16 copy of a row-major [rows x cols] FP32 matrix: straight (dst, ld cols) and/or
// transposed (dst_t [cols x rows], ld rows).
__global__ void k_fi_weight_copy(const float* __restrict__ w, int rows, int cols, uint16_t* __restrict__ dst,
                                 uint16_t* __restrict__ dst_t) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint16_t tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int k = ty; k < 32; k += 8) {
        const int r = r0 + k, c = c0 + tx;
        uint16_t v16 = 0;
        if (r < rows && c < cols) {
            v16 = to_bf16(w[(int64_t)r * cols + c]);
            if (dst) dst[(int64_t)r * cols + c] = v16;
        }
        tile[k][tx] = v16;
    }
    if (!dst_t) return;
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int c = c0 + k, r = r0 + tx;
        if (c < cols && r < rows) dst_t[(int64_t)c * rows + r] = tile[tx][k];
    }
}

dim3 tiles32(int rows, int cols) { return dim3((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32)); }

// The features x = log1p(slice) in BF16, row-major and transposed, for d % 4 == 0 and
// ldt % 16 == 0 (16-byte stores): a block of 256 threads covers 32 rows x 128
// columns; each thread reads four consecutive columns of four rows (float4, 512
// bytes per warp row) and writes their BF16 values (8 bytes); the transposed copy
// goes through shared memory, each thread writing 16 consecutive rows of one
// column of xt (32 bytes, one sector).
constexpr int kFeatRows = 32, kFeatCols = 128;
__global__ void __launch_bounds__(256) k_fi_features_v(const float* __restrict__ src, int n, int d,
                                                       uint16_t* __restrict__ dst, uint16_t* __restrict__ dst_t,
                                                       int ldt) {
    pdl_wait();
    pdl_trigger();
    __shared__ uint16_t tile[kFeatRows][kFeatCols + 8];
    const int c0 = blockIdx.x * kFeatCols, r0 = blockIdx.y * kFeatRows;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    const int c = c0 + 4 * tx;
#pragma unroll
    for (int k = 0; k < kFeatRows / 8; ++k) {
        const int rr = ty + 8 * k, r = r0 + rr;
        uint2 packed = make_uint2(0u, 0u);
        if (r < n && c < d) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(src + (int64_t)r * d + c));
            packed.x = (uint32_t)to_bf16(log1pf(v.x)) | ((uint32_t)to_bf16(log1pf(v.y)) << 16);
            packed.y = (uint32_t)to_bf16(log1pf(v.z)) | ((uint32_t)to_bf16(log1pf(v.w)) << 16);
            if (dst) *reinterpret_cast<uint2*>(dst + (int64_t)r * d + c) = packed;
        }
        *reinterpret_cast<uint2*>(&tile[rr][4 * tx]) = packed;
    }
    if (!dst_t) return;
    __syncthreads();
    // thread t: column c0 + (t >> 1), rows r0 + 16 * (t & 1) .. + 15
    const int cc = threadIdx.x >> 1, half = threadIdx.x & 1;
    const int col = c0 + cc, rbase = r0 + 16 * half;
    if (col >= d) return;
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
        w[q] = (uint32_t)tile[16 * half + 2 * q][cc] | ((uint32_t)tile[16 * half + 2 * q + 1][cc] << 16);
    uint16_t* out = dst_t + (int64_t)col * ldt + rbase;
    if (rbase + 16 <= n) {
        reinterpret_cast<uint4*>(out)[0] = make_uint4(w[0], w[1], w[2], w[3]);
        reinterpret_cast<uint4*>(out)[1] = make_uint4(w[4], w[5], w[6], w[7]);
    } else {
        for (int q = 0; q < 16 && rbase + q < n; ++q) out[q] = (uint16_t)(w[q >> 1] >> (16 * (q & 1)));
    }
}

}  // namespace

cudaError_t launch_fi_features(const float* slices, int n, int d, uint16_t* x, uint16_t* xt, int ldt, cudaStream_t st) {
    const bool vec = d % 4 == 0 && ldt % 8 == 0 && (reinterpret_cast<uintptr_t>(slices) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(x) & 7) == 0 && (reinterpret_cast<uintptr_t>(xt) & 15) == 0;
    if (vec) {
        const dim3 grid((unsigned)((d + kFeatCols - 1) / kFeatCols), (unsigned)((n + kFeatRows - 1) / kFeatRows));
        launch_pdl(k_fi_features_v, grid, 256, 0, st, slices, n, d, x, xt, ldt);
    } else {
        launch_pdl(k_fi_convert_t<1>, tiles32(n, d), kT, 0, st, slices, n, d, x, xt, ldt);
    }
    return cudaGetLastError();
}

cudaError_t launch_fi_bias_act(float* z, const float* b, int n, int h, int act, uint16_t* hb, uint16_t* ht, int ldt,
                               float* out, cudaStream_t st) {
    launch_pdl(k_fi_bias_act, tiles32(n, h), kT, 0, st, z, b, n, h, act, hb, ht, ldt, out);
    return cudaGetLastError();
}

cudaError_t launch_fi_out_grad(const float* out, const float* t, const float* z, int64_t n_el, float inv_count,
                               float* g, double* part, int n_part, cudaStream_t st) {
    launch_pdl(k_fi_out_grad, n_part, kT, 0, st, out, t, z, n_el, inv_count, g, part);
    return cudaGetLastError();
}

cudaError_t launch_fi_relu_grad(float* g, const float* z, int n, int h, uint16_t* gb, uint16_t* gt, int ldt,
                                cudaStream_t st) {
    launch_pdl(k_fi_relu_grad, tiles32(n, h), kT, 0, st, g, z, n, h, gb, gt, ldt);
    return cudaGetLastError();
}

cudaError_t launch_fi_convert(const float* src, int n, int d, uint16_t* dst, uint16_t* dst_t, int ldt,
                              cudaStream_t st) {
    launch_pdl(k_fi_convert_t<0>, tiles32(n, d), kT, 0, st, src, n, d, dst, dst_t, ldt);
    return cudaGetLastError();
}

cudaError_t launch_fi_colsum(const float* g, int n, int h, float* out, cudaStream_t st) {
    launch_pdl(k_fi_colsum, (h + 31) / 32, 32 * kColsumWarps, 0, st, g, n, h, out);
    return cudaGetLastError();
}

cudaError_t launch_fi_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                           float eps, float bc1, float bc2, cudaStream_t st) {
    launch_pdl(k_fi_adam, (unsigned)((n + kT - 1) / kT), kT, 0, st, p, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
    return cudaGetLastError();
}

cudaError_t launch_fi_adam_t(float* p, const float* g, float* m, float* v, int rows, int cols, float lr, float b1,
                             float b2, float eps, float bc1, float bc2, uint16_t* dst_t, cudaStream_t st) {
    launch_pdl(k_fi_adam_t, tiles32(rows, cols), kT, 0, st, p, g, m, v, rows, cols, lr, b1, b2, eps, bc1, bc2, dst_t);
    return cudaGetLastError();
}

cudaError_t launch_fi_weight_copy(const float* w, int rows, int cols, uint16_t* dst, uint16_t* dst_t,
                                  cudaStream_t st) {
    launch_pdl(k_fi_weight_copy, tiles32(rows, cols), kT, 0, st, w, rows, cols, dst, dst_t);
    return cudaGetLastError();
}

}  // namespace nef
