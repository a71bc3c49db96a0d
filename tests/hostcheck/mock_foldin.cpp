// Plain-loop implementations of the fold-in encoder's launchers (nef_internal.h:
// launch_gemm_nt and launch_fi_*), following each kernel's documented meaning,
// so that foldin.cpp (buffer layout, the forward and backward orchestration,
// the transposed copies, Adam and the loss read-back) can be checked against
// the FP64 oracle MLP on a CPU host.
// TEST INFRASTRUCTURE ONLY: built by tests/hostcheck/build.py into a separate
// library that the product never loads.  BF16 copies are rounded to nearest
// even, as the kernels write them; products accumulate in FP32.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "nef_internal.h"

namespace nef {

namespace {

uint16_t bf16_bits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

float bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

float softplus(float z) { return z > 30.f ? z : std::log1p(std::exp(z)); }
float sigmoid(float z) { return 1.f / (1.f + std::exp(-z)); }

// row-major [n x d] BF16 copy and its transpose [d x ldt]
void write_pair(uint16_t* dst, uint16_t* dst_t, int64_t ldt, int n, int d, int64_t r, int64_t c, uint16_t v) {
    if (dst) dst[r * d + c] = v;
    if (dst_t) dst_t[c * ldt + r] = v;
}

}  // namespace

int gemm_splits(int M, int N, int K, int n_sm) {
    // the split count changes nothing in the host double's product; any value will do
    const int64_t tiles = (int64_t)((M + 127) / 128) * ((N + 127) / 128);
    const int nk = (K + 63) / 64;
    int64_t s = std::max<int64_t>(1, n_sm / std::max<int64_t>(1, tiles));
    s = std::min<int64_t>(s, std::max(1, nk / 8));
    return (int)std::min<int64_t>(s, 16);
}

// The split count changes only the order of the FP32 sums, not the product.
cudaError_t launch_gemm_nt(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* C, int64_t ldc,
                           int M, int N, int K, int accumulate, int*, cudaStream_t, float*, int64_t, int) {
    return host_submit([=]() -> cudaError_t {
        for (int i = 0; i < M; ++i)
            for (int j = 0; j < N; ++j) {
                float acc = 0.f;
                for (int k = 0; k < K; ++k) acc += bf16_value(A[(int64_t)i * lda + k]) * bf16_value(B[(int64_t)j * ldb + k]);
                float& c = C[(int64_t)i * ldc + j];
                c = accumulate ? c + acc : acc;
            }
        return cudaSuccess;
    });
}

cudaError_t launch_fi_features(const float* slices, int n, int d, uint16_t* x, uint16_t* xt, int ldt, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        for (int64_t r = 0; r < n; ++r)
            for (int64_t c = 0; c < d; ++c)
                write_pair(x, xt, ldt, n, d, r, c, bf16_bits(std::log1p(slices[r * d + c])));
        return cudaSuccess;
    });
}

cudaError_t launch_fi_bias_act(float* z, const float* b, int n, int h, int act, uint16_t* hb, uint16_t* ht, int ldt,
                               float* out, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        for (int64_t r = 0; r < n; ++r)
            for (int64_t c = 0; c < h; ++c) {
                const int64_t e = r * h + c;
                z[e] += b[c];
                if (act == 1) write_pair(hb, ht, ldt, n, h, r, c, bf16_bits(std::max(z[e], 0.f)));
                else out[e] = softplus(z[e]);
            }
        return cudaSuccess;
    });
}

cudaError_t launch_fi_out_grad(const float* out, const float* t, const float* z, int64_t n_el, float inv_count,
                               float* g, double* part, int n_part, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        double acc = 0.0;
        for (int64_t e = 0; e < n_el; ++e) {
            const float d = std::log1p(out[e]) - std::log1p(t[e]);
            acc += (double)d * d;
            if (g) g[e] = 2.f * d / (1.f + out[e]) * inv_count * sigmoid(z[e]);
        }
        for (int k = 0; k < n_part; ++k) part[k] = k == 0 ? acc : 0.0;
        return cudaSuccess;
    });
}

cudaError_t launch_fi_relu_grad(float* g, const float* z, int n, int h, uint16_t* gb, uint16_t* gt, int ldt,
                                cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        for (int64_t r = 0; r < n; ++r)
            for (int64_t c = 0; c < h; ++c) {
                const int64_t e = r * h + c;
                g[e] = z[e] > 0.f ? g[e] : 0.f;
                write_pair(gb, gt, ldt, n, h, r, c, bf16_bits(g[e]));
            }
        return cudaSuccess;
    });
}

cudaError_t launch_fi_convert(const float* src, int n, int d, uint16_t* dst, uint16_t* dst_t, int ldt,
                              cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        for (int64_t r = 0; r < n; ++r)
            for (int64_t c = 0; c < d; ++c) write_pair(dst, dst_t, ldt, n, d, r, c, bf16_bits(src[r * d + c]));
        return cudaSuccess;
    });
}

cudaError_t launch_fi_colsum(const float* g, int n, int h, float* out, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        for (int64_t c = 0; c < h; ++c) {
            float s = 0.f;
            for (int64_t r = 0; r < n; ++r) s += g[r * h + c];
            out[c] = s;
        }
        return cudaSuccess;
    });
}

cudaError_t launch_fi_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                           float eps, float bc1, float bc2, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        for (int64_t e = 0; e < n; ++e) {
            m[e] = b1 * m[e] + (1.f - b1) * g[e];
            v[e] = b2 * v[e] + (1.f - b2) * g[e] * g[e];
            p[e] -= lr * (m[e] / bc1) / (std::sqrt(v[e] / bc2) + eps);
        }
        return cudaSuccess;
    });
}

cudaError_t launch_fi_adam_t(float* p, const float* g, float* m, float* v, int rows, int cols, float lr, float b1,
                             float b2, float eps, float bc1, float bc2, uint16_t* dst_t, cudaStream_t st) {
    const int64_t n = (int64_t)rows * cols;
    cudaError_t e = launch_fi_adam(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2, st);
    if (e != cudaSuccess) return e;
    return launch_fi_weight_copy(p, rows, cols, nullptr, dst_t, st);
}

cudaError_t launch_fi_weight_copy(const float* w, int rows, int cols, uint16_t* dst, uint16_t* dst_t,
                                  cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        for (int64_t r = 0; r < rows; ++r)
            for (int64_t c = 0; c < cols; ++c) write_pair(dst, dst_t, rows, rows, cols, r, c, bf16_bits(w[r * cols + c]));
        return cudaSuccess;
    });
}

}  // namespace nef
