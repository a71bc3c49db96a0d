// k_view_simt.cuh -- CUDA-core fused pass (FP32 or FP64) of one factor update.
//
// For a tile of TM rows x TN columns of the view Y[row, col]:
//   yhat = P_tile . Q_tile^T                       (Eq. 2.1, factorised through the bond)
//   W_a = M * a(y, yhat),  W_b = M * b(y, yhat)     (App. B weights, masked)
//   S_a += W_a . Q_tile,   S_b += W_b . Q_tile      (the contraction of Eq. 3.6-3.8)
// yhat, W_a and W_b live only in registers and shared memory.  Each CTA owns one
// row block and a range of columns and writes its partial S to
// s_num/s_den[split][row][bond_pad]; the loss (optional) is accumulated in FP64.
#pragma once
#include <algorithm>

#include "nef_device.cuh"
#include "nef_internal.h"
#include "nef_launch.cuh"

namespace nef {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int64_t src_row(const SrcDesc& s, int64_t i) {
    int64_t r = 0;
    for (int t = 0; t < s.nterm; ++t) r += ((i / s.div[t]) % s.mod[t]) * s.mul[t];
    return r;
}

template <typename T>
__device__ __forceinline__ T side_value(const SideDesc& sd, int64_t i, int b) {
    T p = T(1);
    for (int s = 0; s < sd.nsrc; ++s) {
        const T* base = static_cast<const T*>(sd.src[s].ptr);
        p *= base[src_row(sd.src[s], i) * sd.src[s].ld + b];
    }
    return p;
}

template <typename T, int TM, int TN, int BP, bool DEN, bool GEMM2, bool LOSS>
__global__ void __launch_bounds__(kThreads)
k_view_simt(const T* __restrict__ y, const uint32_t* __restrict__ mbits, ViewDesc v, WeightSpec w,
            LossSpec L, int64_t cols_per_split, T* __restrict__ s_num, T* __restrict__ s_den,
            double* __restrict__ loss_part) {
    pdl_wait();
    pdl_trigger();
    constexpr int PAD = 4;
    constexpr int MR = TM / 16, NR = TN / 16;
    constexpr int SR = (TM * BP) / 1024;
    constexpr int SXN = BP / 4;  // threads across the bond in the second product
    static_assert(SR >= 1, "tile too small for the bond");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Pb = reinterpret_cast<T*>(smem_raw);     // [BP][TM+PAD]
    T* Qb = Pb + BP * (TM + PAD);                // [BP][TN+PAD]
    T* Qc = Qb + BP * (TN + PAD);                // [TN][BP+PAD]
    T* Ys = Qc + TN * (BP + PAD);                // [TM][TN+PAD]
    T* Wa = Ys + TM * (TN + PAD);                // [TN][TM+PAD]
    T* Wb = Wa + TN * (TM + PAD);                // [TN][TM+PAD]
    int64_t* coff = reinterpret_cast<int64_t*>(Wb + (DEN ? TN * (TM + PAD) : 0));  // [TN]
    int64_t* qrow = coff + TN;                                                     // [kMaxSrc][TN]

    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int sx = tid % SXN, sy = tid / SXN;
    const int64_t n_rb = (v.rows + TM - 1) / TM;
    const int64_t rb = blockIdx.x % n_rb;
    const int64_t sp = blockIdx.x / n_rb;
    const int64_t r0 = rb * TM;
    const int64_t n_cols = v.c_out * v.c_in;
    const int64_t c_lo = sp * cols_per_split;
    const int64_t c_hi = min(c_lo + cols_per_split, n_cols);
    const bool trans = (v.c_in == 1);

    for (int e = tid; e < TM * BP; e += kThreads) {
        const int r = e / BP, b = e % BP;
        const int64_t row = r0 + r;
        T p = T(0);
        if (row < v.rows && b < v.bond) p = side_value<T>(v.P, row, b);
        Pb[b * (TM + PAD) + r] = p;
    }

    T sa[SR][4], sb[SR][4];
#pragma unroll
    for (int i = 0; i < SR; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { sa[i][j] = T(0); sb[i][j] = T(0); }
    double lsum = 0.0, lcnt = 0.0;

    for (int64_t c0 = c_lo; c0 < c_hi; c0 += TN) {
        __syncthreads();
        if (tid < TN) {
            const int64_t col = c0 + tid;
            const bool ok = col < c_hi;
            coff[tid] = ok ? (col / v.c_in) * v.rows * v.c_in + (col % v.c_in) : -1;
            for (int s = 0; s < v.Q.nsrc; ++s) qrow[s * TN + tid] = ok ? src_row(v.Q.src[s], col) : 0;
        }
        __syncthreads();
        for (int e = tid; e < TN * BP; e += kThreads) {
            const int c = e / BP, b = e % BP;
            T q = T(0);
            if (coff[c] >= 0 && b < v.bond) {
                q = T(1);
                for (int s = 0; s < v.Q.nsrc; ++s)
                    q *= static_cast<const T*>(v.Q.src[s].ptr)[qrow[s * TN + c] * v.Q.src[s].ld + b];
            }
            Qb[b * (TN + PAD) + c] = q;
            Qc[c * (BP + PAD) + b] = q;
        }
        __syncthreads();
        for (int e = tid; e < TM * TN; e += kThreads) {
            int r, c;
            if (trans) { r = e % TM; c = e / TM; } else { c = e % TN; r = e / TN; }
            const int64_t row = r0 + r;
            const int64_t co = coff[c];
            T val = T(-1);
            if (row < v.rows && co >= 0) {
                const int64_t idx = co + row * v.c_in;
                val = y[idx];
                if (mbits && !mask_bit(mbits, idx)) val = T(-1);
            }
            Ys[r * (TN + PAD) + c] = val;
        }
        __syncthreads();

        T acc[MR][NR];
#pragma unroll
        for (int i = 0; i < MR; ++i)
#pragma unroll
            for (int j = 0; j < NR; ++j) acc[i][j] = T(0);
#pragma unroll 4
        for (int b = 0; b < BP; ++b) {
            T pv[MR], qv[NR];
#pragma unroll
            for (int i = 0; i < MR; ++i) pv[i] = Pb[b * (TM + PAD) + ty * MR + i];
#pragma unroll
            for (int j = 0; j < NR; ++j) qv[j] = Qb[b * (TN + PAD) + tx * NR + j];
#pragma unroll
            for (int i = 0; i < MR; ++i)
#pragma unroll
                for (int j = 0; j < NR; ++j) acc[i][j] = fma(pv[i], qv[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < MR; ++i) {
#pragma unroll
            for (int j = 0; j < NR; ++j) {
                const int r = ty * MR + i, c = tx * NR + j;
                const T yv = Ys[r * (TN + PAD) + c];
                T a = T(0), bb = T(0);
                if (yv >= T(0)) {
                    ab_weights(yv, acc[i][j], w, a, bb);
                    if (LOSS) {
                        lsum += (double)divergence(yv, acc[i][j], L);
                        lcnt += 1.0;
                    }
                }
                if (GEMM2) {
                    Wa[c * (TM + PAD) + r] = a;
                    if (DEN) Wb[c * (TM + PAD) + r] = bb;
                }
            }
        }
        if (GEMM2) {
            __syncthreads();
#pragma unroll 4
            for (int k = 0; k < TN; ++k) {
                T qv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) qv[j] = Qc[k * (BP + PAD) + sx * 4 + j];
#pragma unroll
                for (int i = 0; i < SR; ++i) {
                    const T wa = Wa[k * (TM + PAD) + sy * SR + i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) sa[i][j] = fma(wa, qv[j], sa[i][j]);
                    if (DEN) {
                        const T wb = Wb[k * (TM + PAD) + sy * SR + i];
#pragma unroll
                        for (int j = 0; j < 4; ++j) sb[i][j] = fma(wb, qv[j], sb[i][j]);
                    }
                }
            }
        }
    }

    if (GEMM2) {
#pragma unroll
        for (int i = 0; i < SR; ++i) {
            const int64_t row = r0 + sy * SR + i;
            if (row >= v.rows) continue;
            const int64_t base = (sp * v.rows + row) * BP + sx * 4;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                s_num[base + j] = sa[i][j];
                if (DEN) s_den[base + j] = sb[i][j];
            }
        }
    }
    if (LOSS) {
        __shared__ double sh[2][kThreads / 32];
        lsum = warp_sum(lsum);
        lcnt = warp_sum(lcnt);
        if ((tid & 31) == 0) { sh[0][tid >> 5] = lsum; sh[1][tid >> 5] = lcnt; }
        __syncthreads();
        if (tid == 0) {
            double s = 0.0, c = 0.0;
            for (int k = 0; k < kThreads / 32; ++k) { s += sh[0][k]; c += sh[1][k]; }
            loss_part[blockIdx.x] = s;
            loss_part[gridDim.x + blockIdx.x] = c;
        }
    }
}

template <typename T, int TM, int TN, int BP>
size_t smem_bytes(bool den) {
    constexpr int PAD = 4;
    size_t n = (size_t)BP * (TM + PAD) + (size_t)BP * (TN + PAD) + (size_t)TN * (BP + PAD) +
               (size_t)TM * (TN + PAD) + (size_t)TN * (TM + PAD) * (den ? 2 : 1);
    return n * sizeof(T) + (1 + kMaxSrc) * TN * sizeof(int64_t);
}

template <typename T, int TM, int TN, int BP, bool DEN, bool GEMM2, bool LOSS>
cudaError_t run(const T* y, const uint32_t* mbits, const ViewDesc& v, const WeightSpec& w,
                const LossSpec& L, int n_split, T* s_num, T* s_den, double* loss_part,
                cudaStream_t st, int* n_ctas_out) {
    const int64_t n_rb = (v.rows + TM - 1) / TM;
    const int64_t n_cols = v.c_out * v.c_in;
    int64_t tiles = (n_cols + TN - 1) / TN;
    int64_t per = (tiles + n_split - 1) / n_split;
    const int64_t cols_per_split = per * TN;
    const size_t sm = smem_bytes<T, TM, TN, BP>(DEN);
    auto kern = k_view_simt<T, TM, TN, BP, DEN, GEMM2, LOSS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int64_t n_ctas = n_rb * n_split;
    if (n_ctas_out) *n_ctas_out = (int)n_ctas;
    launch_pdl(kern, (unsigned)n_ctas, kThreads, sm, st, y, mbits, v, w, L, cols_per_split, s_num, s_den,
                                                  loss_part);
    return cudaGetLastError();
}

template <typename T, int TM, int TN, int BP>
cudaError_t dispatch_flags(const T* y, const uint32_t* mbits, const ViewDesc& v,
                           const WeightSpec& w, int need_den, int n_split, T* s_num, T* s_den,
                           const LossSpec* loss, double* loss_part, cudaStream_t st, int* n_ctas) {
    LossSpec L{};
    if (loss) L = *loss;
    if (s_num == nullptr) {  // loss-only pass (nef_loss)
        if (!loss) return cudaErrorInvalidValue;
        return run<T, TM, TN, BP, false, false, true>(y, mbits, v, w, L, n_split, s_num, s_den,
                                                      loss_part, st, n_ctas);
    }
    if (loss) {  // update pass that also sums the loss of the current factors
        if (need_den)
            return run<T, TM, TN, BP, true, true, true>(y, mbits, v, w, L, n_split, s_num, s_den,
                                                        loss_part, st, n_ctas);
        return run<T, TM, TN, BP, false, true, true>(y, mbits, v, w, L, n_split, s_num, s_den,
                                                     loss_part, st, n_ctas);
    }
    if (need_den)
        return run<T, TM, TN, BP, true, true, false>(y, mbits, v, w, L, n_split, s_num, s_den,
                                                     loss_part, st, n_ctas);
    return run<T, TM, TN, BP, false, true, false>(y, mbits, v, w, L, n_split, s_num, s_den,
                                                  loss_part, st, n_ctas);
}

}  // namespace

#define NEF_SIMT_INSTANCE(NAME, T, TM, BP)                                                       \
    cudaError_t NAME(const T* y, const uint32_t* mbits, const ViewDesc& v, const WeightSpec& w, \
                     int need_den, int n_split, T* s_num, T* s_den, const LossSpec* loss,       \
                     double* loss_part, cudaStream_t st, int* n_ctas) {                         \
        return dispatch_flags<T, TM, TM, BP>(y, mbits, v, w, need_den, n_split, s_num, s_den,   \
                                             loss, loss_part, st, n_ctas);                      \
    }

}  // namespace nef
