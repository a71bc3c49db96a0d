// k_common.cu -- small kernels of the sweep: the generic einsum used for operand
// preparation and epilogues (Eq. 3.8 with S in place of the weighted tensor),
// mask packing, the data check, split reductions, the update of Eq. 3.4, and the
// unfused fallback that materialises yhat, a(Y,Yhat), b(Y,Yhat) (Algorithm 1 as
// written) for model strings the fused view cannot express.
#include <algorithm>
#include <type_traits>

#include "nef_device.cuh"
#include "nef_internal.h"
#include "nef_launch.cuh"

namespace nef {

long long kernel_launches() { return g_kernel_launches.load(std::memory_order_relaxed); }

namespace {

constexpr int kThreads = 256;

// Destination write of a contraction: out (= or +=), and with out16 the BF16 copy
// and the FP32 value rounded to it (round to nearest even).
template <typename T>
__device__ __forceinline__ void ein_store(const EinDesc& d, void* outp, int64_t dst, T acc) {
    T* out = static_cast<T*>(outp);
    if constexpr (std::is_same<T, float>::value) {
        if (d.out16) {
            const uint32_t u = __float_as_uint(acc);
            const uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);
            d.out16[dst] = (uint16_t)(r >> 16);
            out[dst] = __uint_as_float(r & 0xffff0000u);
            return;
        }
    }
    out[dst] = d.accumulate ? out[dst] + acc : acc;
}

// The index arrays below are walked with loops unrolled over their fixed sizes (and
// guarded by the descriptor's counts), so they stay in registers; the descriptor is a
// __grid_constant__ parameter, read in place.

// Adds the offsets of letters q_lo..q_hi-1 decoded from r (the last letter fastest) to
// every operand's offset, and to *dst with the destination strides.
__device__ __forceinline__ void ein_decode(const EinDesc& d, int q_lo, int q_hi, uint32_t r,
                                           int64_t (&off)[kMaxEinOps], int64_t* dst) {
    for (int q = q_hi - 1; q >= q_lo; --q) {
        const uint32_t dq = (uint32_t)d.dim[q];
        const int64_t v = r % dq;
        r /= dq;
        if (dst) *dst += v * d.out_st[q];
#pragma unroll
        for (int k = 0; k < kMaxEinOps; ++k)
            if (k < d.n_ops) off[k] += v * d.ost[k][q];
    }
}

// Operand 0 at offset off: the value, or the sum of its split partials in split order.
template <typename T>
__device__ __forceinline__ T ein_op0(const EinDesc& d, const void* base, int64_t off) {
    const T* p = static_cast<const T*>(base) + off;
    T v = p[0];
    for (int s = 1; s < d.op0_splits; ++s) v += p[(int64_t)s * d.op0_split_stride];
    return v;
}

// Product of the operands at one free combination: all of them into acc, or (DUAL)
// operand 0 times the rest into acc and operand 0b times the rest into accb.
template <typename T, bool DUAL>
__device__ __forceinline__ void ein_term(const EinDesc& d, const int64_t (&off)[kMaxEinOps], T& acc, T& accb) {
    T p = T(1);
#pragma unroll
    for (int k = 1; k < kMaxEinOps; ++k)
        if (k < d.n_ops) p *= static_cast<const T*>(d.op[k])[off[k]];
    if constexpr (DUAL) {
        acc += ein_op0<T>(d, d.op[0], off[0]) * p;
        accb += ein_op0<T>(d, d.op0b, off[0]) * p;
    } else {
        acc += ein_op0<T>(d, d.op[0], off[0]) * p;
    }
}

// Steps the free letters' multi-index (the last fastest) by one, moving the offsets.
__device__ __forceinline__ void ein_step(const EinDesc& d, int32_t (&idx)[kMaxEinLet], int64_t (&off)[kMaxEinOps]) {
#pragma unroll
    for (int q = kMaxEinLet - 1; q >= 0; --q) {
        if (q < d.n_out || q >= d.n_out + d.n_free) continue;
        idx[q] += 1;
#pragma unroll
        for (int k = 0; k < kMaxEinOps; ++k)
            if (k < d.n_ops) off[k] += d.ost[k][q];
        if (idx[q] < d.dim[q]) break;
#pragma unroll
        for (int k = 0; k < kMaxEinOps; ++k)
            if (k < d.n_ops) off[k] -= d.ost[k][q] * d.dim[q];
        idx[q] = 0;
    }
}

template <typename T>
__global__ void k_einsum_part(const __grid_constant__ EinDesc d, int64_t chunk, T* partial) {
    pdl_wait();
    pdl_trigger();
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int sp = blockIdx.y;
    if (o >= d.n_out_el) return;
    int64_t off[kMaxEinOps];
#pragma unroll
    for (int k = 0; k < kMaxEinOps; ++k) off[k] = 0;
    ein_decode(d, 0, d.n_out, (uint32_t)o, off, nullptr);  // n_out_el < 2^31 (checked at launch)
    const int64_t f0 = (int64_t)sp * chunk;
    const int64_t f1 = min(f0 + chunk, d.n_free_el);
    int32_t idx[kMaxEinLet];
    int64_t frem = f0;
#pragma unroll
    for (int q = kMaxEinLet - 1; q >= 0; --q) {
        idx[q] = 0;
        if (q < d.n_out || q >= d.n_out + d.n_free) continue;
        idx[q] = (int32_t)(frem % d.dim[q]);
        frem /= d.dim[q];
#pragma unroll
        for (int k = 0; k < kMaxEinOps; ++k)
            if (k < d.n_ops) off[k] += (int64_t)idx[q] * d.ost[k][q];
    }
    T acc = T(0), unused = T(0);
    for (int64_t f = f0; f < f1; ++f) {
        ein_term<T, false>(d, off, acc, unused);
        ein_step(d, idx, off);
    }
    partial[(int64_t)sp * d.n_out_el + o] = acc;
}

// Single-split contraction: one thread per output element (false past the last).
template <typename T, bool DUAL>
__device__ __forceinline__ bool ein_direct_eval(const EinDesc& d, int64_t& dst, T& acc, T& accb) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= d.n_out_el) return false;
    int64_t off[kMaxEinOps];
#pragma unroll
    for (int k = 0; k < kMaxEinOps; ++k) off[k] = 0;
    dst = 0;
    ein_decode(d, 0, d.n_out, (uint32_t)o, off, &dst);  // n_out_el < 2^31 (checked at launch)
    int32_t idx[kMaxEinLet];
#pragma unroll
    for (int q = 0; q < kMaxEinLet; ++q) idx[q] = 0;
    acc = T(0);
    accb = T(0);
    for (int64_t f = 0; f < d.n_free_el; ++f) {
        ein_term<T, DUAL>(d, off, acc, accb);
        ein_step(d, idx, off);
    }
    return true;
}

// Single-split contraction written straight to the destination layout.
template <typename T, bool DUAL>
__global__ void k_einsum_direct(const __grid_constant__ EinDesc d) {
    pdl_wait();
    pdl_trigger();
    int64_t dst;
    T acc, accb;
    if (!ein_direct_eval<T, DUAL>(d, dst, acc, accb)) return;
    ein_store<T>(d, d.out, dst, acc);
    if constexpr (DUAL) ein_store<T>(d, d.outb, dst, accb);
}

// Sum over the G threads of a group in a fixed order (xor shuffles within a warp; for
// G = 256 the warp sums are added in warp order).
template <typename T, int G>
__device__ __forceinline__ T group_sum(T acc, T* sh) {
    if constexpr (G <= 32) {
#pragma unroll
        for (int w = G / 2; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
    } else {
        static_assert(G == kThreads, "group size");
        acc = warp_sum(acc);
        __syncthreads();  // sh free from a previous use
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
        __syncthreads();
        acc = T(0);
        for (int k = 0; k < kThreads / 32; ++k) acc += sh[k];
    }
    return acc;
}

// Contraction with G threads per output element: the threads of a group take the
// free combinations f = sub, sub + G, ... (each decodes its own f) and the group
// sums its partials.  Used where G threads cover an output's free combinations in a
// few steps (at most 4 for G = 8 and 32, 64 for G = 256).  Returns true for the
// thread that writes the output.
template <typename T, int G, bool DUAL>
__device__ __forceinline__ bool ein_grouped_eval(const EinDesc& d, T* sh, int64_t& dst, T& acc, T& accb) {
    constexpr int kGroups = kThreads / G;
    const int sub = (int)(threadIdx.x % G);
    const int64_t o = (int64_t)blockIdx.x * kGroups + threadIdx.x / G;
    const bool ok = o < d.n_out_el;
    acc = T(0);
    accb = T(0);
    dst = 0;
    if (ok) {
        int64_t base[kMaxEinOps];
#pragma unroll
        for (int k = 0; k < kMaxEinOps; ++k) base[k] = 0;
        ein_decode(d, 0, d.n_out, (uint32_t)o, base, &dst);  // n_out_el < 2^31 (checked at launch)
#pragma unroll 2
        for (int64_t f = sub; f < d.n_free_el; f += G) {
            int64_t off[kMaxEinOps];
#pragma unroll
            for (int k = 0; k < kMaxEinOps; ++k) off[k] = base[k];
            ein_decode(d, d.n_out, d.n_out + d.n_free, (uint32_t)f, off, nullptr);  // n_free_el < 2^31 here
            ein_term<T, DUAL>(d, off, acc, accb);
        }
    }
    acc = group_sum<T, G>(acc, sh);
    if constexpr (DUAL) accb = group_sum<T, G>(accb, sh);
    return ok && sub == 0;
}

template <typename T, int G, bool DUAL>
__global__ void __launch_bounds__(kThreads) k_einsum_grouped(const __grid_constant__ EinDesc d) {
    pdl_wait();
    pdl_trigger();
    __shared__ T sh[kThreads / 32];
    int64_t dst;
    T acc, accb;
    if (ein_grouped_eval<T, G, DUAL>(d, sh, dst, acc, accb)) {
        ein_store<T>(d, d.out, dst, acc);
        if constexpr (DUAL) ein_store<T>(d, d.outb, dst, accb);
    }
}

template <typename T>
__global__ void k_einsum_final(const __grid_constant__ EinDesc d, int n_split, const T* partial) {
    pdl_wait();
    pdl_trigger();
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= d.n_out_el) return;
    T acc = T(0);
    for (int s = 0; s < n_split; ++s) acc += partial[(int64_t)s * d.n_out_el + o];
    int64_t dst = 0;
    uint32_t rem = (uint32_t)o;  // n_out_el < 2^31 (checked at launch)
    for (int q = d.n_out - 1; q >= 0; --q) {
        const uint32_t dq = (uint32_t)d.dim[q];
        dst += (int64_t)(rem % dq) * d.out_st[q];
        rem /= dq;
    }
    ein_store<T>(d, d.out, dst, acc);
}

__global__ void k_pack_mask(const uint8_t* __restrict__ m, int64_t n, uint32_t* __restrict__ bits) {
    pdl_wait();
    pdl_trigger();
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nw = (n + 31) >> 5;
    if (w >= nw) return;
    uint32_t v = 0;
    const int64_t e0 = w << 5;
    for (int b = 0; b < 32; ++b) {
        const int64_t e = e0 + b;
        if (e < n && m[e]) v |= (1u << b);
    }
    bits[w] = v;
}

template <typename T>
__global__ void k_check_data(const T* __restrict__ y, int64_t n, int* flag) {
    pdl_wait();
    pdl_trigger();
    int bad = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
        T v = y[e];
        if (!(v >= T(0)) || isinf((double)v)) bad = 1;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

template <typename T>
__global__ void k_reduce_splits(const T* __restrict__ part, int n_split, int64_t n, T* __restrict__ out) {
    pdl_wait();
    pdl_trigger();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    T acc = T(0);
    for (int s = 0; s < n_split; ++s) acc += part[(int64_t)s * n + e];
    out[e] = acc;
}

template <typename T>
__global__ void k_reduce_splits2(const T* __restrict__ part_a, const T* __restrict__ part_b, int n_split, int64_t n,
                                 T* __restrict__ out_a, T* __restrict__ out_b) {
    pdl_wait();
    pdl_trigger();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * n) return;
    const bool b = e >= n;
    const int64_t i = b ? e - n : e;
    const T* part = b ? part_b : part_a;
    T acc = T(0);
    for (int s = 0; s < n_split; ++s) acc += part[(int64_t)s * n + i];
    (b ? out_b : out_a)[i] = acc;
}

template <typename T>
__global__ void k_update(T* __restrict__ theta, const T* __restrict__ num, const T* __restrict__ den,
                         int64_t n, UpdateSpec u) {
    pdl_wait();
    pdl_trigger();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    theta[e] = mu_update(theta[e], num[e], den[e], u);
}

template <typename T>
__global__ void k_fill(T* p, int64_t n, T v) {
    pdl_wait();
    pdl_trigger();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) p[e] = v;
}

__global__ void k_sum_f64(const double* __restrict__ part, int n, double* out) {
    pdl_wait();
    pdl_trigger();
    __shared__ double sh[32];
    double acc = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) acc += part[k];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) out[0] = v;
    }
}

// out[0..1] = sums of part[0..n) and part[n..2n) (loss, observed count); the
// loss is also written to trace[*count] (if trace) and *count is incremented.
__global__ void k_loss_append(const double* __restrict__ part, int n, double* trace, int* count, double* out) {
    pdl_wait();
    pdl_trigger();
    __shared__ double sh[2][32];
    double a = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        a += part[k];
        c += part[n + k];
    }
    a = warp_sum(a);
    c = warp_sum(c);
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = a;
        sh[1][threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        const bool ok = threadIdx.x < (blockDim.x >> 5);
        double va = ok ? sh[0][threadIdx.x] : 0.0, vc = ok ? sh[1][threadIdx.x] : 0.0;
        va = warp_sum(va);
        vc = warp_sum(vc);
        if (threadIdx.x == 0) {
            out[0] = va;
            out[1] = vc;
            if (trace) trace[*count] = va;
            *count += 1;
        }
    }
}

// BF16 copy of an operand, and the FP32 operand replaced by the same rounded
// values, so that whatever else reads the FP32 copy (closed-form denominators,
// epilogue contractions) sees exactly the operand the tensor cores multiply.
__global__ void k_convert_bf16(float* __restrict__ src, int64_t n, uint16_t* __restrict__ dst) {
    pdl_wait();
    pdl_trigger();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    // round to nearest even
    uint32_t u = __float_as_uint(src[e]);
    uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);
    dst[e] = (uint16_t)(r >> 16);
    src[e] = __uint_as_float(r & 0xffff0000u);
}

// Unfused path: yhat at every entry by a loop over all latent combinations,
// then the masked weights and (optionally) the divergence.
template <typename T>
__global__ void k_generic_weights(GenericRecon g, const T* __restrict__ y, const uint32_t* mbits,
                                  WeightSpec w, T* __restrict__ wa, T* __restrict__ wb,
                                  int has_loss, LossSpec L, double* loss_part) {
    pdl_wait();
    pdl_trigger();
    __shared__ double sh_loss[kThreads / 32];
    __shared__ double sh_cnt[kThreads / 32];
    double lsum = 0.0, lcnt = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < g.n;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t idx[kMaxLet];
        int64_t rem = e;
        for (int m = g.n_obs - 1; m >= 0; --m) {
            idx[m] = rem % g.dim[m];
            rem /= g.dim[m];
        }
        int64_t off[kMaxFac];
        for (int f = 0; f < g.n_fac; ++f) {
            off[f] = 0;
            for (int m = 0; m < g.n_obs; ++m) off[f] += idx[m] * g.fst[f][m];
        }
        for (int x = g.n_obs; x < g.n_let; ++x) idx[x] = 0;
        T yh = T(0);
        for (int64_t c = 0; c < g.n_lat_el; ++c) {
            T p = T(1);
            for (int f = 0; f < g.n_fac; ++f) p *= static_cast<const T*>(g.fac[f])[off[f]];
            yh += p;
            for (int x = g.n_let - 1; x >= g.n_obs; --x) {
                idx[x] += 1;
                for (int f = 0; f < g.n_fac; ++f) off[f] += g.fst[f][x];
                if (idx[x] < g.dim[x]) break;
                for (int f = 0; f < g.n_fac; ++f) off[f] -= g.fst[f][x] * g.dim[x];
                idx[x] = 0;
            }
        }
        const int obs = mbits ? mask_bit(mbits, e) : 1;
        const T yv = y[e];
        T a = T(0), b = T(0);
        if (obs) {
            ab_weights(yv, yh, w, a, b);
            if (has_loss) {
                lsum += (double)divergence(yv, yh, L);
                lcnt += 1.0;
            }
        }
        if (wa) wa[e] = a;
        if (wb) wb[e] = b;
    }
    if (has_loss) {
        lsum = warp_sum(lsum);
        lcnt = warp_sum(lcnt);
        if ((threadIdx.x & 31) == 0) {
            sh_loss[threadIdx.x >> 5] = lsum;
            sh_cnt[threadIdx.x >> 5] = lcnt;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0, c = 0.0;
            for (int k = 0; k < kThreads / 32; ++k) { s += sh_loss[k]; c += sh_cnt[k]; }
            loss_part[blockIdx.x] = s;
            loss_part[gridDim.x + blockIdx.x] = c;
        }
    }
}

__device__ __forceinline__ uint16_t bf16_bits(float x) {
    uint32_t u = __float_as_uint(x);
    uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);  // round to nearest even (finite inputs)
    return (uint16_t)(r >> 16);
}

template <typename T>
__device__ __forceinline__ void decode_letters(int64_t e, int nlet, const int64_t* dim, int64_t (&idx)[kMaxFacLet]) {
#pragma unroll
    for (int q = kMaxFacLet - 1; q >= 0; --q) {
        idx[q] = 0;
        if (q >= nlet) continue;
        idx[q] = e % dim[q];
        e /= dim[q];
    }
}

// The factor's operand copies.  A copy with a BF16 twin (BF16 plans) holds the
// BF16-rounded value in its own element type too, so that the closed-form
// denominators and contracted operands built from it see exactly the factor the
// tensor cores multiply (otherwise the rounding of a whole factor column biases
// num/den of that column, and the exponential updates scale the bias by num/den).
template <typename T>
__device__ __forceinline__ void write_mirrors(const MirrorDesc& m, const int64_t (&idx)[kMaxFacLet], int nlet, T v) {
#pragma unroll
    for (int k = 0; k < kMaxMirror; ++k) {
        if (k >= m.n) break;
        int64_t off = 0;
#pragma unroll
        for (int q = 0; q < kMaxFacLet; ++q)
            if (q < nlet) off += idx[q] * m.st[k][q];
        if (m.p16[k]) {
            const uint16_t b = bf16_bits((float)v);
            m.p16[k][off] = b;
            static_cast<T*>(m.p32[k])[off] = (T)__uint_as_float((uint32_t)b << 16);
        } else {
            static_cast<T*>(m.p32[k])[off] = v;
        }
    }
}

// One block per 32 consecutive factor elements: the 8 warps sum the split
// partials s = g, g + 8, ... (lane = element, so the reads are coalesced), and
// warp 0 adds the 8 group sums in order and applies the update.
constexpr int kFinEl = 32;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_finish(const __grid_constant__ FinishDesc d,
                                                     const __grid_constant__ UpdateSpec u) {
    pdl_wait();
    pdl_trigger();
    constexpr int kGrp = kThreads / kFinEl;
    __shared__ T sn[kGrp][kFinEl], sd[kGrp][kFinEl];
    const int lane = (int)(threadIdx.x % kFinEl), g = (int)(threadIdx.x / kFinEl);
    const int64_t e = (int64_t)blockIdx.x * kFinEl + lane;
    const bool ok = e < d.n;
    int64_t idx[kMaxFacLet] = {};
    int64_t soff = 0, boff = 0;
    T num = T(0), den = T(0);
    if (ok) {
        decode_letters<T>(e, d.nlet, d.dim, idx);
#pragma unroll
        for (int q = 0; q < kMaxFacLet; ++q) {
            if (q >= d.nlet) continue;
            soff += idx[q] * d.s_st[q];
            boff += idx[q] * d.b_st[q];
        }
        const T* pn = static_cast<const T*>(d.part_num);
        for (int s = g; s < d.n_split; s += kGrp) num += pn[(int64_t)s * d.s_size + soff];
        if (d.part_den) {
            const T* pd = static_cast<const T*>(d.part_den);
            for (int s = g; s < d.n_split; s += kGrp) den += pd[(int64_t)s * d.s_size + soff];
        }
    }
    sn[g][lane] = num;
    sd[g][lane] = den;
    __syncthreads();
    if (g != 0 || !ok) return;
    num = T(0);
    for (int k = 0; k < kGrp; ++k) num += sn[k][lane];
    if (d.part_den) {
        den = T(0);
        for (int k = 0; k < kGrp; ++k) den += sd[k][lane];
    } else {
        den = T(1);
        for (int s = 0; s < d.n_cs; ++s) den *= static_cast<const T*>(d.cs[s])[boff];
    }
    T* th = static_cast<T*>(d.theta);
    const T v = mu_update(th[e], num, den, u);
    th[e] = v;
    write_mirrors<T>(d.mir, idx, d.nlet, v);
}

struct LetterDims {
    int64_t d[kMaxFacLet];
};

// The epilogue's last contraction with Eq. 3.4 applied to its outputs (EinUpdate).
template <typename T, bool DUAL>
__device__ __forceinline__ void ein_update_out(const EinDesc& d, const EinUpdate& up, int64_t dst, T acc, T accb) {
    ein_store<T>(d, d.out, dst, acc);
    if constexpr (DUAL) ein_store<T>(d, d.outb, dst, accb);
    const T num = DUAL ? acc : static_cast<const T*>(up.num)[dst];
    const T den = DUAL ? accb : acc;
    T* th = static_cast<T*>(up.theta);
    const T v = mu_update(th[dst], num, den, up.u);
    th[dst] = v;
    // the element's letters (term order, the last fastest) and its place in each copy
    // (unrolled over the fixed sizes, so the index stays in registers)
    uint32_t idx[kMaxFacLet];
    uint32_t rem = (uint32_t)dst;  // factors have < 2^31 elements
#pragma unroll
    for (int q = kMaxFacLet - 1; q >= 0; --q) {
        idx[q] = 0;
        if (q >= up.nlet) continue;
        const uint32_t dq = (uint32_t)up.dim[q];
        idx[q] = rem % dq;
        rem /= dq;
    }
#pragma unroll
    for (int k = 0; k < kMaxMirror; ++k) {
        if (k >= up.mir.n) break;
        int64_t off = 0;
#pragma unroll
        for (int q = 0; q < kMaxFacLet; ++q)
            if (q < up.nlet) off += (int64_t)idx[q] * up.mir.st[k][q];
        if (up.mir.p16[k]) {
            const uint16_t b = bf16_bits((float)v);
            up.mir.p16[k][off] = b;
            static_cast<T*>(up.mir.p32[k])[off] = (T)__uint_as_float((uint32_t)b << 16);
        } else {
            static_cast<T*>(up.mir.p32[k])[off] = v;
        }
    }
}

template <typename T, bool DUAL>
__global__ void k_einsum_direct_upd(const __grid_constant__ EinDesc d, const __grid_constant__ EinUpdate up) {
    pdl_wait();
    pdl_trigger();
    int64_t dst;
    T acc, accb;
    if (ein_direct_eval<T, DUAL>(d, dst, acc, accb)) ein_update_out<T, DUAL>(d, up, dst, acc, accb);
}

template <typename T, int G, bool DUAL>
__global__ void __launch_bounds__(kThreads) k_einsum_grouped_upd(const __grid_constant__ EinDesc d,
                                                                  const __grid_constant__ EinUpdate up) {
    pdl_wait();
    pdl_trigger();
    __shared__ T sh[kThreads / 32];
    int64_t dst;
    T acc, accb;
    if (ein_grouped_eval<T, G, DUAL>(d, sh, dst, acc, accb)) ein_update_out<T, DUAL>(d, up, dst, acc, accb);
}

template <typename T>
__global__ void k_update_mirror(T* __restrict__ theta, const T* __restrict__ num, const T* __restrict__ den,
                                int64_t n, const __grid_constant__ UpdateSpec u, int nlet,
                                const __grid_constant__ LetterDims dim, const __grid_constant__ MirrorDesc m) {
    pdl_wait();
    pdl_trigger();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const T v = mu_update(theta[e], num[e], den[e], u);
    theta[e] = v;
    int64_t idx[kMaxFacLet];
    decode_letters<T>(e, nlet, dim.d, idx);
    write_mirrors<T>(m, idx, nlet, v);
}

template <typename T>
__global__ void k_mirror_init(const T* __restrict__ theta, int64_t n, int nlet, const __grid_constant__ LetterDims dim,
                              const __grid_constant__ MirrorDesc m) {
    pdl_wait();
    pdl_trigger();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    int64_t idx[kMaxFacLet];
    decode_letters<T>(e, nlet, dim.d, idx);
    write_mirrors<T>(m, idx, nlet, theta[e]);
}

// Column sums of canonical operands: block (job, column).
template <typename T>
__global__ void k_colsums(const __grid_constant__ ColsumDesc d) {
    pdl_wait();
    pdl_trigger();
    const ColsumJob& j = d.job[blockIdx.x];
    const int64_t b = blockIdx.y;
    if (b >= j.ld) return;
    const T* src = static_cast<const T*>(j.src);
    T acc = T(0);
    for (int64_t r = threadIdx.x; r < j.n_rows; r += blockDim.x) acc += src[r * j.ld + b];
    __shared__ T sh[kThreads / 32];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        T t = T(0);
        for (int k = 0; k < kThreads / 32; ++k) t += sh[k];
        static_cast<T*>(j.out)[b] = t;
    }
}

inline unsigned blocks_for(int64_t n, int threads = kThreads) {
    return (unsigned)((n + threads - 1) / threads);
}

}  // namespace

// How a contraction runs: a group of G threads per output (returns G), one thread per
// output (1), or split over the free combinations with a partial buffer (0).
static int ein_mode(const EinDesc& d, int64_t partial_cap, int64_t* n_split_out) {
    *n_split_out = 1;
    // few free combinations per output: a group of G threads per output, unless there are
    // outputs enough for one thread each and few combinations (a short loop beats the
    // group's idle threads and its reduction)
    const bool short_loop = d.n_free_el <= 16 && d.n_out_el >= 32768;
    if (d.n_free_el > 4 && !short_loop && d.n_free_el < ((int64_t)1 << 31)) {
        const int g = d.n_free_el <= 32 ? 8 : (d.n_free_el <= 128 ? 32 : kThreads);
        const bool part_ok = partial_cap >= 2 * d.n_out_el;
        if (d.n_free_el / g <= 64 || !part_ok) {
            const int64_t blocks = (d.n_out_el + kThreads / g - 1) / (kThreads / g);
            if (blocks < ((int64_t)1 << 31)) return g;
        }
    }
    // split the free combinations so that the grid has enough threads
    const int64_t want = (int64_t)152 * 2048;
    int64_t n_split = 1;
    if (d.n_free_el > 64 && d.n_out_el < want && partial_cap >= 2 * d.n_out_el) {
        n_split = std::min<int64_t>((want + d.n_out_el - 1) / d.n_out_el, d.n_free_el / 32);
        n_split = std::min<int64_t>(n_split, 65535);
        n_split = std::min<int64_t>(n_split, partial_cap / d.n_out_el);
        n_split = std::max<int64_t>(n_split, 1);
    }
    *n_split_out = n_split;
    return n_split == 1 ? 1 : 0;
}

template <typename T>
cudaError_t launch_einsum(const EinDesc& d, T* partial, int64_t partial_cap, cudaStream_t st) {
    if (d.n_out_el <= 0) return cudaSuccess;
    if (d.n_out_el >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;  // 32-bit output decode
    const bool dual = d.op0b != nullptr && d.outb != nullptr && d.n_ops >= 1;
    int64_t n_split = 1;
    const int mode = ein_mode(d, partial_cap, &n_split);
    if (mode > 1) {
        const unsigned blocks = (unsigned)((d.n_out_el + kThreads / mode - 1) / (kThreads / mode));
        if (dual) {
            if (mode == 8) launch_pdl(k_einsum_grouped<T, 8, true>, blocks, kThreads, 0, st, d);
            else if (mode == 32) launch_pdl(k_einsum_grouped<T, 32, true>, blocks, kThreads, 0, st, d);
            else launch_pdl(k_einsum_grouped<T, kThreads, true>, blocks, kThreads, 0, st, d);
        } else {
            if (mode == 8) launch_pdl(k_einsum_grouped<T, 8, false>, blocks, kThreads, 0, st, d);
            else if (mode == 32) launch_pdl(k_einsum_grouped<T, 32, false>, blocks, kThreads, 0, st, d);
            else launch_pdl(k_einsum_grouped<T, kThreads, false>, blocks, kThreads, 0, st, d);
        }
        return cudaGetLastError();
    }
    if (mode == 1) {
        // one pass straight into the destination
        if (dual) launch_pdl(k_einsum_direct<T, true>, blocks_for(d.n_out_el), kThreads, 0, st, d);
        else launch_pdl(k_einsum_direct<T, false>, blocks_for(d.n_out_el), kThreads, 0, st, d);
        return cudaGetLastError();
    }
    if (dual) {
        // the split form computes one contraction: the two, one after the other
        EinDesc a = d, b = d;
        a.op0b = nullptr;
        a.outb = nullptr;
        b.op[0] = d.op0b;
        b.out = d.outb;
        b.op0b = nullptr;
        b.outb = nullptr;
        cudaError_t e = launch_einsum<T>(a, partial, partial_cap, st);
        return e != cudaSuccess ? e : launch_einsum<T>(b, partial, partial_cap, st);
    }
    const int64_t chunk = (d.n_free_el + n_split - 1) / n_split;
    dim3 grid(blocks_for(d.n_out_el), (unsigned)n_split);
    launch_pdl(k_einsum_part<T>, grid, kThreads, 0, st, d, chunk, partial);
    launch_pdl(k_einsum_final<T>, blocks_for(d.n_out_el), kThreads, 0, st, d, (int)n_split, partial);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_einsum_update(const EinDesc& d, const EinUpdate& up, T* partial, int64_t partial_cap,
                                 cudaStream_t st) {
    if (d.n_out_el <= 0) return cudaSuccess;
    if (d.n_out_el >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    const bool dual = d.op0b != nullptr && d.outb != nullptr && d.n_ops >= 1;
    if (dual == (up.num != nullptr)) return cudaErrorInvalidValue;  // num from the dual form or from up.num
    int64_t n_split = 1;
    const int mode = ein_mode(d, partial_cap, &n_split);
    if (mode > 1) {
        const unsigned blocks = (unsigned)((d.n_out_el + kThreads / mode - 1) / (kThreads / mode));
        if (dual) {
            if (mode == 8) launch_pdl(k_einsum_grouped_upd<T, 8, true>, blocks, kThreads, 0, st, d, up);
            else if (mode == 32) launch_pdl(k_einsum_grouped_upd<T, 32, true>, blocks, kThreads, 0, st, d, up);
            else launch_pdl(k_einsum_grouped_upd<T, kThreads, true>, blocks, kThreads, 0, st, d, up);
        } else {
            if (mode == 8) launch_pdl(k_einsum_grouped_upd<T, 8, false>, blocks, kThreads, 0, st, d, up);
            else if (mode == 32) launch_pdl(k_einsum_grouped_upd<T, 32, false>, blocks, kThreads, 0, st, d, up);
            else launch_pdl(k_einsum_grouped_upd<T, kThreads, false>, blocks, kThreads, 0, st, d, up);
        }
        return cudaGetLastError();
    }
    if (mode == 1) {
        if (dual) launch_pdl(k_einsum_direct_upd<T, true>, blocks_for(d.n_out_el), kThreads, 0, st, d, up);
        else launch_pdl(k_einsum_direct_upd<T, false>, blocks_for(d.n_out_el), kThreads, 0, st, d, up);
        return cudaGetLastError();
    }
    // split over the free combinations: the contraction(s), then the update on its own
    cudaError_t e = launch_einsum<T>(d, partial, partial_cap, st);
    if (e != cudaSuccess) return e;
    LetterDims ld{};
    for (int q = 0; q < up.nlet; ++q) ld.d[q] = up.dim[q];
    const T* num = dual ? static_cast<const T*>(d.out) : static_cast<const T*>(up.num);
    const T* den = dual ? static_cast<const T*>(d.outb) : static_cast<const T*>(d.out);
    launch_pdl(k_update_mirror<T>, blocks_for(d.n_out_el), kThreads, 0, st, static_cast<T*>(up.theta), num, den,
               d.n_out_el, up.u, up.nlet, ld, up.mir);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_finish(const FinishDesc& d, const UpdateSpec& u, cudaStream_t st) {
    launch_pdl(k_finish<T>, blocks_for(d.n, kFinEl), kThreads, 0, st, d, u);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update_mirror(T* theta, const T* num, const T* den, int64_t n, const UpdateSpec& u,
                                 int nlet, const int64_t* dim, const MirrorDesc& m, cudaStream_t st) {
    LetterDims ld{};
    for (int q = 0; q < nlet; ++q) ld.d[q] = dim[q];
    launch_pdl(k_update_mirror<T>, blocks_for(n), kThreads, 0, st, theta, num, den, n, u, nlet, ld, m);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_mirror_init(const T* theta, int64_t n, int nlet, const int64_t* dim,
                               const MirrorDesc& m, cudaStream_t st) {
    if (m.n == 0) return cudaSuccess;
    LetterDims ld{};
    for (int q = 0; q < nlet; ++q) ld.d[q] = dim[q];
    launch_pdl(k_mirror_init<T>, blocks_for(n), kThreads, 0, st, theta, n, nlet, ld, m);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_colsums(const ColsumDesc& d, int64_t max_ld, cudaStream_t st) {
    if (d.n == 0) return cudaSuccess;
    launch_pdl(k_colsums<T>, dim3((unsigned)d.n, (unsigned)max_ld), kThreads, 0, st, d);
    return cudaGetLastError();
}

cudaError_t launch_pack_mask(const uint8_t* mask, int64_t n, uint32_t* bits, cudaStream_t st) {
    const int64_t nw = (n + 31) >> 5;
    launch_pdl(k_pack_mask, blocks_for(nw), kThreads, 0, st, mask, n, bits);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_check_data(const T* y, int64_t n, int* flag, cudaStream_t st) {
    unsigned nb = (unsigned)std::min<int64_t>(blocks_for(n), 152 * 8);
    launch_pdl(k_check_data<T>, nb, kThreads, 0, st, y, n, flag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reduce_splits(const T* part, int n_split, int64_t n, T* out, cudaStream_t st) {
    launch_pdl(k_reduce_splits<T>, blocks_for(n), kThreads, 0, st, part, n_split, n, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reduce_splits2(const T* part_a, const T* part_b, int n_split, int64_t n, T* out_a, T* out_b,
                                  cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    launch_pdl(k_reduce_splits2<T>, blocks_for(2 * n), kThreads, 0, st, part_a, part_b, n_split, n, out_a, out_b);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update(T* theta, const T* num, const T* den, int64_t n, const UpdateSpec& u,
                          cudaStream_t st) {
    launch_pdl(k_update<T>, blocks_for(n), kThreads, 0, st, theta, num, den, n, u);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fill(T* p, int64_t n, T v, cudaStream_t st) {
    launch_pdl(k_fill<T>, blocks_for(n), kThreads, 0, st, p, n, v);
    return cudaGetLastError();
}

cudaError_t launch_sum_f64(const double* part, int n, double* out, cudaStream_t st) {
    launch_pdl(k_sum_f64, 1, 1024, 0, st, part, n, out);
    return cudaGetLastError();
}

cudaError_t launch_loss_append(const double* part, int n, double* trace, int* count, double* out,
                               cudaStream_t st) {
    launch_pdl(k_loss_append, 1, 1024, 0, st, part, n, trace, count, out);
    return cudaGetLastError();
}

// The stopping rules of App. B on the device (one thread, fit_rule_step); inside
// a graph loop the result also becomes the loop's condition.
__global__ void k_fit_check(FitCtlState* s, const double* out_loss, const double* out_val,
                            cudaGraphConditionalHandle handle, int set_handle, int mode) {
    pdl_wait();
    pdl_trigger();
    const int cont = fit_rule_step(s, out_loss, out_val, mode);
    if (set_handle && mode == 0) cudaGraphSetConditional(handle, cont ? 1u : 0u);
}

__global__ void k_fit_set_cond(const FitCtlState* s, cudaGraphConditionalHandle handle) {
    pdl_wait();
    pdl_trigger();
    cudaGraphSetConditional(handle, s->cont ? 1u : 0u);
}

cudaError_t launch_fit_check(FitCtlState* s, const double* out_loss, const double* out_val,
                             cudaGraphConditionalHandle handle, int set_handle, int mode, cudaStream_t st) {
    launch_pdl(k_fit_check, 1, 1, 0, st, s, out_loss, out_val, handle, set_handle, mode);
    return cudaGetLastError();
}

cudaError_t launch_fit_set_cond(const FitCtlState* s, cudaGraphConditionalHandle handle, cudaStream_t st) {
    launch_pdl(k_fit_set_cond, 1, 1, 0, st, s, handle);
    return cudaGetLastError();
}

cudaError_t launch_convert_bf16(float* src, int64_t n, uint16_t* dst, cudaStream_t st) {
    launch_pdl(k_convert_bf16, blocks_for(n), kThreads, 0, st, src, n, dst);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_generic_weights(const GenericRecon& g, const T* y, const uint32_t* mbits,
                                   const WeightSpec& w, T* wa, T* wb, const LossSpec* loss,
                                   double* loss_part, int n_part, cudaStream_t st) {
    const unsigned nb = loss ? (unsigned)n_part : (unsigned)std::min<int64_t>(blocks_for(g.n), 152 * 16);
    LossSpec L{};
    if (loss) L = *loss;
    launch_pdl(k_generic_weights<T>, nb, kThreads, 0, st, g, y, mbits, w, wa, wb, loss ? 1 : 0, L, loss_part);
    return cudaGetLastError();
}

#define NEF_INST(T)                                                                          \
    template cudaError_t launch_einsum<T>(const EinDesc&, T*, int64_t, cudaStream_t);        \
    template cudaError_t launch_einsum_update<T>(const EinDesc&, const EinUpdate&, T*, int64_t, cudaStream_t); \
    template cudaError_t launch_check_data<T>(const T*, int64_t, int*, cudaStream_t);        \
    template cudaError_t launch_reduce_splits<T>(const T*, int, int64_t, T*, cudaStream_t);  \
    template cudaError_t launch_reduce_splits2<T>(const T*, const T*, int, int64_t, T*, T*, cudaStream_t); \
    template cudaError_t launch_update<T>(T*, const T*, const T*, int64_t, const UpdateSpec&, \
                                          cudaStream_t);                                     \
    template cudaError_t launch_fill<T>(T*, int64_t, T, cudaStream_t);                       \
    template cudaError_t launch_generic_weights<T>(const GenericRecon&, const T*,             \
                                                   const uint32_t*, const WeightSpec&, T*, T*, \
                                                   const LossSpec*, double*, int, cudaStream_t);

#define NEF_INST2(T)                                                                          \
    template cudaError_t launch_finish<T>(const FinishDesc&, const UpdateSpec&, cudaStream_t);    \
    template cudaError_t launch_update_mirror<T>(T*, const T*, const T*, int64_t, const UpdateSpec&, \
                                                 int, const int64_t*, const MirrorDesc&, cudaStream_t); \
    template cudaError_t launch_mirror_init<T>(const T*, int64_t, int, const int64_t*,             \
                                               const MirrorDesc&, cudaStream_t);                   \
    template cudaError_t launch_colsums<T>(const ColsumDesc&, int64_t, cudaStream_t);

NEF_INST(float)
NEF_INST(double)
NEF_INST2(float)
NEF_INST2(double)

}  // namespace nef
