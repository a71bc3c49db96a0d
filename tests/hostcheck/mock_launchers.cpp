// Plain-loop implementations of the launcher interface in nef_internal.h,
// following each descriptor's documented meaning, so that plan.cpp (the real
// planner and sweep driver) can be checked against the oracle on a CPU host.
// TEST INFRASTRUCTURE ONLY: built by tests/hostcheck/build.py into a separate
// library that the product never loads.  The element math (weights, divergence,
// update) is the product's own nef_device.cuh compiled for the host.
#include <cmath>
#include <cstring>
#include <vector>

#define __device__
#define __host__
#define __forceinline__ inline
#define __shfl_xor_sync(m, v, o) (v)
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
using std::isinf;
#include "nef_device.cuh"
#include "nef_internal.h"

namespace nef {

template <typename T>
cudaError_t launch_einsum(const EinDesc& d, T*, int64_t, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
    const int nl = d.n_out + d.n_free;
    std::vector<int64_t> idx(nl);
    for (int64_t o = 0; o < d.n_out_el; ++o) {
        int64_t rem = o, dst = 0;
        for (int q = d.n_out - 1; q >= 0; --q) {
            idx[q] = rem % d.dim[q];
            dst += idx[q] * d.out_st[q];
            rem /= d.dim[q];
        }
        // with op0b/outb: the same contraction with op0b in place of operand 0, into outb
        const bool dual = d.op0b != nullptr && d.outb != nullptr;
        for (int pass = 0; pass < (dual ? 2 : 1); ++pass) {
            T acc = 0;
            for (int64_t f = 0; f < d.n_free_el; ++f) {
                int64_t r2 = f;
                for (int q = nl - 1; q >= d.n_out; --q) {
                    idx[q] = r2 % d.dim[q];
                    r2 /= d.dim[q];
                }
                T p = 1;
                for (int k = 0; k < d.n_ops; ++k) {
                    int64_t off = 0;
                    for (int q = 0; q < nl; ++q) off += idx[q] * d.ost[k][q];
                    const T* base = static_cast<const T*>(k == 0 && pass == 1 ? d.op0b : d.op[k]);
                    T v = base[off];
                    // operand 0 as the sum of its split partials
                    if (k == 0)
                        for (int sp = 1; sp < d.op0_splits; ++sp) v += base[off + sp * d.op0_split_stride];
                    p *= v;
                }
                acc += p;
            }
            T* out = static_cast<T*>(pass == 1 ? d.outb : d.out);
            if (d.out16) {  // BF16 copy, and the value rounded to it (nearest even)
                uint32_t u;
                float v = (float)acc;
                std::memcpy(&u, &v, 4);
                const uint32_t r = u + 0x7fffu + ((u >> 16) & 1u);
                d.out16[dst] = (uint16_t)(r >> 16);
                const uint32_t hi = r & 0xffff0000u;
                std::memcpy(&v, &hi, 4);
                out[dst] = (T)v;
            } else {
                out[dst] = d.accumulate ? out[dst] + acc : acc;
            }
        }
    }
    return cudaSuccess;
    });
}

cudaError_t launch_pack_mask(const uint8_t* m, int64_t n, uint32_t* bits, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
    for (int64_t w = 0; w < (n + 31) / 32; ++w) {
        uint32_t v = 0;
        for (int b = 0; b < 32; ++b)
            if (w * 32 + b < n && m[w * 32 + b]) v |= 1u << b;
        bits[w] = v;
    }
    return cudaSuccess;
    });
}

template <typename T>
cudaError_t launch_check_data(const T* y, int64_t n, int* flag, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
    for (int64_t e = 0; e < n; ++e)
        if (!(y[e] >= 0) || std::isinf((double)y[e])) *flag = 1;
    return cudaSuccess;
    });
}

template <typename T>
static T side_value(const SideDesc& sd, int64_t i, int b) {
    T p = 1;
    for (int s = 0; s < sd.nsrc; ++s) {
        const SrcDesc& d = sd.src[s];
        int64_t r = 0;
        for (int t = 0; t < d.nterm; ++t) r += ((i / d.div[t]) % d.mod[t]) * d.mul[t];
        p *= static_cast<const T*>(d.ptr)[r * d.ld + b];
    }
    return p;
}

template <typename T>
cudaError_t launch_view_simt(const T* y, const uint32_t* mbits, const ViewDesc& v,
                             const WeightSpec& w, int need_den, int n_split, T* s_num, T* s_den,
                             const LossSpec* loss_in, double* loss_part, cudaStream_t, int* n_ctas) {
    if (n_ctas) *n_ctas = 1;
    const bool has_loss = loss_in != nullptr;
    const LossSpec lval = loss_in ? *loss_in : LossSpec{};
    return host_submit([=]() -> cudaError_t {
    const LossSpec* loss = has_loss ? &lval : nullptr;
    const int64_t ncols = v.c_out * v.c_in;
    const int BP = v.bond_pad;
    if (s_num) {
        for (int64_t e = 0; e < (int64_t)n_split * v.rows * BP; ++e) {
            s_num[e] = 0;
            if (need_den) s_den[e] = 0;
        }
    }
    double ls = 0, lc = 0;
    std::vector<T> P(BP), Q(BP);
    for (int64_t row = 0; row < v.rows; ++row) {
        for (int b = 0; b < BP; ++b) P[b] = b < v.bond ? side_value<T>(v.P, row, b) : T(0);
        for (int64_t col = 0; col < ncols; ++col) {
            const int64_t idx = (col / v.c_in) * v.rows * v.c_in + row * v.c_in + (col % v.c_in);
            if (mbits && !mask_bit(mbits, idx)) continue;
            T yh = 0;
            for (int b = 0; b < BP; ++b) {
                Q[b] = b < v.bond ? side_value<T>(v.Q, col, b) : T(0);
                yh += P[b] * Q[b];
            }
            T a, bb;
            ab_weights(y[idx], yh, w, a, bb);
            if (loss) { ls += (double)divergence(y[idx], yh, *loss); lc += 1; }
            if (s_num)
                for (int b = 0; b < BP; ++b) {
                    s_num[row * BP + b] += a * Q[b];
                    if (need_den) s_den[row * BP + b] += bb * Q[b];
                }
        }
    }
    if (loss) { loss_part[0] = ls; loss_part[1] = lc; }
    return cudaSuccess;
    });
}

template <typename T>
cudaError_t launch_reduce_splits(const T* part, int n_split, int64_t n, T* out, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
    for (int64_t e = 0; e < n; ++e) {
        T acc = 0;
        for (int s = 0; s < n_split; ++s) acc += part[s * n + e];
        out[e] = acc;
    }
    return cudaSuccess;
    });
}

long long kernel_launches() { return 0; }

template <typename T>
cudaError_t launch_reduce_splits2(const T* part_a, const T* part_b, int n_split, int64_t n, T* out_a, T* out_b,
                                  cudaStream_t st) {
    cudaError_t e = launch_reduce_splits<T>(part_a, n_split, n, out_a, st);
    return e != cudaSuccess ? e : launch_reduce_splits<T>(part_b, n_split, n, out_b, st);
}

template <typename T>
cudaError_t launch_update(T* theta, const T* num, const T* den, int64_t n, const UpdateSpec& u,
                          cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
    for (int64_t e = 0; e < n; ++e) theta[e] = mu_update(theta[e], num[e], den[e], u);
    return cudaSuccess;
    });
}

template <typename T>
cudaError_t launch_fill(T* p, int64_t n, T v, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
    for (int64_t e = 0; e < n; ++e) p[e] = v;
    return cudaSuccess;
    });
}

cudaError_t launch_sum_f64(const double* part, int n, double* out, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
    double s = 0;
    for (int k = 0; k < n; ++k) s += part[k];
    *out = s;
    return cudaSuccess;
    });
}

cudaError_t launch_convert_bf16(float*, int64_t, uint16_t*, cudaStream_t) {
    return cudaErrorNotSupported;
}

template <typename T>
cudaError_t launch_generic_weights(const GenericRecon& g, const T* y, const uint32_t* mbits,
                                   const WeightSpec& w, T* wa, T* wb, const LossSpec* loss_in,
                                   double* loss_part, int n_part, cudaStream_t) {
    const bool has_loss = loss_in != nullptr;
    const LossSpec lval = loss_in ? *loss_in : LossSpec{};
    return host_submit([=]() -> cudaError_t {
    const LossSpec* loss = has_loss ? &lval : nullptr;
    double ls = 0, lc = 0;
    std::vector<int64_t> idx(g.n_let);
    for (int64_t e = 0; e < g.n; ++e) {
        int64_t rem = e;
        for (int m = g.n_obs - 1; m >= 0; --m) { idx[m] = rem % g.dim[m]; rem /= g.dim[m]; }
        T yh = 0;
        for (int64_t c = 0; c < g.n_lat_el; ++c) {
            int64_t r2 = c;
            for (int x = g.n_let - 1; x >= g.n_obs; --x) { idx[x] = r2 % g.dim[x]; r2 /= g.dim[x]; }
            T p = 1;
            for (int f = 0; f < g.n_fac; ++f) {
                int64_t off = 0;
                for (int x = 0; x < g.n_let; ++x) off += idx[x] * g.fst[f][x];
                p *= static_cast<const T*>(g.fac[f])[off];
            }
            yh += p;
        }
        T a = 0, b = 0;
        if (!mbits || mask_bit(mbits, e)) {
            ab_weights(y[e], yh, w, a, b);
            if (loss) { ls += (double)divergence(y[e], yh, *loss); lc += 1; }
        }
        if (wa) wa[e] = a;
        if (wb) wb[e] = b;
    }
    if (loss) {
        for (int k = 0; k < 2 * n_part; ++k) loss_part[k] = 0;
        loss_part[0] = ls;
        loss_part[n_part] = lc;
    }
    return cudaSuccess;
    });
}

static uint16_t bf16_bits_host(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

// A copy with a BF16 twin holds the BF16-rounded value in its own type too.
template <typename T>
static void write_mirrors_host(const MirrorDesc& m, const int64_t* idx, int nlet, T v) {
    for (int k = 0; k < m.n; ++k) {
        int64_t off = 0;
        for (int q = 0; q < nlet; ++q) off += idx[q] * m.st[k][q];
        if (m.p16[k]) {
            const uint16_t b = bf16_bits_host((float)v);
            m.p16[k][off] = b;
            const uint32_t u = (uint32_t)b << 16;
            float f;
            std::memcpy(&f, &u, 4);
            static_cast<T*>(m.p32[k])[off] = (T)f;
        } else {
            static_cast<T*>(m.p32[k])[off] = v;
        }
    }
}

static void decode(int64_t e, int nlet, const int64_t* dim, int64_t* idx) {
    for (int q = nlet - 1; q >= 0; --q) { idx[q] = e % dim[q]; e /= dim[q]; }
}

template <typename T>
cudaError_t launch_finish(const FinishDesc& d, const UpdateSpec& u, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
    for (int64_t e = 0; e < d.n; ++e) {
        int64_t idx[kMaxFacLet];
        decode(e, d.nlet, d.dim, idx);
        int64_t soff = 0, boff = 0;
        for (int q = 0; q < d.nlet; ++q) { soff += idx[q] * d.s_st[q]; boff += idx[q] * d.b_st[q]; }
        T num = 0, den;
        for (int s = 0; s < d.n_split; ++s) num += static_cast<const T*>(d.part_num)[s * d.s_size + soff];
        if (d.part_den) {
            den = 0;
            for (int s = 0; s < d.n_split; ++s) den += static_cast<const T*>(d.part_den)[s * d.s_size + soff];
        } else {
            den = 1;
            for (int s = 0; s < d.n_cs; ++s) den *= static_cast<const T*>(d.cs[s])[boff];
        }
        T* th = static_cast<T*>(d.theta);
        th[e] = mu_update(th[e], num, den, u);
        write_mirrors_host<T>(d.mir, idx, d.nlet, th[e]);
    }
    return cudaSuccess;
    });
}

template <typename T>
cudaError_t launch_update_mirror(T* theta, const T* num, const T* den, int64_t n, const UpdateSpec& u,
                                 int nlet, const int64_t* dim_in, const MirrorDesc& m, cudaStream_t) {
    const std::vector<int64_t> dv(dim_in, dim_in + nlet);
    return host_submit([=]() -> cudaError_t {
    const int64_t* dim = dv.data();
    for (int64_t e = 0; e < n; ++e) {
        theta[e] = mu_update(theta[e], num[e], den[e], u);
        int64_t idx[kMaxFacLet];
        decode(e, nlet, dim, idx);
        write_mirrors_host<T>(m, idx, nlet, theta[e]);
    }
    return cudaSuccess;
    });
}

// The contraction, then Eq. 3.4 over its outputs (num from the dual form or up.num).
template <typename T>
cudaError_t launch_einsum_update(const EinDesc& d, const EinUpdate& up, T* partial, int64_t cap, cudaStream_t st) {
    const bool dual = d.op0b != nullptr && d.outb != nullptr;
    if (dual == (up.num != nullptr)) return cudaErrorInvalidValue;
    cudaError_t e = launch_einsum<T>(d, partial, cap, st);
    if (e != cudaSuccess) return e;
    const T* num = dual ? static_cast<const T*>(d.out) : static_cast<const T*>(up.num);
    const T* den = dual ? static_cast<const T*>(d.outb) : static_cast<const T*>(d.out);
    return launch_update_mirror<T>(static_cast<T*>(up.theta), num, den, d.n_out_el, up.u, up.nlet, up.dim, up.mir,
                                   st);
}

template <typename T>
cudaError_t launch_mirror_init(const T* theta, int64_t n, int nlet, const int64_t* dim_in,
                               const MirrorDesc& m, cudaStream_t) {
    const std::vector<int64_t> dv(dim_in, dim_in + nlet);
    return host_submit([=]() -> cudaError_t {
    const int64_t* dim = dv.data();
    for (int64_t e = 0; e < n; ++e) {
        int64_t idx[kMaxFacLet];
        decode(e, nlet, dim, idx);
        write_mirrors_host<T>(m, idx, nlet, theta[e]);
    }
    return cudaSuccess;
    });
}

template <typename T>
cudaError_t launch_colsums(const ColsumDesc& d, int64_t, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
    for (int k = 0; k < d.n; ++k) {
        const ColsumJob& j = d.job[k];
        for (int64_t b = 0; b < j.ld; ++b) {
            T acc = 0;
            for (int64_t r = 0; r < j.n_rows; ++r) acc += static_cast<const T*>(j.src)[r * j.ld + b];
            static_cast<T*>(j.out)[b] = acc;
        }
    }
    return cudaSuccess;
    });
}

bool tc_view_supported(const ViewDesc&, int) { return false; }
cudaError_t launch_view_tc(const float*, const uint32_t*, const ViewDesc&, const WeightSpec&, int,
                           int, float*, float*, int*, cudaStream_t, TcLaunchInfo*, unsigned long long*,
                           const LossSpec*, double*, long long, const TcTileConfig*) {
    return cudaErrorNotSupported;
}

cudaError_t launch_fit_check(FitCtlState* s, const double* out_loss, const double* out_val,
                             cudaGraphConditionalHandle handle, int set_handle, int mode, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        const int cont = fit_rule_step(s, out_loss, out_val, mode);
        if (set_handle && mode == 0) *reinterpret_cast<unsigned*>(handle) = cont ? 1u : 0u;
        return cudaSuccess;
    });
}

cudaError_t launch_fit_set_cond(const FitCtlState* s, cudaGraphConditionalHandle handle, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        *reinterpret_cast<unsigned*>(handle) = s->cont ? 1u : 0u;
        return cudaSuccess;
    });
}

cudaError_t launch_loss_append(const double* part, int n, double* trace, int* count, double* out, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        double a = 0, c = 0;
        for (int k = 0; k < n; ++k) {
            a += part[k];
            c += part[n + k];
        }
        out[0] = a;
        out[1] = c;
        if (trace) trace[*count] = a;
        *count += 1;
        return cudaSuccess;
    });
}

#define INST(T)                                                                                  \
    template cudaError_t launch_einsum<T>(const EinDesc&, T*, int64_t, cudaStream_t);            \
    template cudaError_t launch_check_data<T>(const T*, int64_t, int*, cudaStream_t);            \
    template cudaError_t launch_view_simt<T>(const T*, const uint32_t*, const ViewDesc&,         \
                                             const WeightSpec&, int, int, T*, T*,                \
                                             const LossSpec*, double*, cudaStream_t, int*);      \
    template cudaError_t launch_reduce_splits<T>(const T*, int, int64_t, T*, cudaStream_t);      \
    template cudaError_t launch_reduce_splits2<T>(const T*, const T*, int, int64_t, T*, T*, cudaStream_t); \
    template cudaError_t launch_update<T>(T*, const T*, const T*, int64_t, const UpdateSpec&,     \
                                          cudaStream_t);                                         \
    template cudaError_t launch_fill<T>(T*, int64_t, T, cudaStream_t);                           \
    template cudaError_t launch_generic_weights<T>(const GenericRecon&, const T*,                 \
                                                   const uint32_t*, const WeightSpec&, T*, T*,     \
                                                   const LossSpec*, double*, int, cudaStream_t);
#define INST2(T)                                                                                 \
    template cudaError_t launch_finish<T>(const FinishDesc&, const UpdateSpec&, cudaStream_t);       \
    template cudaError_t launch_einsum_update<T>(const EinDesc&, const EinUpdate&, T*, int64_t, cudaStream_t); \
    template cudaError_t launch_update_mirror<T>(T*, const T*, const T*, int64_t, const UpdateSpec&,  \
                                                 int, const int64_t*, const MirrorDesc&, cudaStream_t); \
    template cudaError_t launch_mirror_init<T>(const T*, int64_t, int, const int64_t*,                \
                                               const MirrorDesc&, cudaStream_t);                      \
    template cudaError_t launch_colsums<T>(const ColsumDesc&, int64_t, cudaStream_t);
INST(float)
INST(double)
INST2(float)
INST2(double)

}  // namespace nef
