// Plain-loop implementations of the batched engine's launchers (nef_batched.h),
// following each descriptor's documented meaning, so that batched.cpp (the real
// work tables, padded layouts, partial offsets and graph-captured sweep loop)
// can be checked against the oracle on a CPU host.
// TEST INFRASTRUCTURE ONLY: built by tests/hostcheck/build.py into a separate
// library that the product never loads.  The element math (weights, divergence,
// update) is the product's own nef_device.cuh compiled for the host.  Operands
// are rounded to BF16 where the tensor-core pass rounds them (factor copies, Q
// rows, weights); products and sums are FP32.
#include <cmath>
#include <cstring>
#include <vector>

#define __device__
#define __host__
#define __forceinline__ inline
#define __shfl_xor_sync(m, v, o) (v)
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
using std::isinf;
#include "nef_batched.h"
#include "nef_device.cuh"

namespace nef {

namespace {

constexpr int kTM = 128, kTN = 64;

struct MockUnit {
    const float* y;
    const uint32_t* mbits;
    ViewDesc v;
    WeightSpec w;
    int n_split;
    float* s_num;
    float* s_den;
    int64_t n_cib, n_tiles, tiles_per_split;
};

std::vector<MockUnit>& registry() {
    static std::vector<MockUnit> r;
    return r;
}

float bf16_round(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

float bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

uint16_t bf16_bits(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return (uint16_t)((u + 0x7fffu + ((u >> 16) & 1u)) >> 16);
}

int64_t src_row(const SrcDesc& d, int64_t i) {
    int64_t r = 0;
    for (int t = 0; t < d.nterm; ++t) r += ((i / d.div[t]) % d.mod[t]) * d.mul[t];
    return r;
}

}  // namespace

bool tc_make_unit(const float* y, const uint32_t* mbits, const ViewDesc& v, const WeightSpec& w, int n_split,
                  float* s_num, float* s_den, int*, TcUnit* unit, int* n_rb) {
    MockUnit m{y, mbits, v, w, n_split, s_num, s_den, 0, 0, 0};
    const bool trans = v.c_in == 1;
    m.n_cib = trans ? 1 : (v.c_in + kTN - 1) / kTN;
    m.n_tiles = trans ? (v.c_out + kTN - 1) / kTN : v.c_out * m.n_cib;
    m.tiles_per_split = (m.n_tiles + n_split - 1) / n_split;
    registry().push_back(m);
    const int64_t id = (int64_t)registry().size() - 1;
    std::memset(unit, 0, sizeof(TcUnit));
    std::memcpy(unit->prm, &id, sizeof(id));
    *n_rb = (int)((v.rows + kTM - 1) / kTM);
    return true;
}

// One work item: S[split][row][:] = sum over the split's columns of W(y, yhat) Q[col, :]
// for the rows of one row block (Eq. 3.8 with the bond re-association).
static void mock_item(const TcUnit* units, int um, int rb, int sp, int bp, int need_den) {
    int64_t id;
    std::memcpy(&id, units[um].prm, sizeof(id));
    const MockUnit& m = registry()[(size_t)id];
    const ViewDesc& v = m.v;
    const bool trans = v.c_in == 1;
    const int64_t t_lo = (int64_t)sp * m.tiles_per_split;
    const int64_t t_hi = std::min(t_lo + m.tiles_per_split, m.n_tiles);
    std::vector<float> q(bp), sn(bp), sd(bp);
    for (int64_t row = (int64_t)rb * kTM; row < std::min(v.rows, (int64_t)(rb + 1) * kTM); ++row) {
        std::fill(sn.begin(), sn.end(), 0.f);
        std::fill(sd.begin(), sd.end(), 0.f);
        const uint16_t* prow = static_cast<const uint16_t*>(v.P.src[0].ptr) + src_row(v.P.src[0], row) * bp;
        for (int64_t t = t_lo; t < t_hi; ++t) {
            int64_t col0, nvalid;
            if (trans) {
                col0 = t * kTN;
                nvalid = std::min<int64_t>(kTN, v.c_out - col0);
            } else {
                const int64_t co = t / m.n_cib, ci = t % m.n_cib;
                col0 = co * v.c_in + ci * kTN;
                nvalid = std::min<int64_t>(kTN, v.c_in - ci * kTN);
            }
            for (int64_t c = 0; c < nvalid; ++c) {
                const int64_t col = col0 + c;
                const int64_t e = trans ? col * v.rows + row
                                        : ((col / v.c_in) * v.rows + row) * v.c_in + col % v.c_in;
                if (m.mbits && !mask_bit(m.mbits, e)) continue;
                for (int b = 0; b < bp; ++b) q[b] = 1.f;
                for (int s = 0; s < v.Q.nsrc; ++s) {
                    const uint16_t* qrow =
                        static_cast<const uint16_t*>(v.Q.src[s].ptr) + src_row(v.Q.src[s], col) * bp;
                    for (int b = 0; b < bp; ++b) q[b] *= bf16_value(qrow[b]);
                }
                float yh = 0.f;
                for (int b = 0; b < bp; ++b) {
                    q[b] = bf16_round(q[b]);
                    yh += bf16_value(prow[b]) * q[b];
                }
                float wa, wb;
                ab_weights(m.y[e], yh, m.w, wa, wb);
                wa = bf16_round(wa);
                wb = bf16_round(wb);
                for (int b = 0; b < bp; ++b) {
                    sn[b] += wa * q[b];
                    sd[b] += wb * q[b];
                }
            }
        }
        float* dn = m.s_num + ((int64_t)sp * v.rows + row) * bp;
        for (int b = 0; b < bp; ++b) dn[b] = sn[b];
        if (need_den) {
            float* dd = m.s_den + ((int64_t)sp * v.rows + row) * bp;
            for (int b = 0; b < bp; ++b) dd[b] = sd[b];
        }
    }
}

// The update of one (unit, mode) stage: split reduction, Eq. 3.4, operand copies.
static void mock_finish(const BatchFinish& f, const UpdateSpec& u) {
    for (int64_t e = 0; e < f.rows * f.rank; ++e) {
        const int64_t so = (e / f.rank) * f.bp + e % f.rank;
        float num = 0.f, den = 0.f;
        for (int s = 0; s < f.n_split; ++s) {
            num += f.part_num[(int64_t)s * f.s_size + so];
            den += f.part_den[(int64_t)s * f.s_size + so];
        }
        const float v = mu_update(f.theta[e], num, den, u);
        f.theta[e] = v;
        f.canon32[so] = v;
        f.canon16[so] = bf16_bits(v);
    }
}

// The persistent launch, one CTA: items taken in queue order; before an item the
// unit's preceding stage must be finished (the launch would wait for it), after it
// the stage counter rule decides whether this item applies the stage's update.
cudaError_t launch_batched_persistent(const PersistDesc& d, const WeightSpec&, int, cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        const uint64_t total = (uint64_t)d.n_items * (uint64_t)d.n_sweeps;
        for (uint64_t q = *d.queue; q < total; q = ++*d.queue) {
            const int sl = (int)(q / (uint64_t)d.n_items);
            const PersistItem it = d.items[q - (uint64_t)sl * d.n_items];
            const int s = d.sweep0 + sl;
            const int l = it.um / d.n_units, unit = it.um - l * d.n_units;
            const unsigned int seq = (unsigned int)(s * 3 + l);
            if (d.stage[unit] < seq) return cudaErrorInvalidValue;  // a CTA would wait for an item it holds
            mock_item(d.units, it.um, it.rb, it.sp, d.bp, 1);
            const unsigned int cum = (unsigned int)s * d.sweep_items[unit] + d.prefix_items[it.um] +
                                     d.stage_items[it.um];
            if (++d.done[unit] == cum) {
                mock_finish(d.fin[it.um], d.u);
                d.stage[unit] = seq + 1;
            }
        }
        return cudaSuccess;
    });
}

cudaError_t launch_pad_problem(const float* y, const uint8_t* mask, const int64_t* dims, const int64_t* pdims,
                               float* yp, uint32_t* bits, cudaStream_t) {
    const int64_t I = dims[0], J = dims[1], K = dims[2], Ip = pdims[0], Jp = pdims[1], Kp = pdims[2];
    return host_submit([=]() -> cudaError_t {
        const int64_t np = Ip * Jp * Kp;
        for (int64_t w = 0; w < (np + 31) / 32; ++w) bits[w] = 0u;
        for (int64_t i = 0; i < Ip; ++i)
            for (int64_t j = 0; j < Jp; ++j)
                for (int64_t k = 0; k < Kp; ++k) {
                    const int64_t e = (i * Jp + j) * Kp + k;
                    float v = 0.f;
                    bool obs = false;
                    if (i < I && j < J && k < K) {
                        const int64_t src = (i * J + j) * K + k;
                        v = y[src];
                        obs = mask ? mask[src] != 0 : true;
                    }
                    yp[e] = v;
                    if (obs) bits[e >> 5] |= 1u << (e & 31);
                }
        return cudaSuccess;
    });
}

cudaError_t launch_mirror_batched(const BatchFinish* fin, const int64_t* prefix, int n_units, int64_t,
                                  cudaStream_t) {
    return host_submit([=]() -> cudaError_t {
        for (int x = 0; x < n_units; ++x) {
            const BatchFinish& f = fin[x];
            for (int64_t e = 0; e < prefix[x + 1] - prefix[x]; ++e) {
                const int64_t so = (e / f.rank) * f.bp + e % f.rank;
                f.canon32[so] = f.theta[e];
                f.canon16[so] = bf16_bits(f.theta[e]);
            }
        }
        return cudaSuccess;
    });
}

cudaError_t launch_loss_batched(const float* y, const uint8_t* mask, const int64_t* dims, int rank, int restarts,
                                const BatchFactors& fac, const LossSpec& L, double*, int, double* out,
                                cudaStream_t) {
    const int64_t I = dims[0], J = dims[1], K = dims[2];
    return host_submit([=]() -> cudaError_t {
        for (int q = 0; q < restarts; ++q) {
            double acc = 0.0;
            const float *A = fac.f[q][0], *B = fac.f[q][1], *C = fac.f[q][2];
            for (int64_t e = 0; e < I * J * K; ++e) {
                if (mask && !mask[e]) continue;
                const int64_t k3 = e % K, j = (e / K) % J, i = e / (J * K);
                float yh = 0.f;
                for (int r = 0; r < rank; ++r) yh = std::fma(A[i * rank + r] * B[j * rank + r], C[k3 * rank + r], yh);
                acc += (double)divergence(y[e], yh, L);
            }
            out[q] = acc;
        }
        return cudaSuccess;
    });
}

}  // namespace nef
