// k_tc_probe.cu -- isolated check of the tcgen05 operand layouts used by the
// fused pass: one MMA1 (K-major A and B, swizzle by bond width) and one MMA2
// (K-major A, MN-major B) on caller-given BF16 tiles, with the A operands
// either in shared memory (128B-swizzled) or in tensor memory (written by the
// threads with tcgen05.st, one row per lane).
#include "nef_probe.h"
#include "k_view_tc.cuh"

namespace nef {
namespace tc {

constexpr uint32_t kProbeCols = 512;

template <int BP>
__global__ void __launch_bounds__(128, 1)
k_tc_probe(const uint16_t* __restrict__ P, const uint16_t* __restrict__ Q, const uint16_t* __restrict__ W,
           float* __restrict__ D1, float* __restrict__ D2, int* err, int a_tmem) {
    constexpr int RB = BP * 2;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* sm = smem_raw + (base - raw);
    constexpr int kP = 0, kQ = kP + TM * RB, kW = ((kQ + TN * RB + 1023) / 1024) * 1024,
                  kBar = kW + TM * TN * 2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kBar + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kBar + 20);
    const uint32_t bar = base + kBar;
    for (int e = tid; e < TM * BP / 8; e += 128) {
        const int r = e / (BP / 8), j = e % (BP / 8);
        *reinterpret_cast<uint4*>(sm + kP + swz<RB>(r * RB + j * 16)) =
            *reinterpret_cast<const uint4*>(P + r * BP + j * 8);
    }
    for (int e = tid; e < TN * BP / 8; e += 128) {
        const int r = e / (BP / 8), j = e % (BP / 8);
        *reinterpret_cast<uint4*>(sm + kQ + swz<RB>(r * RB + j * 16)) =
            *reinterpret_cast<const uint4*>(Q + r * BP + j * 8);
    }
    for (int e = tid; e < TM * TN / 8; e += 128) {
        const int r = e / (TN / 8), j = e % (TN / 8);
        *reinterpret_cast<uint4*>(sm + kW + swz<128>(r * 128 + j * 16)) =
            *reinterpret_cast<const uint4*>(W + r * TN + j * 8);
    }
    fence_proxy_async();
    if (tid == 0) {
        mbar_init(bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "r"(kProbeCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    const int row = warp * 32 + lane;
    // A operands in TMEM: P at columns 256.., W at 320.. (row = lane)
    const uint32_t t_p = tmem + 256, t_w = tmem + 320;
    if (a_tmem) {
        uint32_t pr[BP / 2], wr[TN / 2];
        for (int c = 0; c < BP / 2; ++c) pr[c] = reinterpret_cast<const uint32_t*>(P + row * BP)[c];
        for (int c = 0; c < TN / 2; ++c) wr[c] = reinterpret_cast<const uint32_t*>(W + row * TN)[c];
        tmem_st<BP / 2>(t_p + lane_off, pr);
        tmem_st<TN / 2>(t_w + lane_off, wr);
        tmem_wait_st();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        constexpr uint32_t idesc1 = make_idesc(TM, TN, 0, 0);
        constexpr uint32_t idesc2 = make_idesc(TM, BP, 0, 1);
        for (int k = 0; k < BP / 16; ++k) {
            const uint64_t bd = make_sdesc(base + kQ + k * 32, 16, 8 * RB, swz_code(RB));
            if (a_tmem)
                tc_mma_ts(tmem, t_p + k * 8, bd, idesc1, k > 0);
            else
                tc_mma(tmem, make_sdesc(base + kP + k * 32, 16, 8 * RB, swz_code(RB)), bd, idesc1, k > 0);
        }
        for (int k = 0; k < TN / 16; ++k) {
            const uint64_t bd = make_sdesc(base + kQ + k * 16 * RB, TN * RB, 8 * RB, swz_code(RB));
            if (a_tmem)
                tc_mma_ts(tmem + 128, t_w + k * 8, bd, idesc2, k > 0);
            else
                tc_mma(tmem + 128, make_sdesc(base + kW + k * 32, 16, 1024, swz_code(128)), bd, idesc2, k > 0);
        }
        tc_commit(bar);
    }
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar, 0, abort_flag, err, 1));
    tc_fence_after();
    if (ok) {
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + lane_off + c0, r);
            tmem_wait_ld();
            for (int k = 0; k < 16; ++k) D1[row * TN + c0 + k] = __uint_as_float(r[k]);
        }
        for (int c0 = 0; c0 < BP; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + 128 + lane_off + c0, r);
            tmem_wait_ld();
            for (int k = 0; k < 16; ++k) D2[row * BP + c0 + k] = __uint_as_float(r[k]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kProbeCols)
                     : "memory");
    }
}

template <int BP>
cudaError_t run_probe(const uint16_t* P, const uint16_t* Q, const uint16_t* W, float* D1, float* D2, int* err,
                      int a_tmem, cudaStream_t st) {
    constexpr int RB = BP * 2;
    constexpr int kQ = TM * RB, kW = ((kQ + TN * RB + 1023) / 1024) * 1024, kBar = kW + TM * TN * 2;
    const int sm = kBar + 64 + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_tc_probe<BP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    k_tc_probe<BP><<<1, 128, sm, st>>>(P, Q, W, D1, D2, err, a_tmem);
    return cudaGetLastError();
}

}  // namespace tc
}  // namespace nef

extern "C" int nef_tc_probe(int bond_pad, int a_in_tmem, const uint16_t* P, const uint16_t* Q, const uint16_t* W,
                            float* D1, float* D2, int* err, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (bond_pad) {
        case 16: e = nef::tc::run_probe<16>(P, Q, W, D1, D2, err, a_in_tmem != 0, st); break;
        case 32: e = nef::tc::run_probe<32>(P, Q, W, D1, D2, err, a_in_tmem != 0, st); break;
        case 64: e = nef::tc::run_probe<64>(P, Q, W, D1, D2, err, a_in_tmem != 0, st); break;
        default: return 1;
    }
    return e == cudaSuccess ? 0 : 5;
}
