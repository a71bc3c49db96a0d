// k_tc_probe.cu -- isolated check of the tcgen05 operand layouts used by the
// fused pass: one MMA1 (K-major A and B, swizzle by bond width) and one MMA2
// (K-major 128B-swizzled A, MN-major B) on caller-given BF16 tiles.
#include "../../include/nef_debug.h"
#include "k_view_tc.cuh"

namespace nef {
namespace tc {

template <int BP>
__global__ void __launch_bounds__(128, 1)
k_tc_probe(const uint16_t* __restrict__ P, const uint16_t* __restrict__ Q, const uint16_t* __restrict__ W,
           float* __restrict__ D1, float* __restrict__ D2, int* err) {
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
                     "r"(256u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    if (tid == 0) {
        constexpr uint32_t idesc1 = make_idesc(TM, TN, 0, 0);
        constexpr uint32_t idesc2 = make_idesc(TM, BP, 0, 1);
        for (int k = 0; k < BP / 16; ++k)
            tc_mma(tmem, make_sdesc(base + kP + k * 32, 16, 8 * RB, swz_code(RB)),
                   make_sdesc(base + kQ + k * 32, 16, 8 * RB, swz_code(RB)), idesc1, k > 0);
        for (int k = 0; k < TN / 16; ++k)
            tc_mma(tmem + 128, make_sdesc(base + kW + k * 32, 16, 1024, swz_code(128)),
                   make_sdesc(base + kQ + k * 16 * RB, TN * RB, 8 * RB, swz_code(RB)), idesc2, k > 0);
        tc_commit(bar);
    }
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar, 0, abort_flag, err, 1));
    tc_fence_after();
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    const int row = warp * 32 + lane;
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
    }
}

template <int BP>
cudaError_t run_probe(const uint16_t* P, const uint16_t* Q, const uint16_t* W, float* D1, float* D2, int* err,
                      cudaStream_t st) {
    constexpr int RB = BP * 2;
    constexpr int kQ = TM * RB, kW = ((kQ + TN * RB + 1023) / 1024) * 1024, kBar = kW + TM * TN * 2;
    const int sm = kBar + 64 + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_tc_probe<BP>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e != cudaSuccess) return e;
    k_tc_probe<BP><<<1, 128, sm, st>>>(P, Q, W, D1, D2, err);
    return cudaGetLastError();
}

}  // namespace tc
}  // namespace nef

extern "C" int nef_tc_probe(int bond_pad, const uint16_t* P, const uint16_t* Q, const uint16_t* W, float* D1,
                            float* D2, int* err, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (bond_pad) {
        case 16: e = nef::tc::run_probe<16>(P, Q, W, D1, D2, err, st); break;
        case 32: e = nef::tc::run_probe<32>(P, Q, W, D1, D2, err, st); break;
        case 64: e = nef::tc::run_probe<64>(P, Q, W, D1, D2, err, st); break;
        default: return 1;
    }
    return e == cudaSuccess ? 0 : 5;
}
