// k_view_tc.cuh -- tcgen05 fused pass (BF16 operands, FP32 TMEM accumulators).
//
// One CTA owns a block of 128 rows of the view Y[row, col] and a range of
// 64-column tiles.  Per tile:
//   TMA      : Y tile (128 x 64 FP32) -> shared memory (multi-stage ring)
//   Q warps  : Q tile (64 cols x BP bond, BF16, shared memory) = Hadamard
//              product of the source rows (Eq. 2.1 restricted to the column side)
//   MMA1     : yhat[128 x 64] = P[128 x BP] . Q^T       -> TMEM (P in TMEM)
//   epilogue : W_a = M*a(y, yhat), W_b = M*b(y, yhat)  (App. B) in FP32 registers,
//              rounded to BF16 and stored into TMEM (one tile row per lane)
//   MMA2     : S_a[128 x BP] += W_a[128 x 64] . Q[64 x BP]  -> TMEM (Eq. 3.6-3.8)
//              (and S_b with W_b when the denominator needs the contraction)
// yhat and the weights never leave the chip, and both A operands (P, W) are
// read by the tensor cores from TMEM, so shared-memory bandwidth is spent on
// the Y stream, the staged source rows and Q only.  At the end the epilogue
// warps copy S from TMEM to the per-split partial buffers.
//
// Warp roles (512 threads, 128 registers each): warp 0 TMA producer (Y tiles
// and the staged source rows) + TMEM allocator, warp 1 MMA issuer, warps 2-3
// Q operand builders (one thread per tile column), warps 4-15 epilogue in three
// groups of four that take turns on the tiles.  Epilogue warp w reads TMEM
// lanes 32*(w%4).. (one tile row per thread), so every SM sub-partition runs
// one warp of each group.  Every mbarrier wait is bounded: on timeout the CTA
// raises an error flag, drains its own in-flight copies and MMAs, frees TMEM
// and exits.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <type_traits>

#include "nef_batched.h"
#include "nef_device.cuh"
#include "nef_internal.h"
#include "nef_launch.cuh"

#ifndef NEF_TC_TRACE
#define NEF_TC_TRACE 0  // 1: per-site wait and phase cycle counters (nef_tc_trace; slows the pass)
#endif
#ifndef NEF_TC_SUSPEND_NS
#define NEF_TC_SUSPEND_NS 20000u
#endif
// ring depths (compile-time; the layout's static_asserts check shared memory and TMEM)
#ifndef NEF_TC_NSY64
#define NEF_TC_NSY64 4
#endif
#ifndef NEF_TC_NSV64
#define NEF_TC_NSV64 6
#endif
#ifndef NEF_TC_NSQ64
#define NEF_TC_NSQ64 5
#endif
#ifndef NEF_TC_NW
#define NEF_TC_NW 4
#endif
#ifndef NEF_TC_ND
#define NEF_TC_ND 4
#endif

namespace nef {
namespace tc {

constexpr int TM = 128;        // rows per CTA (TMEM lanes)
constexpr int TN = 64;         // columns per tile
constexpr int kThreads = 512;   // 16 warps: 128 registers per thread
constexpr int kOpWarps = 2;
constexpr int kGroupWarps = 4;  // one epilogue group: one warp per TMEM lane quarter
constexpr int kEpiGroups = 3;
constexpr int kEpiWarps = kEpiGroups * kGroupWarps;
constexpr int kEpiWarp0 = 2 + kOpWarps;  // first epilogue warp
constexpr int kYStageBytes = TM * TN * 4;   // 32 KB
constexpr uint32_t kTmemCols = 512;
// Default limit of the bounded waits (~2 s at 2 GHz).  The pipeline waits use the
// launch's limit (Params::wait_cycles); the drains at the end of a CTA, which wait
// for the CTA's own copies and products already in flight, always use this one,
// so that no copy into shared memory or product into tensor memory is still
// running when the CTA frees them, whatever the launch's limit.
constexpr long long kWaitCycles = 4000000000LL;

// Weight kinds with their own instances: the App. B (alpha,beta) cases KL (1,0),
// (1,-1/2) and (1/2,1/2), the likelihood families negative binomial, binomial on
// the odds and Jensen-Shannon, and the generic evaluation (any (alpha,beta) or
// family, selected at run time).
enum WeightKind { WK_GEN = 0, WK_KL = 1, WK_B05 = 2, WK_HEL = 3, WK_NB = 4, WK_BIN = 5, WK_JS = 6, WK_RKL = 7 };

struct Params {
    const uint32_t* mbits;
    ViewDesc v;
    WeightSpec w;
    int64_t n_tiles;          // column tiles of the whole view
    int64_t tiles_per_split;
    int64_t n_cib;            // column tiles per c_out slice (non-transposed view)
    int trans;                // 1: rows are the contiguous dimension (c_in == 1)
    float* s_num;
    float* s_den;
    int* err;
    unsigned long long* trace;  // optional: [kTraceSites] summed wait cycles per wait site
    // Q operand mode: 0 = gathered rows (any view); 1 = within every tile source
    // q_var has consecutive rows (TMA-staged with the Y tile) and source q_const
    // (or none, -1) a single row
    int qmode, q_var, q_const;
    // optional loss of the current factors (Eq. 3.1 with App. B's D): per-CTA
    // sums over observed entries at loss_part[cta], their count at
    // loss_part[n_ctas + cta]; NULL = not computed
    double* loss_part;
    LossSpec L;
    long long wait_cycles;    // limit of the pipeline waits (kWaitCycles by default)
};

constexpr int kTraceSites = 32;   // 0: CTA lifetime cycles, 1..13: wait sites, 16..: busy phases

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// Potentially blocking test of a phase: the thread may sleep until the phase
// completes or kSuspendNs nanoseconds pass, so waiting warps spend no issue slots.
constexpr uint32_t kSuspendNs = NEF_TC_SUSPEND_NS;
__device__ __forceinline__ uint32_t mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok;
}

// Non-blocking probe of a phase.
__device__ __forceinline__ uint32_t mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok;
}

// Limits below this many cycles poll without suspending and check the clock on
// every poll (a suspended try_wait can sleep for kSuspendNs, far beyond such a
// limit); longer limits suspend between polls and check every 16th.
constexpr long long kShortWait = 1LL << 20;

// Bounded wait.  Returns false (and raises the CTA abort flag) on timeout or
// when another role already aborted.  With a trace array, the cycles spent
// waiting are added to trace[code].
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err, int code, unsigned long long* trace = nullptr,
                                          long long limit = kWaitCycles) {
    const bool fast = limit < kShortWait;
    long long t0 = trace ? clock64() : 0;
    if (fast ? mbar_test(bar, parity) : mbar_try(bar, parity)) {
        if (trace) atomicAdd(&trace[code], (unsigned long long)(clock64() - t0));
        return true;
    }
    if (!trace) t0 = clock64();
    for (uint32_t it = 1;; ++it) {
        if (fast ? mbar_test(bar, parity) : mbar_try(bar, parity)) {
            if (trace) atomicAdd(&trace[code], (unsigned long long)(clock64() - t0));
            return true;
        }
        if (fast || (it & 15) == 0) {
            if (*abort_flag) return false;
            if (clock64() - t0 > limit) {
                *abort_flag = 1;
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}

// Busy-phase timer for the trace (lane 0 of a warp adds cycles since *t to site).
__device__ __forceinline__ void phase_mark(unsigned long long* tr, int site, long long& t) {
    if (tr) {
        const long long now = clock64();
        atomicAdd(&tr[site], (unsigned long long)(now - t));
        t = now;
    }
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accum)
        : "memory");
}

// Same product with the A operand read from tensor memory: rows of A in TMEM
// lanes 0..127, K packed along columns (two BF16 values per 32-bit column, the
// lower K index in the low half), starting at column address a_tmem.
__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// Elected-issue forms: the whole warp executes them with warp-uniform operands
// and elect.sync lets one lane issue.  Issuing from warp-uniform code keeps the
// operands in uniform registers; issuing from a one-lane branch costs several
// times more per instruction.  The same lane is elected every time, so commits
// track the MMAs that lane issued.
__device__ __forceinline__ void tc_mma_ts_e(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void tc_commit_e(uint32_t bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx_e(uint32_t bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n\t}" ::"r"(bar), "r"(bytes)
        : "memory");
}

__device__ __forceinline__ void tma_load_3d_e(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                              uint32_t bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n\t}" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d_e(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n\t}" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

// Store 8/16/32 consecutive 32-bit columns of this thread's TMEM lane.
template <int N>
__device__ __forceinline__ void tmem_st(uint32_t taddr, const uint32_t* r) {
    if constexpr (N == 8) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                     "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                     : "memory");
    } else if constexpr (N == 16) {
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
            "%13, %14, %15, %16};" ::"r"(taddr),
            "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
            "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
            : "memory");
    } else {
        static_assert(N == 32, "8, 16 or 32 columns");
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
            "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
            "%32};" ::"r"(taddr),
            "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
            "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]),
            "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]),
            "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
            : "memory");
    }
}

__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor (tcgen05): start address, leading and stride
// byte offsets, fixed version bits 46-48 = 0b001, swizzle mode in bits 61-63.
__device__ __forceinline__ uint64_t make_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t swz) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)(swz & 7u) << 61;
    return d;
}

// Swizzle-mode code of the descriptor for rows of `row_bytes` (32, 64 or 128 B).
__host__ __device__ constexpr uint32_t swz_code(int row_bytes) {
    return row_bytes == 128 ? 2u : (row_bytes == 64 ? 4u : 6u);
}

// Physical byte offset of logical byte offset `a` inside a swizzled tile whose
// rows are `row_bytes` long (32/64/128 B swizzle: address bits 7.. XOR into 4..).
template <int ROW_BYTES>
__device__ __forceinline__ uint32_t swz(uint32_t a) {
    constexpr uint32_t m = ROW_BYTES == 128 ? 7u : (ROW_BYTES == 64 ? 3u : 1u);
    return a ^ (((a >> 7) & m) << 4);
}

// Instruction descriptor of tcgen05.mma kind::f16: BF16 A and B, FP32 D.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N, int a_mn_major, int b_mn_major) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn_major << 15) |
           ((uint32_t)b_mn_major << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t mul_bf16x2(uint32_t a, uint32_t b) {
    const __nv_bfloat162 r =
        __hmul2(*reinterpret_cast<const __nv_bfloat162*>(&a), *reinterpret_cast<const __nv_bfloat162*>(&b));
    return *reinterpret_cast<const uint32_t*>(&r);
}

__device__ __forceinline__ void unpack_bf16x8(const uint4& q, float (&f)[8]) {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 t = __bfloat1622float2(h[i]);
        f[2 * i] = t.x;
        f[2 * i + 1] = t.y;
    }
}

// sqrt.approx / rsqrt.approx with subnormals flushed (one SFU operation each):
// the weights are rounded to BF16 next, so neither the correctly rounded square
// root nor subnormal inputs (yhat below 1.2e-38) buy anything here.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Mask of BF16 pair q of a 32-entry half: low half kept if bit 2q of the
// observed bits is set, high half if bit 2q+1 is.  sh[k] = obs << (7 - k)
// carries bits k, k+8, k+16, k+24 in the sign bits of its four bytes, so one
// byte permute with sign replication (prmt selector nibbles with the msb set)
// builds the mask from sh[2q mod 8] and sh[2q+1 mod 8].
__device__ __forceinline__ uint32_t pair_mask(const uint32_t (&sh)[8], int q) {
    const uint32_t b = (uint32_t)(q >> 2);
    const uint32_t sel = ((8u | b) * 0x11u) | (((8u | (4u + b)) * 0x11u) << 8);
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(sh[(2 * q) & 7]), "r"(sh[(2 * q + 1) & 7]), "r"(sel));
    return d;
}

// 32 x 32 bit transpose across a warp: lane c holds column c (bit r = row r); on
// return lane r holds row r (bit c = column c).  Five exchange steps swap the
// off-diagonal blocks of halving size (16, 8, 4, 2, 1 bits).
__device__ __forceinline__ uint32_t warp_transpose_bits(uint32_t x, int lane) {
    const uint32_t masks[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const int j = 16 >> k;
        const uint32_t m = masks[k];
        const uint32_t p = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? ((x & ~m) | ((p >> j) & m)) : ((x & m) | ((p & m) << j));
    }
    return x;
}

// One loss term D(y, yhat) in FP32 (App. B).  For KL the weight a = y / yhat
// is already at hand: D = y log(a) - y + yhat.
// log2 by one SFU operation, subnormals flushed; the loss terms built from it are
// summed over many entries in FP64, far beyond what its ~2^-22 error can change.
__device__ __forceinline__ float lg2_approx(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
constexpr float kLn2 = 0.69314718056f;
constexpr float kTiny = 1.17549435e-38f;  // smallest normal float

template <int WK>
__device__ __forceinline__ void tc_weights(float y, float yh, const WeightSpec& w, float& wa, float& wb) {
    if (WK == WK_KL) {
        wa = __fdividef(y, yh);
        wb = 1.0f;
    } else if (WK == WK_RKL) {
        wa = kLn2 * lg2_approx(__fdividef(y, yh));
        wb = 1.0f;
    } else if (WK == WK_NB) {
        const float phi = (float)w.par;
        wa = __fdividef(y, yh);
        wb = __fdividef(phi + y, phi + yh);
    } else if (WK == WK_BIN) {
        wa = __fdividef(y, yh);
        wb = __fdividef((float)w.par, 1.0f + yh);
    } else if (WK == WK_JS) {
        wa = kLn2 * lg2_approx(__fdividef(0.5f * (y + yh), yh));
        wb = 1.0f;
    } else if (WK == WK_B05) {
        const float r = rsqrt_approx(yh);
        wb = r;
        wa = y * r * r * r;
    } else if (WK == WK_HEL) {
        wa = sqrt_approx(y) * rsqrt_approx(yh);
        wb = 1.0f;
    } else {
        ab_weights(y, yh, w, wa, wb);
    }
}

// One loss term D(y, yhat) in FP32 (App. B), from the weights already at hand
// where the kind allows (a, b: the FP32 weights of tc_weights):
//   KL (1,0):        D = y ln(y/yhat) - y + yhat, a = y/yhat (a floored at the
//                    smallest normal float, so y = 0 gives 0 * finite = 0);
//   reverse KL (0,1): D = yhat ln(yhat/y) - yhat + y = y - yhat (1 + a), a = ln(y/yhat);
//   (1,-1/2):        D = 2y/sqrt(yhat) + 2 sqrt(yhat) - 4 sqrt(y) = 2 b (y + yhat) - 4 sqrt(y),
//                    b = 1/sqrt(yhat);
//   (1/2,1/2):       D = 2 (sqrt(y) - sqrt(yhat))^2 = 2 (y + yhat (1 - 2a)), a = sqrt(y/yhat);
//   Jensen-Shannon:  a = ln((y + yhat)/(2 yhat)) = -ln(yhat/m), m = (y + yhat)/2, so
//                    D = (y ln(y/m) + yhat ln(yhat/m))/2 = (y ln(y/m) - yhat a)/2;
//   negative binomial: D = (phi + y) ln(phi + yhat) - y ln yhat;
//   binomial on odds:  D = n ln(1 + yhat) - y ln yhat;
//   otherwise the generic five-case divergence.
template <int WK>
__device__ __forceinline__ float tc_loss(float y, float yh, float a, float b, const LossSpec& L) {
    if (WK == WK_KL) return fmaf(y * kLn2, lg2_approx(fmaxf(a, kTiny)), yh - y);
    if (WK == WK_RKL) return fmaf(-yh, 1.0f + a, y);
    if (WK == WK_B05) return fmaf(2.0f * b, y + yh, -4.0f * sqrt_approx(y));
    if (WK == WK_HEL) return 2.0f * fmaf(yh, fmaf(-2.0f, a, 1.0f), y);
    if (WK == WK_JS) {
        const float m = 0.5f * (y + yh);
        const float ly = y > 0.f ? y * (kLn2 * lg2_approx(__fdividef(y, m))) : 0.f;
        return 0.5f * (ly - yh * a);
    }
    if (WK == WK_NB) {
        const float phi = (float)L.par;
        return kLn2 * ((phi + y) * lg2_approx(phi + yh) - (y > 0.f ? y * lg2_approx(yh) : 0.f));
    }
    if (WK == WK_BIN) {
        return kLn2 * ((float)L.par * lg2_approx(1.0f + yh) - (y > 0.f ? y * lg2_approx(yh) : 0.f));
    }
    return divergence<float>(y, yh, L);
}

// 16 bytes of an operand row.  CG: through L2 only (ld.global.cg), for operands
// that an earlier stage of the same persistent launch rewrote from another SM,
// where a line left in this SM's L1 by an earlier stage could be stale.
template <bool CG>
__device__ __forceinline__ uint4 ld_row16(const uint16_t* p) {
    if constexpr (CG) return __ldcg(reinterpret_cast<const uint4*>(p));
    return *reinterpret_cast<const uint4*>(p);
}

__device__ __forceinline__ int64_t src_row_tc(const SrcDesc& s, int64_t i) {
    int64_t r = 0;
    if ((uint64_t)i < 0xffffffffull) {  // 32-bit division when the index fits (div, mod <= index range)
        const uint32_t i32 = (uint32_t)i;
        for (int t = 0; t < s.nterm; ++t) {
            const uint32_t d = (uint32_t)min(s.div[t], (int64_t)0xffffffff);
            const uint32_t m = (uint32_t)min(s.mod[t], (int64_t)0xffffffff);
            r += (int64_t)((i32 / d) % m) * s.mul[t];
        }
        return r;
    }
    for (int t = 0; t < s.nterm; ++t) r += ((i / s.div[t]) % s.mod[t]) * s.mul[t];
    return r;
}

// ---------------------------------------------------------- shared layout
// Ring depths of a layout: configuration 0 (the default) and configuration 1 (an
// alternative the autotuner may choose per view: one more Y stage at the cost of
// the staged-row and Q rings where shared memory allows, else deeper operand rings).
template <int BP, int CFG>
struct Rings {
    static constexpr int NSY = CFG == 0 ? ((BP == 64) ? NEF_TC_NSY64 : (BP == 32 ? 5 : 6))
                                        : ((BP == 64) ? 5 : (BP == 32 ? 6 : 5));
    static constexpr int NSV = CFG == 0 ? ((BP == 64) ? NEF_TC_NSV64 : 8) : ((BP == 64) ? 3 : (BP == 32 ? 4 : 12));
    static constexpr int NSQ = CFG == 0 ? ((BP == 64) ? NEF_TC_NSQ64 : 6) : ((BP == 64) ? 4 : (BP == 32 ? 4 : 8));
};

template <int BP, bool DEN, int CFG = 0>
struct Layout {
    // Shared memory holds only what the async proxy brings in (Y, staged source
    // rows) and the Q operand; the A operands of both products (P, W) live in
    // tensor memory, so the shared-memory bandwidth of a tile goes to the Y
    // stream.  Ring depths: as many Y stages (bytes in flight towards HBM
    // latency) as fit next to the Q stages.
    static constexpr int NSY = Rings<BP, CFG>::NSY;  // Y stages
    static constexpr int NSV = Rings<BP, CFG>::NSV;  // staged source-row stages
    static constexpr int NSQ = Rings<BP, CFG>::NSQ;  // Q stages
    static constexpr int NW = DEN ? (BP == 16 ? 3 : 2) : NEF_TC_NW;              // W buffers (TMEM)
    static constexpr int ND = DEN ? (BP == 64 ? 3 : 4) : NEF_TC_ND;             // yhat buffers (TMEM)
    static constexpr int RB = BP * 2;                        // bytes per bond row (BF16)
    static constexpr int kY = 0;                             // NSY x 32 KB
    static constexpr int kV = kY + NSY * kYStageBytes;       // NSV x TN x RB: TMA-staged source rows
    static constexpr int kQ = kV + NSV * TN * RB;            // NSQ x TN x RB
    static constexpr int kQStage = TN * RB;
    // NSV slots of kGSlot bytes: TMA-staged constant row (tensor-copy destinations are
    // 128-byte aligned)
    static constexpr int kGSlot = 128;
    static constexpr int kG = kQ + NSQ * kQStage;
    static constexpr int kBar = kG + NSV * kGSlot;
    static_assert(kY % 1024 == 0 && kV % 1024 == 0 && (TN * RB) % 256 == 0 && kG % 128 == 0 &&
                      kGSlot >= RB,
                  "TMA destinations must stay aligned");
    // barriers: yfull[NSY], yempty[NSY], qfull[NSQ], qempty[NSQ], dfull[ND], dempty[ND],
    //           wfull[NW], wempty[NW], pfull, sfull, drain, vfull[NSV], vempty[NSV]
    static constexpr int kNumBars = 2 * NSY + 2 * NSQ + 2 * ND + 2 * NW + 3 + 2 * NSV;
    static constexpr int kMisc = kBar + kNumBars * 8;         // tmem slot + abort flag
    static constexpr int kTrace = kMisc + 16;                 // kTraceSites counters
    static constexpr int kLoss = kTrace + kTraceSites * 8;    // per epilogue warp: loss sum, count
    static constexpr int kTotal = kLoss + kEpiWarps * 16;
    static constexpr int kAlloc = kTotal + 1024;              // slack for 1024-B alignment
    static_assert(kAlloc <= 232448, "shared memory per CTA");
    // tensor-memory columns (128 lanes x 32 bit): yhat buffers, S_num, S_den, P
    // (BF16 pairs), W_a and W_b buffers (64 BF16 = 32 columns each)
    static constexpr uint32_t cS = ND * TN;
    static constexpr uint32_t cP = ((cS + (DEN ? 2 : 1) * BP + 31) / 32) * 32;
    static constexpr uint32_t cWa = cP + ((BP / 2 + 31) / 32) * 32;
    static constexpr uint32_t cWb = cWa + NW * 32;
    static_assert(cWb + (DEN ? NW * 32 : 0) <= kTmemCols, "tensor-memory columns");
};

// The fused pass of one CTA: rows [rb*TM, rb*TM + TM) of the view and the
// column tiles of split sp.
// QM: the Q-operand path compiled in: 0 gathered rows, 1 TMA-staged rows
// (prm.qmode must match), 2 both, chosen by prm.qmode at run time (batched launches)
// CG: operand rows by L2-only loads and, at the end, every mbarrier invalidated so
// that the next work item of a persistent CTA can initialise them again.
template <int BP, bool DEN, int WK, bool LOSS, int QM, bool CG = false, int CFG = 0>
__device__ __forceinline__ void view_tc_body(const CUtensorMap* ymap, const CUtensorMap* vmap,
                                             const CUtensorMap* cmap, const Params& prm, const int64_t rb,
                                             const int64_t sp) {
    using LY = Layout<BP, DEN, CFG>;
    constexpr int RB = LY::RB;
    constexpr int NSY = LY::NSY;
    constexpr int NSQ = LY::NSQ;
    constexpr int NW = LY::NW;
    constexpr int ND = LY::ND;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw_addr = smem_u32(smem_raw);
    const uint32_t base = (raw_addr + 1023u) & ~1023u;
    uint8_t* sm = smem_raw + (base - raw_addr);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const ViewDesc& v = prm.v;
    const int64_t r0 = rb * TM;
    const int64_t t_lo = sp * prm.tiles_per_split;
    const int64_t t_hi = min(t_lo + prm.tiles_per_split, prm.n_tiles);
    const int T = (int)max((int64_t)0, t_hi - t_lo);

    const uint32_t bar0 = base + LY::kBar;
    auto yfull = [&](int s) { return bar0 + 8u * s; };
    auto yempty = [&](int s) { return bar0 + 8u * (NSY + s); };
    auto qfull = [&](int s) { return bar0 + 8u * (2 * NSY + s); };
    auto qempty = [&](int s) { return bar0 + 8u * (2 * NSY + NSQ + s); };
    auto dfull = [&](int b) { return bar0 + 8u * (2 * NSY + 2 * NSQ + b); };
    auto dempty = [&](int b) { return bar0 + 8u * (2 * NSY + 2 * NSQ + ND + b); };
    auto wfull = [&](int b) { return bar0 + 8u * (2 * NSY + 2 * NSQ + 2 * ND + b); };
    auto wempty = [&](int b) { return bar0 + 8u * (2 * NSY + 2 * NSQ + 2 * ND + NW + b); };
    const uint32_t pfull = bar0 + 8u * (2 * NSY + 2 * NSQ + 2 * ND + 2 * NW);
    const uint32_t sfull = pfull + 8u;
    const uint32_t drain = pfull + 16u;
    auto vfull = [&](int s) { return drain + 8u * (1 + s); };
    auto vempty = [&](int s) { return drain + 8u * (1 + LY::NSV + s); };
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + LY::kMisc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + LY::kMisc + 4);
#if NEF_TC_TRACE
    unsigned long long* tr = prm.trace ? reinterpret_cast<unsigned long long*>(sm + LY::kTrace) : nullptr;
#else
    constexpr unsigned long long* tr = nullptr;  // wait counters compiled out (build with NEF_TC_TRACE=1)
#endif
    const bool qmode = (QM == 2) ? (prm.qmode != 0) : (QM == 1);
    const long long t_start = clock64();
    if (tr && tid < kTraceSites) tr[tid] = 0ull;

    if (tid == 0) {
        for (int s = 0; s < NSY; ++s) {
            mbar_init(yfull(s), 1);
            mbar_init(yempty(s), kGroupWarps);
        }
        for (int s = 0; s < LY::NSV; ++s) {
            mbar_init(vfull(s), 1);
            mbar_init(vempty(s), kOpWarps);
        }
        for (int s = 0; s < NSQ; ++s) { mbar_init(qfull(s), kOpWarps); mbar_init(qempty(s), 1); }
        // yhat, Y and W buffers of a tile are released by the four warps of the
        // epilogue group that processes it; P is written by epilogue group 0
        for (int b = 0; b < ND; ++b) {
            mbar_init(dfull(b), 1);
            mbar_init(dempty(b), kGroupWarps);
        }
        for (int b = 0; b < NW; ++b) {
            mbar_init(wfull(b), kGroupWarps);
            mbar_init(wempty(b), 1);
        }
        mbar_init(pfull, kGroupWarps);
        mbar_init(sfull, 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        // a CTA that gives up its allocation permit may not allocate again: a persistent
        // CTA (CG), which allocates once per work item, keeps it
        if constexpr (!CG) asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t t_snum = tmem + LY::cS;
    const uint32_t t_sden = tmem + LY::cS + BP;
    const uint32_t t_p = tmem + LY::cP;
    const uint32_t t_wa = tmem + LY::cWa;
    const uint32_t t_wb = tmem + LY::cWb;

    // Column-tile cursor: tile t is tile `ci` of c_out slice `co` (non-transposed
    // view) or tile t of the transposed view (co stays 0).  Every role starts one
    // at t_lo and advances it tile by tile, so no role divides per tile.
    struct Cursor {
        int64_t co, ci;
    };
    auto cursor_at = [&](int64_t t) {
        Cursor c;
        if (prm.trans) {
            c.co = 0;
            c.ci = t;
        } else {
            c.co = t / prm.n_cib;
            c.ci = t - c.co * prm.n_cib;
        }
        return c;
    };
    auto advance = [&](Cursor& c) {
        if (++c.ci == prm.n_cib && !prm.trans) {
            c.ci = 0;
            ++c.co;
        }
    };
    auto tile_info = [&](const Cursor& c, int64_t& col0, int& nvalid, int& x0, int& z0) {
        const int64_t ci0 = c.ci * TN;
        x0 = (int)ci0;
        if (prm.trans) {
            col0 = ci0;
            nvalid = (int)min((int64_t)TN, v.c_out - ci0);
            z0 = 0;
        } else {
            col0 = c.co * v.c_in + ci0;
            nvalid = (int)min((int64_t)TN, v.c_in - ci0);
            z0 = (int)c.co;
        }
    };

    // waits of the warp-uniform producer and MMA loops (every lane polls)
    const long long wlim = prm.wait_cycles;
    auto uwait = [&](uint32_t bar, uint32_t par, int code) {
        return __all_sync(0xffffffffu,
                          mbar_wait(bar, par, abort_flag, prm.err, code, lane == 0 ? tr : nullptr, wlim));
    };
    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        // The whole warp runs the loop; one elected lane issues the copies.
        {
            // Staged source rows (qmode 1) run NSV - 1 tiles ahead of the Y stream.
            // When c_in is 1 or a multiple of TN, tile t starts at column t*TN: the
            // staged row (col mod m, m a multiple of TN) advances by TN per tile and
            // the constant row ((col / d) mod m, d a multiple of TN) by one every
            // d / TN tiles.  In the block form (c_in > 1 not a multiple of TN) the
            // tiles restart at every c_in block: the staged row is the tile's offset
            // in the block (m == c_in) and the constant row advances by one every
            // d / c_in blocks.  All are kept as counters.
            constexpr int NSV = LY::NSV;
            const bool has_c = prm.q_const >= 0;
            const bool block = !prm.trans && (v.c_in % TN) != 0;
            int64_t vrow = 0, vmod = 1, crow = 0, cmod = 1, cc = 0, per = 1, ci = 0;
            if (qmode) {
                const SrcDesc& dv = v.Q.src[prm.q_var];
                vmod = dv.mod[0];
                const int64_t unit = block ? v.c_in : TN;  // columns per step of the constant row
                const int64_t step = block ? t_lo / prm.n_cib : t_lo;  // blocks (or tiles) before t_lo
                ci = block ? t_lo - step * prm.n_cib : 0;
                vrow = block ? ci * TN : (t_lo * TN) % vmod;
                if (has_c) {
                    const SrcDesc& dc = v.Q.src[prm.q_const];
                    per = dc.div[0] / unit;
                    cmod = dc.mod[0];
                    const int64_t g = step / per;
                    cc = step - g * per;
                    crow = g % cmod;
                }
            }
            int iv = 0;
            bool vok = true;
            auto issue_v = [&]() {
                const int sv = iv % NSV;
                // slot of tile iv - NSV: free once every operand warp has built that Q
                if (!uwait(vempty(sv), ((iv / NSV) & 1) ^ 1, 14)) {
                    vok = false;
                    return;
                }
                mbar_expect_tx_e(vfull(sv), TN * RB + (has_c ? RB : 0));
                tma_load_2d_e(base + LY::kV + sv * (TN * RB), vmap, 0, (int)vrow, vfull(sv));
                if (has_c) tma_load_2d_e(base + LY::kG + sv * LY::kGSlot, cmap, 0, (int)crow, vfull(sv));
                bool next_c = true;
                if (block) {
                    vrow += TN;
                    next_c = ++ci == prm.n_cib;
                    if (next_c) {
                        ci = 0;
                        vrow = 0;
                    }
                } else {
                    vrow += TN;
                    if (vrow == vmod) vrow = 0;
                }
                if (next_c && ++cc == per) {
                    cc = 0;
                    if (++crow == cmod) crow = 0;
                }
                ++iv;
            };
            if (qmode)
                while (vok && iv < T && iv < NSV - 1) issue_v();
            int issued = 0;
            Cursor cur = cursor_at(t_lo);
            for (int i = 0; i < T; ++i) {
                if (qmode && vok && iv < T) issue_v();  // rows of tile i + NSV - 1
                if (!vok) break;
                const int s = i % NSY;
                if (!uwait(yempty(s), ((i / NSY) & 1) ^ 1, 1)) break;
                int64_t col0;
                int nvalid, x0, z0;
                tile_info(cur, col0, nvalid, x0, z0);
                advance(cur);
                const uint32_t dst = base + LY::kY + s * kYStageBytes;
                mbar_expect_tx_e(yfull(s), kYStageBytes);
                if (prm.trans) {
                    tma_load_2d_e(dst, ymap, (int)r0, x0, yfull(s));
                } else {
                    tma_load_3d_e(dst, ymap, x0, (int)r0, z0, yfull(s));
                    tma_load_3d_e(dst + kYStageBytes / 2, ymap, x0 + 32, (int)r0, z0, yfull(s));
                }
                issued = i + 1;
            }
            // drain: make sure no bulk copy into this CTA's memory is still in flight
            for (int i = max(0, issued - NSY); i < issued; ++i) {
                volatile int dummy_abort = 0;
                mbar_wait(yfull(i % NSY), (i / NSY) & 1, &dummy_abort, prm.err, 2);
            }
            for (int k = max(0, iv - NSV); k < iv; ++k) {
                volatile int dummy_abort = 0;
                mbar_wait(vfull(k % NSV), (k / NSV) & 1, &dummy_abort, prm.err, 2);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        // The whole warp runs the loop; one elected lane (the same one every time)
        // issues the MMAs and the commits that track them.
        {
            constexpr uint32_t idesc1 = make_idesc(TM, TN, 0, 0);
            constexpr uint32_t idesc2 = make_idesc(TM, BP, 0, 1);
            bool ok = uwait(pfull, 0, 3);
            // Q descriptors of stage 0 (the 14-bit start-address field of a stage or
            // K-step offset is added to it; shared addresses stay below 256 KB)
            const uint64_t qdesc1 = make_sdesc(base + LY::kQ, 16, 8 * RB, swz_code(RB));
            const uint64_t qdesc2 = make_sdesc(base + LY::kQ, TN * RB, 8 * RB, swz_code(RB));
            // MMA1 of tile i: yhat into TMEM buffer i % ND
            auto mma1 = [&](int i) -> bool {
                const int sq = i % NSQ, b = i % ND;
                if (!uwait(qfull(sq), (i / NSQ) & 1, 4)) return false;
                if (!uwait(dempty(b), ((i / ND) & 1) ^ 1, 5)) return false;
                tc_fence_after();
                // descriptor of K-step k: start address field advanced by k * 32 B
                const uint64_t bd0 = qdesc1 + (uint64_t)((sq * LY::kQStage) >> 4);
#pragma unroll
                for (int k = 0; k < BP / 16; ++k)
                    tc_mma_ts_e(tmem + b * TN, t_p + k * 8, bd0 + (uint64_t)(k * 2), idesc1, k > 0 ? 1u : 0u);
                tc_commit_e(dfull(b));
                return true;
            };
            // MMA2 of tile i: S += W(i) . Q(i); frees the W buffer and the Q stage
            auto mma2 = [&](int i) {
                const int bw = i % NW, sq = i % NSQ;
                tc_fence_after();
                const uint64_t bd0 = qdesc2 + (uint64_t)((sq * LY::kQStage) >> 4);
#pragma unroll
                for (int k = 0; k < TN / 16; ++k) {
                    const uint64_t bd = bd0 + (uint64_t)((k * 16 * RB) >> 4);
                    const uint32_t acc = (i > 0 || k > 0) ? 1u : 0u;
                    tc_mma_ts_e(t_snum, t_wa + bw * 32 + k * 8, bd, idesc2, acc);
                    if (DEN) tc_mma_ts_e(t_sden, t_wb + bw * 32 + k * 8, bd, idesc2, acc);
                }
                tc_commit_e(wempty(bw));
                tc_commit_e(qempty(sq));
            };
            // MMA1 runs LA tiles ahead of MMA2.  LA < NSQ keeps the Q stage of tile
            // i + LA free once MMA2(i - 1) is issued, LA < ND the yhat buffer once the
            // epilogue has finished tile i - 1, so the blocking waits cannot deadlock.
            // With LA >= kEpiGroups, the group that finishes tile i - kEpiGroups finds
            // yhat of its next tile i already issued.
            constexpr int LA = ND - 1;
            static_assert(LA < NSQ && LA < ND, "MMA1 look-ahead");
            for (int j = 0; ok && j < LA && j < T; ++j) ok = mma1(j);
            for (int i = 0; ok && i < T; ++i) {
                if (i + LA < T && !mma1(i + LA)) break;
                if (!uwait(wfull(i % NW), (i / NW) & 1, 6)) break;
                mma2(i);
            }
            tc_commit_e(sfull);
            // drain: wait until every MMA issued by the elected lane has completed
            tc_commit_e(drain);
            volatile int dummy_abort = 0;
            mbar_wait(drain, 0, &dummy_abort, prm.err, 7);
        }
    } else if (warp < kEpiWarp0) {
        // ------------------------------------------------------ Q operand builders
        // Thread q builds column cq of every Q tile (all bond chunks; in the
        // gathered mode in two halves of NH chunks).
        const int q = tid - 64;                 // 0 .. kOpWarps*32 - 1
        constexpr int NCH = BP / 8;             // 16-byte chunks per bond row
        static_assert(kOpWarps * 32 == TN, "one operand thread per tile column");
        const int cq = q;
        if (QM != 0 && qmode) {
            // The rows of source q_var and the single row of source q_const (if any) of
            // each tile are staged by TMA in their own ring, NSV - 1 tiles ahead of the
            // tile's Y (they are small and mostly L2-resident), so Q and yhat can be
            // ready before the Y tile arrives.  Q = the elementwise product of the rows.
            constexpr int NSV = LY::NSV;
            const bool has_c = prm.q_const >= 0;
            long long tp = clock64();
            const bool trl = tr && lane == 0;
            // A qmode-1 tile is full (c_in is a multiple of TN, or c_in == 1 and c_out
            // is a multiple of the staged source's extent) or, in the block form, ends
            // at its c_in block, where the staged rows past c_in arrive as zeros: the
            // build has no column predicate.
#pragma unroll 1
            for (int i = 0; i < T; ++i) {
                const int s = i % NSV, sq = i % NSQ;
                if (!__all_sync(0xffffffffu, mbar_wait(vfull(s), (i / NSV) & 1, abort_flag, prm.err, 13,
                                                       lane == 0 ? tr : nullptr, wlim)))
                    break;
                if (!__all_sync(0xffffffffu, mbar_wait(qempty(sq), ((i / NSQ) & 1) ^ 1, abort_flag, prm.err, 8,
                                                       lane == 0 ? tr : nullptr, wlim)))
                    break;
                if (trl) tp = clock64();
                const uint8_t* vsrc = sm + LY::kV + s * (TN * RB);
                const uint8_t* gsrc = sm + LY::kG + s * LY::kGSlot;
                uint8_t* qdst = sm + LY::kQ + sq * LY::kQStage;
                uint4 vv[NCH];
#pragma unroll
                for (int jj = 0; jj < NCH; ++jj)
                    vv[jj] = *reinterpret_cast<const uint4*>(vsrc + swz<RB>(cq * RB + jj * 16));
                if (has_c) {
                    // packed BF16 products: the exact product of two BF16 values fits
                    // in FP32, so this rounds exactly like an FP32 product converted
                    // to BF16
#pragma unroll
                    for (int jj = 0; jj < NCH; ++jj) {
                        const uint4 gv = *reinterpret_cast<const uint4*>(gsrc + jj * 16);
                        vv[jj].x = mul_bf16x2(vv[jj].x, gv.x);
                        vv[jj].y = mul_bf16x2(vv[jj].y, gv.y);
                        vv[jj].z = mul_bf16x2(vv[jj].z, gv.z);
                        vv[jj].w = mul_bf16x2(vv[jj].w, gv.w);
                    }
                }
#pragma unroll
                for (int jj = 0; jj < NCH; ++jj)
                    *reinterpret_cast<uint4*>(qdst + swz<RB>(cq * RB + jj * 16)) = vv[jj];
                if (trl) phase_mark(tr, 17, tp);
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(vempty(s));
                    mbar_arrive(qfull(sq));
                }
                if (trl) phase_mark(tr, 18, tp);
            }

        } else if constexpr (QM != 1) {
        // Gathered rows, in steps of half a column: step 2i + h builds chunks
        // [h*NH, h*NH + NH) of tile i.  The rows of the next step are loaded while
        // the current one is built, so the L2 latency of the gathers overlaps the
        // build and the wait for a free stage.
        constexpr int NH = NCH / 2;
        const int nsrc = v.Q.nsrc;
        const uint16_t* s0 = static_cast<const uint16_t*>(v.Q.src[0].ptr);
        const uint16_t* s1 = static_cast<const uint16_t*>(v.Q.src[nsrc > 1 ? 1 : 0].ptr);
        const int64_t ld0 = v.Q.src[0].ld, ld1 = v.Q.src[nsrc > 1 ? 1 : 0].ld;
        uint4 nx0[NH], nx1[NH];
        int64_t nrow[kMaxSrc];
        bool nok = false;
        Cursor gcur = cursor_at(t_lo);
        auto issue = [&](int hs) {  // rows of half hs of the tile at gcur into nx0/nx1
            int64_t col0;
            int nvalid, x0, z0;
            tile_info(gcur, col0, nvalid, x0, z0);
            if (hs == 1) advance(gcur);
            nok = cq < nvalid;
            const int64_t col = col0 + cq;
#pragma unroll
            for (int s2 = 0; s2 < kMaxSrc; ++s2)
                nrow[s2] = (nok && s2 < nsrc) ? src_row_tc(v.Q.src[s2], col) : 0;
#pragma unroll
            for (int j = 0; j < NH; ++j) {
                const int jj = hs * NH + j;
                nx0[j] = nok ? ld_row16<CG>(s0 + nrow[0] * ld0 + jj * 8) : make_uint4(0, 0, 0, 0);
                nx1[j] = (nok && nsrc > 1) ? ld_row16<CG>(s1 + nrow[1] * ld1 + jj * 8)
                                           : make_uint4(0, 0, 0, 0);
            }
        };
        if (T > 0) issue(0);
#pragma unroll 1
        for (int st = 0; st < 2 * T; ++st) {
            const int i = st >> 1, hh = st & 1;
            uint4 c0[NH], c1[NH];
            int64_t crow[kMaxSrc];
#pragma unroll
            for (int j = 0; j < NH; ++j) { c0[j] = nx0[j]; c1[j] = nx1[j]; }
#pragma unroll
            for (int s2 = 0; s2 < kMaxSrc; ++s2) crow[s2] = nrow[s2];
            const bool cok = nok;
            if (st + 1 < 2 * T) issue((st + 1) & 1);
            const int sq = i % NSQ;
            if (hh == 0 && !__all_sync(0xffffffffu, mbar_wait(qempty(sq), ((i / NSQ) & 1) ^ 1, abort_flag,
                                                              prm.err, 8, lane == 0 ? tr : nullptr, wlim)))
                break;
            uint8_t* qdst = sm + LY::kQ + sq * LY::kQStage;
#pragma unroll
            for (int j = 0; j < NH; ++j) {
                const int jj = hh * NH + j;
                float acc[8], f[8];
                unpack_bf16x8(c0[j], acc);
                if (nsrc > 1) {
                    unpack_bf16x8(c1[j], f);
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc[e] *= f[e];
                }
                for (int s2 = 2; s2 < nsrc; ++s2) {
                    const uint16_t* sb = static_cast<const uint16_t*>(v.Q.src[s2].ptr);
                    const uint4 raw = cok ? ld_row16<CG>(sb + crow[s2] * v.Q.src[s2].ld + jj * 8)
                                          : make_uint4(0, 0, 0, 0);
                    unpack_bf16x8(raw, f);
#pragma unroll
                    for (int e = 0; e < 8; ++e) acc[e] *= f[e];
                }
                uint4 outv;
                outv.x = pack_bf16(acc[0], acc[1]);
                outv.y = pack_bf16(acc[2], acc[3]);
                outv.z = pack_bf16(acc[4], acc[5]);
                outv.w = pack_bf16(acc[6], acc[7]);
                *reinterpret_cast<uint4*>(qdst + swz<RB>(cq * RB + jj * 16)) = outv;
            }
            if (hh == 1) {
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) mbar_arrive(qfull(sq));
            }
        }
        }
    } else {
        // ------------------------------------------------------ epilogue
        // kEpiGroups groups of four warps take turns on the tiles (group h: tiles
        // h, h + kEpiGroups, ...), so one group's weight arithmetic overlaps the
        // others' waits and loads.  Warp w of a group owns TMEM lanes 32*(w%4)..
        // (one tile row per thread) and all 64 columns of its tiles, in two halves
        // of 32.  Group 0 also writes P into TMEM before its first tile.
        const int e = ((warp & 3) << 5) + lane;      // tile row == TMEM lane
        const int h = (warp - kEpiWarp0) >> 2;        // group
        const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;
        const int64_t row = r0 + e;
        const bool row_ok = row < v.rows;
        const WeightSpec w = prm.w;
        auto wwait = [&](uint32_t bar, uint32_t par, int code) {
            const bool ok = mbar_wait(bar, par, abort_flag, prm.err, code, lane == 0 ? tr : nullptr, wlim);
            return __all_sync(0xffffffffu, ok);
        };
        const bool trl = tr && lane == 0;
        long long tp = clock64();
        if (h == 0) {
            // P row of TMEM lane e (this warp's lane quarter)
            const SrcDesc& ps = v.P.src[0];
            const uint16_t* pbase = static_cast<const uint16_t*>(ps.ptr);
            constexpr int NCH = BP / 8;
            const int64_t pr = row_ok ? src_row_tc(ps, row) : 0;
            uint32_t pv[BP / 2];
#pragma unroll
            for (int j = 0; j < NCH; ++j) {
                const uint4 x =
                    row_ok ? ld_row16<CG>(pbase + pr * ps.ld + j * 8) : make_uint4(0, 0, 0, 0);
                pv[4 * j] = x.x;
                pv[4 * j + 1] = x.y;
                pv[4 * j + 2] = x.z;
                pv[4 * j + 3] = x.w;
            }
            tmem_st<(BP / 2 < 8 ? 8 : BP / 2)>(t_p + lane_off, pv);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(pfull);
        }
        Cursor cur = cursor_at(t_lo);
        for (int k = 0; k < h; ++k) advance(cur);
        constexpr bool do_loss = LOSS;
        double lsum = 0.0, lcnt = 0.0;
#pragma unroll 1
        for (int i = h; i < T; i += kEpiGroups) {
            const int bd = i % ND, b = i % NW, s = i % NSY;
            int64_t col0;
            int nvalid, x0, z0;
            tile_info(cur, col0, nvalid, x0, z0);
            for (int k = 0; k < kEpiGroups; ++k) advance(cur);
            // mask words of both halves, loaded before the waits so that their
            // latency overlaps them (masked views only; see below for the layouts)
            uint32_t mw0a = 0u, mw0b = 0u, mw1a = 0u, mw1b = 0u;
            if constexpr (DEN) {
                if (prm.mbits) {
                    const int nv0 = min(32, nvalid), nv1 = min(32, max(0, nvalid - 32));
                    if (prm.trans) {
                        if ((v.rows & 31) == 0 && row_ok) {
                            const int64_t wstride = v.rows >> 5;
                            const int64_t wb0 = (col0 * v.rows + r0 + 32 * (warp & 3)) >> 5;
                            const int64_t wb1 = wb0 + 32 * wstride;
                            if (lane < nv0) mw0a = prm.mbits[wb0 + (int64_t)lane * wstride];
                            if (lane < nv1) mw1a = prm.mbits[wb1 + (int64_t)lane * wstride];
                        }
                    } else if (row_ok) {
                        // a tile lies inside one c_in block: its block is z0, its offset x0
                        const int64_t idx0 = ((int64_t)z0 * v.rows + row) * v.c_in + x0;
                        const int64_t i1 = idx0 + 32;
                        if (nv0 > 0) {
                            mw0a = prm.mbits[idx0 >> 5];
                            if (idx0 & 31) mw0b = prm.mbits[(idx0 >> 5) + 1];
                        }
                        if (nv1 > 0) {
                            mw1a = prm.mbits[i1 >> 5];
                            if (i1 & 31) mw1b = prm.mbits[(i1 >> 5) + 1];
                        }
                    }
                }
            }
            if (!wwait(dfull(bd), (i / ND) & 1, 9)) break;
            if (!wwait(yfull(s), (i / NSY) & 1, 10)) break;
            if (!wwait(wempty(b), ((i / NW) & 1) ^ 1, 11)) break;
            if (trl) tp = clock64();
            tc_fence_after();
            const uint8_t* ys = sm + LY::kY + s * kYStageBytes;
#pragma unroll 1
            for (int hh = 0; hh < 2; ++hh) {
                uint32_t yh[32];
                tmem_ld32(tmem + lane_off + bd * TN + 32 * hh, yh);
                float yv[32];
                if (prm.trans) {
#pragma unroll
                    for (int c = 0; c < 32; ++c)
                        yv[c] = *reinterpret_cast<const float*>(ys + (32 * hh + c) * (TM * 4) + e * 4);
                } else {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float4 f = *reinterpret_cast<const float4*>(ys + hh * (kYStageBytes / 2) + e * 128 +
                                                                          ((j ^ (e & 7)) << 4));
                        yv[4 * j + 0] = f.x;
                        yv[4 * j + 1] = f.y;
                        yv[4 * j + 2] = f.z;
                        yv[4 * j + 3] = f.w;
                    }
                }
                tmem_wait_ld();
                if (hh == 1) {
                    // both halves of yhat and Y are in registers: release the buffers
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(dempty(bd));
                        mbar_arrive(yempty(s));
                    }
                }
                // observed columns of this row within the half: bit c of `obs`
                const int nv = min(32, max(0, nvalid - 32 * hh));
                uint32_t obs = row_ok ? (nv >= 32 ? 0xffffffffu : ((1u << nv) - 1u)) : 0u;
                // masked views always carry the denominator contraction (a mask rules out
                // the closed form), so only DEN instances compile the mask code
                if constexpr (DEN) {
                if (prm.mbits && prm.trans && (v.rows & 31) == 0) {
                    // rows are the contiguous dimension and a warp's 32 rows are one mask
                    // word per column: lane c loaded the word of column c, and a 32 x 32 bit
                    // transpose hands row b its 32 column bits (warp-uniform: nv and, with
                    // rows a multiple of 32, row_ok are the same for every lane)
                    obs &= warp_transpose_bits(hh ? mw1a : mw0a, lane);
                } else if (prm.mbits && obs) {
                    if (prm.trans) {
                        const int64_t cbase = col0 + 32 * hh;
                        uint32_t m = 0;
                        for (int c = 0; c < nv; ++c)
                            m |= (uint32_t)mask_bit(prm.mbits, (cbase + c) * v.rows + row) << c;
                        obs &= m;
                    } else {
                        // bits idx0 .. idx0 + 31 of the row, idx0 = offset of the half's
                        // first column: one or two words
                        const int sh = (int)((((int64_t)z0 * v.rows + row) * v.c_in + x0 + 32 * hh) & 31);
                        uint64_t m = hh ? mw1a : mw0a;
                        if (sh) m |= (uint64_t)(hh ? mw1b : mw0b) << 32;
                        obs &= (uint32_t)(m >> sh);
                    }
                }
                }
                uint32_t wa2[16], wb2[16];
                float t = 0.f;  // loss terms of the observed entries (FP32 within the half)
                // weights of the 32 entries (and their loss terms); a half whose entries are
                // all observed and in range (every full tile of an unmasked view) sums the
                // loss terms without a per-entry test
                auto weights_half = [&](auto all_tag) {
                    constexpr bool ALL = decltype(all_tag)::value;
#pragma unroll
                    for (int c = 0; c < 32; c += 2) {
                        float a0, b0, a1, b1;
                        tc_weights<WK>(yv[c], __uint_as_float(yh[c]), w, a0, b0);
                        tc_weights<WK>(yv[c + 1], __uint_as_float(yh[c + 1]), w, a1, b1);
                        wa2[c >> 1] = pack_bf16(a0, a1);
                        if (DEN) wb2[c >> 1] = pack_bf16(b0, b1);
                        if (do_loss) {
                            const float d0 = tc_loss<WK>(yv[c], __uint_as_float(yh[c]), a0, b0, prm.L);
                            const float d1 = tc_loss<WK>(yv[c + 1], __uint_as_float(yh[c + 1]), a1, b1, prm.L);
                            if constexpr (ALL) {
                                t += d0 + d1;
                            } else {
                                t += ((obs >> c) & 1u) ? d0 : 0.f;
                                t += ((obs >> (c + 1)) & 1u) ? d1 : 0.f;
                            }
                        }
                    }
                };
                if (do_loss && !DEN && obs == 0xffffffffu)
                    weights_half(std::true_type{});
                else
                    weights_half(std::false_type{});
                if (do_loss) {
                    lsum += (double)t;
                    lcnt += (double)__popc(obs);
                }
                if (obs != 0xffffffffu) {
                    // unobserved, padding or out-of-range entries: clear their BF16 halves
                    // (this also drops the Inf/NaN weights of entries with yhat == 0)
                    uint32_t sh[8];
#pragma unroll
                    for (int k = 0; k < 8; ++k) sh[k] = obs << (7 - k);
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const uint32_t m = pair_mask(sh, q);
                        wa2[q] &= m;
                        if (DEN) wb2[q] &= m;
                    }
                }
                // W row half into TMEM: this warp's lanes, columns 16*hh.. of buffer b
                tmem_st<16>(t_wa + lane_off + b * 32 + 16 * hh, wa2);
                if (DEN) tmem_st<16>(t_wb + lane_off + b * 32 + 16 * hh, wb2);
            }
            if (trl) phase_mark(tr, 22, tp);
            tmem_wait_st();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(wfull(b));
            if (trl) phase_mark(tr, 24, tp);
        }
        if (do_loss) {
            // per-CTA loss partial: warp sums, then the epilogue warps (named barrier 1)
            lsum = warp_sum(lsum);
            lcnt = warp_sum(lcnt);
            double* lred = reinterpret_cast<double*>(sm + LY::kLoss);
            const int ew = warp - kEpiWarp0;
            if (lane == 0) {
                lred[2 * ew] = lsum;
                lred[2 * ew + 1] = lcnt;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(kEpiWarps * 32) : "memory");
            if (ew == 0 && lane == 0) {
                double ts = 0.0, tcn = 0.0;
                for (int k = 0; k < kEpiWarps; ++k) {
                    ts += lred[2 * k];
                    tcn += lred[2 * k + 1];
                }
                prm.loss_part[blockIdx.x] = ts;
                prm.loss_part[gridDim.x + blockIdx.x] = tcn;
            }
        }
        // ---- S readout: group 0 copies S_num, group 1 S_den
        bool have = (T > 0) && mbar_wait(sfull, 0, abort_flag, prm.err, 12, lane == 0 ? tr : nullptr, wlim);
        have = __all_sync(0xffffffffu, have);
        tc_fence_after();
        if (h == 0 || (DEN && h == 1)) {
            const uint32_t tsrc = (h == 0) ? t_snum : t_sden;
            float* dst = ((h == 0) ? prm.s_num : prm.s_den) + (sp * v.rows + row) * BP;
#pragma unroll 1
            for (int c0 = 0; c0 < BP; c0 += 16) {
                uint32_t r[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) r[k] = 0u;
                if (have) {
                    tmem_ld16(tsrc + lane_off + c0, r);
                    tmem_wait_ld();
                }
                if (row_ok) {
#pragma unroll
                    for (int k = 0; k < 16; k += 4)
                        *reinterpret_cast<float4*>(dst + c0 + k) =
                            make_float4(__uint_as_float(r[k]), __uint_as_float(r[k + 1]),
                                        __uint_as_float(r[k + 2]), __uint_as_float(r[k + 3]));
                }
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (tr && tid < kTraceSites) {
        const unsigned long long v = (tid == 0) ? (unsigned long long)(clock64() - t_start) : tr[tid];
        atomicAdd(&prm.trace[tid], v);
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
    if constexpr (CG) {
        // every wait of this item has completed or was drained: the barriers are idle
        if (tid == 0)
            for (int b = 0; b < LY::kNumBars; ++b)
                asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar0 + 8u * b) : "memory");
        __syncthreads();
    }
}

// LOSS: also sum the loss terms into prm.loss_part (a separate instance, so the
// plain pass carries none of that code).
template <int BP, bool DEN, int WK, bool LOSS, int QM, int CFG = 0>
__global__ void __launch_bounds__(kThreads, 1)
k_view_tc(const __grid_constant__ CUtensorMap ymap, const __grid_constant__ CUtensorMap vmap,
          const __grid_constant__ CUtensorMap cmap, const __grid_constant__ Params prm) {
    pdl_wait();
    pdl_trigger();
    const int64_t n_rb = (prm.v.rows + TM - 1) / TM;
    view_tc_body<BP, DEN, WK, LOSS, QM, false, CFG>(&ymap, &vmap, &cmap, prm, blockIdx.x % n_rb,
                                                    blockIdx.x / n_rb);
}

// ---------------------------------------------------------- persistent batched fit
// Spin (bounded) until *flag >= target; false on timeout (raises the error flag
// and the abort flag) or when another CTA aborted.
__device__ __forceinline__ bool wait_stage(const unsigned int* flag, unsigned int target, const PersistDesc& d) {
    const long long t0 = clock64();
    for (;;) {
        unsigned int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
        if (v >= target) return true;
        if (*(volatile int*)d.abort) return false;
        if (clock64() - t0 > d.wait_cycles) {
            atomicCAS(d.err, 0, 20);
            atomicExch(d.abort, 1);
            return false;
        }
        __nanosleep(256);
    }
}

// The update of one (unit, mode) stage by the whole CTA: split reduction of the
// partials (L2-only loads: other SMs wrote them), Eq. 3.4 and the operand copies.
__device__ __forceinline__ void persist_finish(const BatchFinish& f, const UpdateSpec& u) {
    const int64_t n_el = f.rows * f.rank;
    for (int64_t e = threadIdx.x; e < n_el; e += blockDim.x) {
        const int64_t row = e / f.rank, r = e - row * f.rank;
        const int64_t so = row * f.bp + r;
        float num = 0.f, den = 0.f;
        for (int s = 0; s < f.n_split; ++s) {
            num += __ldcg(f.part_num + (int64_t)s * f.s_size + so);
            den += __ldcg(f.part_den + (int64_t)s * f.s_size + so);
        }
        const float v = mu_update(__ldcg(f.theta + e), num, den, u);
        f.theta[e] = v;
        f.canon32[so] = v;
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        f.canon16[so] = *reinterpret_cast<const uint16_t*>(&b);
    }
    // the copies are read by later stages' bulk tensor copies (async proxy) and loads
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __threadfence();
}

template <int BP, int WK>
__global__ void __launch_bounds__(kThreads, 1) k_batched_persistent(const __grid_constant__ PersistDesc d) {
    __shared__ __align__(16) unsigned char prm_sh[(sizeof(Params) + 15) / 16 * 16];
    __shared__ unsigned int item_sh;
    __shared__ int finish_sh;
    const unsigned int total = (unsigned int)d.n_items * (unsigned int)d.n_sweeps;
    for (;;) {
        if (threadIdx.x == 0) item_sh = *(volatile int*)d.abort ? total : atomicAdd(d.queue, 1u);
        __syncthreads();
        const unsigned int q = item_sh;
        if (q >= total) break;
        const int sl = (int)(q / (unsigned int)d.n_items);
        const PersistItem it = d.items[q - (unsigned int)sl * (unsigned int)d.n_items];
        const int s = d.sweep0 + sl;  // the item's sweep
        const int l = it.um / d.n_units, unit = it.um - l * d.n_units;
        // stages of the unit finish in the order (sweep 0, mode 0), (0, 1), (0, 2), (1, 0), ...
        const unsigned int seq = (unsigned int)(s * 3 + l);
        bool go = true;
        if (threadIdx.x == 0 && seq > 0) go = wait_stage(d.stage + unit, seq, d);
        if (threadIdx.x == 0) finish_sh = go ? 1 : 0;
        __syncthreads();
        if (!finish_sh) break;
        asm volatile("fence.proxy.async.global;" ::: "memory");
        const TcUnit* U = d.units + it.um;
        for (int i = threadIdx.x; i < (int)(sizeof(prm_sh) / 16); i += blockDim.x)
            reinterpret_cast<uint4*>(prm_sh)[i] = __ldcg(reinterpret_cast<const uint4*>(U->prm) + i);
        __syncthreads();
        const Params& prm = *reinterpret_cast<const Params*>(prm_sh);
        view_tc_body<BP, true, WK, false, 2, true>(&U->ymap, &U->vmap, &U->cmap, prm, it.rb, it.sp);
        // partials written: count the item; the stage's last item applies the update
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned int cum = (unsigned int)s * (unsigned int)d.sweep_items[unit] +
                                     (unsigned int)d.prefix_items[it.um] + (unsigned int)d.stage_items[it.um];
            const unsigned int old = atomicAdd(d.done + unit, 1u);
            finish_sh = (old + 1u == cum) ? 1 : 0;
            __threadfence();
        }
        __syncthreads();
        if (finish_sh) {
            persist_finish(d.fin[it.um], d.u);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(d.stage + unit), "r"(seq + 1u) : "memory");
            }
        }
        __syncthreads();
    }
}

}  // namespace tc
}  // namespace nef
