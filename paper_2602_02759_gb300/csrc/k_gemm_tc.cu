// k_gemm_tc.cu -- BF16 tensor-core GEMM C = A . B^T (FP32 out) on tcgen05, for
// the fold-in encoder's forward and backward products.
//
// A is [M x K] and B is [N x K], both row-major BF16 (K contiguous, "K-major");
// C is [M x N] row-major FP32 (ldc).  One CTA computes a 128 x 128 tile of C
// over one range of the K blocks (split-K: blockIdx.z; with several splits each
// writes its partial tile to a workspace and k_gemm_reduce sums the splits in a
// fixed order, so the result does not depend on scheduling):
//   warp 0 (one elected lane): TMA loads of 128 x 64 tiles of A and B into a
//          4-stage ring (128B swizzle), out-of-range rows/columns read as zero;
//   warp 1 (one elected lane): tcgen05.mma kind::f16, M = 128, N = 128, K = 16
//          steps, accumulator in TMEM (128 columns);
//   all four warps: epilogue, TMEM lane = tile row.  Each warp stages 32 x 32
//          FP32 blocks of its rows in shared memory (128B swizzle, two buffers)
//          and writes them with TMA tensor stores, which clip the edges of C;
//          the accumulate form and row pitches TMA cannot address use guarded
//          per-element stores instead.
//   The producer also prefetches the K block NST ahead into L2, so the ring's
//   loads mostly hit L2.
// The operand layouts and descriptors are those of the fused pass's first
// product (yhat = P . Q^T).  Every mbarrier wait is bounded; a timeout sets the
// error flag and the CTA drains its copies and MMAs before freeing TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "k_view_tc.cuh"
#include "nef_internal.h"
#include "nef_launch.cuh"

namespace nef {
namespace gemm {

using namespace tc;

// tcgen05.mma with both operands from shared-memory descriptors, issued by one
// elected lane of a warp-uniform loop.
__device__ __forceinline__ void tc_mma_ss_e(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_2d_e(const CUtensorMap* map, int x, int y) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];\n\t}" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(x), "r"(y)
        : "memory");
}

// TMA tensor stores from shared memory (bulk-group completion), issued by one thread.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, int x, int y, int z, uint32_t src) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most one group still reading its shared-memory source
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// every group complete (writes performed)
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void st_shared_v4(uint32_t a, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}

constexpr int BM = 128, BK = 64, NST = 4;
constexpr int kThreadsG = 128;
constexpr int kTileBytes = BM * BK * 2;  // 16 KB: the A tile, and each 128-row half of the B tile
constexpr int kEpiBlock = 32 * 32 * 4;   // one staged 32 x 32 FP32 block (4 KB)

// C's store path: guarded per-element stores, TMA stores into C ([M x N], pitch
// ldc), or TMA stores into the split partials ([n_split][M][ldc]).
enum GemmStore { kStoreElem = 0, kStoreTma2d = 1, kStoreTma3d = 2 };

// Shared layout of a CTA computing a 128 x BN tile (BN = 128 or 256).
template <int BN>
struct GemmLayout {
    static constexpr int kStage = kTileBytes * (1 + BN / 128);
    static constexpr int kBar = NST * kStage;            // full[NST], empty[NST], done
    static constexpr int kMisc = kBar + (2 * NST + 1) * 8;
    static constexpr int kEpi = (kMisc + 16 + 1023) / 1024 * 1024;  // 4 warps x 2 staged blocks
    static constexpr int kSmem = kEpi + 4 * 2 * kEpiBlock + 1024;   // + alignment slack
    static_assert(kSmem <= 232448, "shared memory per CTA");
};

template <int BN>
__global__ void __launch_bounds__(kThreadsG, 1)
k_gemm_nt(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
          const __grid_constant__ CUtensorMap cmap, float* __restrict__ C, int M, int N, int K, int ldc,
          int accumulate, int kb_per_split, int store, int* err) {
    pdl_wait();
    pdl_trigger();
    constexpr int kStage = GemmLayout<BN>::kStage;
    constexpr int kBar = GemmLayout<BN>::kBar;
    constexpr int kMisc = GemmLayout<BN>::kMisc;
    constexpr int kEpi = GemmLayout<BN>::kEpi;
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* sm = smem_raw + (base - raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * kb_per_split;
    const int nk = max(0, min((K + BK - 1) / BK - kb0, kb_per_split));  // K blocks of this split
    if (gridDim.z > 1) C += (int64_t)blockIdx.z * M * ldc;                 // this split's partial tile
    const uint32_t bar0 = base + kBar;
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (NST + s); };
    const uint32_t done = bar0 + 8u * (2 * NST);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kMisc);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kMisc + 4);
    if (tid == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    auto uwait = [&](uint32_t bar, uint32_t par, int code) {
        return __all_sync(0xffffffffu, mbar_wait(bar, par, abort_flag, err, code));
    };
    if (warp == 0) {
        // ---- TMA producer (warp-uniform loop, elected issue)
        int issued = 0;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % NST;
            if (!uwait(empty(s), ((kb / NST) & 1) ^ 1, 1)) break;
            mbar_expect_tx_e(full(s), kStage);
            tma_load_2d_e(base + s * kStage, &amap, (kb0 + kb) * BK, m0, full(s));
#pragma unroll
            for (int hb = 0; hb < BN / 128; ++hb)  // B rows n0 + 128 hb .. (consecutive 128-row boxes)
                tma_load_2d_e(base + s * kStage + kTileBytes * (1 + hb), &bmap, (kb0 + kb) * BK, n0 + 128 * hb,
                              full(s));
            if (kb + NST < nk) {  // the block this stage takes next, into L2
                tma_prefetch_2d_e(&amap, (kb0 + kb + NST) * BK, m0);
#pragma unroll
                for (int hb = 0; hb < BN / 128; ++hb) tma_prefetch_2d_e(&bmap, (kb0 + kb + NST) * BK, n0 + 128 * hb);
            }
            issued = kb + 1;
        }
        for (int kb = max(0, issued - NST); kb < issued; ++kb) {
            volatile int dummy = 0;
            mbar_wait(full(kb % NST), (kb / NST) & 1, &dummy, err, 2);
        }
    } else if (warp == 1) {
        // ---- MMA issuer (warp-uniform loop, elected issue)
        constexpr uint32_t idesc = make_idesc(BM, BN, 0, 0);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % NST;
            if (!uwait(full(s), (kb / NST) & 1, 3)) break;
            tc_fence_after();
            const uint64_t ad = make_sdesc(base + s * kStage, 16, 8 * 128, swz_code(128));
            const uint64_t bd = make_sdesc(base + s * kStage + kTileBytes, 16, 8 * 128, swz_code(128));
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)
                tc_mma_ss_e(tmem, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), idesc, (kb > 0 || k > 0) ? 1u : 0u);
            tc_commit_e(empty(s));
        }
        tc_commit_e(done);
    }
    // ---- epilogue: every warp reads its 32 TMEM lanes (rows) of the 128 columns
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, 0, abort_flag, err, 4));
    tc_fence_after();
    const int row = m0 + warp * 32 + lane;
    const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
    if (store != kStoreElem) {
        // staged blocks: row `lane` of a 32 x 32 block at lane * 128 bytes, its 16-byte
        // chunk j at chunk j ^ (lane & 7) (the tensor map's 128B swizzle)
        const uint32_t stage0 = base + kEpi + (uint32_t)warp * 2u * kEpiBlock;
        const bool rows_in = m0 + warp * 32 < M;  // warp-uniform; the store clips rows >= M
        int nb = 0;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + lane_off + c0, r);
            tmem_wait_ld();
            if (!ok || !rows_in || n0 + c0 >= N) break;  // warp-uniform
            if (nk == 0) {
#pragma unroll
                for (int k = 0; k < 32; ++k) r[k] = 0u;
            }
            const uint32_t sb = stage0 + (uint32_t)(nb & 1) * kEpiBlock;
            if (nb >= 2) {  // the store issued from this buffer two blocks ago has read it
                if (lane == 0) bulk_wait_read1();
                __syncwarp();
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
                st_shared_v4(sb + (uint32_t)lane * 128u + ((uint32_t)(j ^ (lane & 7)) << 4), r[4 * j], r[4 * j + 1],
                             r[4 * j + 2], r[4 * j + 3]);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) {
                if (store == kStoreTma3d) tma_store_3d(&cmap, n0 + c0, m0 + warp * 32, (int)blockIdx.z, sb);
                else tma_store_2d(&cmap, n0 + c0, m0 + warp * 32, sb);
                bulk_commit();
            }
            ++nb;
        }
        if (lane == 0) bulk_wait_all();
        __syncwarp();
    }
#pragma unroll 1
    for (int c0 = 0; c0 < BN && store == kStoreElem; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + lane_off + c0, r);
        tmem_wait_ld();
        if (ok && row < M) {
            float* dst = C + (int64_t)row * ldc + n0 + c0;
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                if (n0 + c0 + k < N) {
                    const float v = (nk > 0) ? __uint_as_float(r[k]) : 0.f;
                    dst[k] = (accumulate && gridDim.z == 1) ? dst[k] + v : v;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN) : "memory");
    }
}

// C (=, or += with accumulate) the sum of the splits' partial tiles, in split order.
__global__ void k_gemm_reduce(const float* __restrict__ part, int n_split, int M, int N, int ldc,
                              float* __restrict__ C, int accumulate) {
    pdl_wait();
    pdl_trigger();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * N) return;
    const int64_t r = e / N, c = e - r * N;
    const int64_t off = r * ldc + c, stride = (int64_t)M * ldc;
    float v = 0.f;
    for (int z = 0; z < n_split; ++z) v += part[z * stride + off];
    C[off] = accumulate ? C[off] + v : v;
}

}  // namespace gemm

namespace {
PFN_cuTensorMapEncodeTiled_v12000 gemm_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// Tensor map of a row-major BF16 [rows x K] matrix (row pitch ld elements), box 64 x 128.
bool encode_kmajor(CUtensorMap* map, const uint16_t* p, int64_t rows, int64_t K, int64_t ld) {
    auto enc = gemm_encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)gemm::BK, (cuuint32_t)gemm::BM};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(p), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor map of FP32 C for the TMA-store epilogue: [M x N] with row pitch ldc, or the
// split partials [n_split][M][ldc] (3-d); box 32 x 32 (x 1), 128B swizzle.
bool encode_c(CUtensorMap* map, float* p, int64_t M, int64_t N, int64_t ldc, int n_split) {
    auto enc = gemm_encode_fn();
    if (!enc) return false;
    cuuint64_t dims[3] = {(cuuint64_t)N, (cuuint64_t)M, (cuuint64_t)n_split};
    cuuint64_t strides[2] = {(cuuint64_t)ldc * 4, (cuuint64_t)(M * ldc * 4)};
    cuuint32_t box[3] = {32, 32, 1};
    cuuint32_t es[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, n_split > 1 ? 3 : 2, p, dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

namespace {
// Splits for tiles of width bn: about one wave of CTAs over the SMs, each split
// keeping >= 8 K blocks of 64.
int splits_for(int M, int N, int K, int n_sm, int bn) {
    const int64_t tiles = (int64_t)((M + gemm::BM - 1) / gemm::BM) * ((N + bn - 1) / bn);
    const int nk = (K + gemm::BK - 1) / gemm::BK;
    int64_t s = std::max<int64_t>(1, n_sm / std::max<int64_t>(1, tiles));
    s = std::min<int64_t>(s, std::max(1, nk / 8));
    return (int)std::min<int64_t>(s, 16);
}

int64_t ctas_for(int M, int N, int K, int n_sm, int bn) {
    return (int64_t)((M + gemm::BM - 1) / gemm::BM) * ((N + bn - 1) / bn) * splits_for(M, N, K, n_sm, bn);
}
}  // namespace

// 128 x 256 tiles (half the re-reads of A) where they give at least as many CTAs,
// up to one wave, as 128 x 128 tiles; else 128 x 128 (short products with few
// tiles are latency-bound and want more CTAs).
int gemm_bn(int M, int N, int K, int n_sm) {
    if (N < 256) return 128;
    const int64_t c256 = std::min<int64_t>(ctas_for(M, N, K, n_sm, 256), n_sm);
    const int64_t c128 = std::min<int64_t>(ctas_for(M, N, K, n_sm, 128), n_sm);
    return c256 >= c128 ? 256 : 128;
}

int gemm_splits(int M, int N, int K, int n_sm) { return splits_for(M, N, K, n_sm, gemm_bn(M, N, K, n_sm)); }

cudaError_t launch_gemm_nt(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* C, int64_t ldc,
                           int M, int N, int K, int accumulate, int* err, cudaStream_t st, float* ws,
                           int64_t ws_floats, int n_split) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    // TMA: 16-byte aligned base and row pitch
    if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15) || (lda * 2) % 16 ||
        (ldb * 2) % 16 || K < 0)
        return cudaErrorInvalidValue;
    CUtensorMap am, bm;
    if (!encode_kmajor(&am, A, M, K, lda) || !encode_kmajor(&bm, B, N, K, ldb)) return cudaErrorInvalidValue;
    int n_sm = 152;
    {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n_sm = v;
    }
    const int bn = gemm_bn(M, N, K, n_sm);
    auto kern = bn == 256 ? gemm::k_gemm_nt<256> : gemm::k_gemm_nt<128>;
    const int smem = bn == 256 ? gemm::GemmLayout<256>::kSmem : gemm::GemmLayout<128>::kSmem;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int nk = (K + gemm::BK - 1) / gemm::BK;
    if (n_split < 1 || ws == nullptr || (int64_t)n_split * M * ldc > ws_floats) n_split = 1;
    n_split = std::max(1, std::min(n_split, std::max(1, nk)));
    const int per = (nk + n_split - 1) / n_split;
    n_split = std::max(1, (nk + per - 1) / per);  // no empty split
    dim3 grid((unsigned)((M + gemm::BM - 1) / gemm::BM), (unsigned)((N + bn - 1) / bn), (unsigned)n_split);
    // TMA stores need a 16-byte aligned destination and a row pitch of whole 16-byte units
    float* out = n_split > 1 ? ws : C;
    CUtensorMap cm;
    std::memset(&cm, 0, sizeof(cm));
    int store = gemm::kStoreElem;
    if (!accumulate || n_split > 1) {
        if ((reinterpret_cast<uintptr_t>(out) & 15) == 0 && ldc % 4 == 0 && encode_c(&cm, out, M, N, ldc, n_split))
            store = n_split > 1 ? gemm::kStoreTma3d : gemm::kStoreTma2d;
    }
    launch_pdl(kern, grid, gemm::kThreadsG, smem, st, am, bm, cm, out, M, N, K, (int)ldc, accumulate, std::max(per, 1), store,
                                               err);
    if (n_split > 1) {
        const int64_t n = (int64_t)M * N;
        launch_pdl(gemm::k_gemm_reduce, (unsigned)((n + 255) / 256), 256, 0, st, ws, n_split, M, N, (int)ldc, C, accumulate);
    }
    return cudaGetLastError();
}

}  // namespace nef
