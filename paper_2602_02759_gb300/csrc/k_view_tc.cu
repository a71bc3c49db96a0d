// k_view_tc.cu -- host side of the tcgen05 fused pass: support check, TMA tensor
// map for the Y view, weight-kind selection and launch.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "k_view_tc.cuh"
#include "nef_internal.h"

namespace nef {
namespace tc {
cudaError_t launch_bp16(const CUtensorMap&, const Params&, int, int, int, cudaStream_t);
cudaError_t launch_bp32(const CUtensorMap&, const Params&, int, int, int, cudaStream_t);
cudaError_t launch_bp64(const CUtensorMap&, const Params&, int, int, int, cudaStream_t);
}  // namespace tc

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

int weight_kind(const WeightSpec& w) {
    if (w.log_case) return tc::WK_GEN;
    if (w.y_code == POW_ID && w.a_code == POW_RCP && w.b_code == POW_ONE) return tc::WK_KL;
    if (w.y_code == POW_ID && w.a_code == POW_RSQRT3 && w.b_code == POW_RSQRT) return tc::WK_B05;
    if (w.y_code == POW_SQRT && w.a_code == POW_RSQRT && w.b_code == POW_ONE) return tc::WK_HEL;
    return tc::WK_GEN;
}

}  // namespace

bool tc_view_supported(const ViewDesc& v, int) {
    if (v.bond_pad != 16 && v.bond_pad != 32 && v.bond_pad != 64) return false;
    if (v.P.nsrc != 1 || v.Q.nsrc < 1 || v.Q.nsrc > kMaxSrc) return false;
    if (v.P.src[0].ld != v.bond_pad) return false;
    for (int s = 0; s < v.Q.nsrc; ++s)
        if (v.Q.src[s].ld != v.bond_pad) return false;
    const int64_t lim = (int64_t)1 << 31;
    if (v.rows >= lim || v.c_in >= lim || v.c_out >= lim) return false;
    if (v.c_in == 1) {
        if (v.rows % 4 != 0) return false;  // TMA stride of the column dimension: 16-byte multiple
    } else {
        if (v.c_in % 4 != 0) return false;
    }
    return true;
}

cudaError_t launch_view_tc(const float* y, const uint32_t* mbits, const ViewDesc& v, const WeightSpec& w,
                           int need_den, int n_split, float* s_num, float* s_den, int* err_flag,
                           cudaStream_t st, TcLaunchInfo* info) {
    if (!tc_view_supported(v, need_den)) return cudaErrorNotSupported;
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const bool trans = (v.c_in == 1);
    CUresult r;
    if (trans) {
        cuuint64_t dims[2] = {(cuuint64_t)v.rows, (cuuint64_t)v.c_out};
        cuuint64_t strides[1] = {(cuuint64_t)v.rows * 4};
        cuuint32_t box[2] = {(cuuint32_t)tc::TM, (cuuint32_t)tc::TN};
        cuuint32_t es[2] = {1, 1};
        r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(y), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        cuuint64_t dims[3] = {(cuuint64_t)v.c_in, (cuuint64_t)v.rows, (cuuint64_t)v.c_out};
        cuuint64_t strides[2] = {(cuuint64_t)v.c_in * 4, (cuuint64_t)v.c_in * v.rows * 4};
        cuuint32_t box[3] = {32, (cuuint32_t)tc::TM, 1};
        cuuint32_t es[3] = {1, 1, 1};
        r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(y), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    tc::Params p{};
    p.mbits = mbits;
    p.v = v;
    p.w = w;
    p.trans = trans ? 1 : 0;
    p.n_cib = trans ? 1 : (v.c_in + tc::TN - 1) / tc::TN;
    p.n_tiles = trans ? (v.c_out + tc::TN - 1) / tc::TN : v.c_out * p.n_cib;
    p.tiles_per_split = (p.n_tiles + n_split - 1) / n_split;
    p.s_num = s_num;
    p.s_den = s_den;
    p.err = err_flag;
    const int64_t n_rb = (v.rows + tc::TM - 1) / tc::TM;
    const int grid = (int)(n_rb * n_split);
    if (info) {
        info->n_ctas = grid;
        info->smem_bytes = 0;
    }
    const int wk = weight_kind(w);
    switch (v.bond_pad) {
        case 16: return tc::launch_bp16(map, p, need_den, wk, grid, st);
        case 32: return tc::launch_bp32(map, p, need_den, wk, grid, st);
        default: return tc::launch_bp64(map, p, need_den, wk, grid, st);
    }
}

}  // namespace nef
