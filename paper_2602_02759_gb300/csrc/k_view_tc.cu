// k_view_tc.cu -- host side of the tcgen05 fused pass: support check, TMA tensor
// map for the Y view, weight-kind selection and launch.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "k_view_tc.cuh"
#include "nef_internal.h"

namespace nef {
namespace tc {
cudaError_t launch_bp16(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp32(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp64(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp16_loss(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp32_loss(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp64_loss(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp16_g(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp32_g(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp64_g(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp16_g_loss(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp32_g_loss(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp64_g_loss(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp16_r1(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                           cudaStream_t);
cudaError_t launch_bp32_r1(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                           cudaStream_t);
cudaError_t launch_bp64_r1(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                           cudaStream_t);
cudaError_t launch_bp16_lik(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp32_lik(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp64_lik(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int, int,
                        cudaStream_t);
cudaError_t launch_bp16_lik_loss(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int,
                                 int, cudaStream_t);
cudaError_t launch_bp32_lik_loss(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int,
                                 int, cudaStream_t);
cudaError_t launch_bp64_lik_loss(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const Params&, int, int,
                                 int, cudaStream_t);
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
    switch (w.lik) {
        case LIK_NEGBIN: return tc::WK_NB;
        case LIK_BINOMIAL: return tc::WK_BIN;
        case LIK_JS: return tc::WK_JS;
        default: break;
    }
    if (w.log_case) return tc::WK_RKL;
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

namespace {

// Kernel parameters and tensor maps of one view pass.
cudaError_t make_params(const float* y, const uint32_t* mbits, const ViewDesc& v, const WeightSpec& w, int n_split,
                        float* s_num, float* s_den, int* err_flag, unsigned long long* trace, CUtensorMap* map,
                        CUtensorMap* vmap, CUtensorMap* cmap, tc::Params* p, int* n_rb_out,
                        bool force_gather = false) {
    auto enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const bool trans = (v.c_in == 1);
    CUresult r;
    if (trans) {
        cuuint64_t dims[2] = {(cuuint64_t)v.rows, (cuuint64_t)v.c_out};
        cuuint64_t strides[1] = {(cuuint64_t)v.rows * 4};
        cuuint32_t box[2] = {(cuuint32_t)tc::TM, (cuuint32_t)tc::TN};
        cuuint32_t es[2] = {1, 1};
        r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(y), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    } else {
        cuuint64_t dims[3] = {(cuuint64_t)v.c_in, (cuuint64_t)v.rows, (cuuint64_t)v.c_out};
        cuuint64_t strides[2] = {(cuuint64_t)v.c_in * 4, (cuuint64_t)v.c_in * v.rows * 4};
        cuuint32_t box[3] = {32, (cuuint32_t)tc::TM, 1};
        cuuint32_t es[3] = {1, 1, 1};
        r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(y), dims, strides, box, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    *p = tc::Params{};
    *vmap = *map;  // unused unless the Q operand is TMA-staged
    *cmap = *map;
    int q_var = -1, q_const = -1;
    if (!force_gather && q_rows_staged(v, tc::TN, &q_var, &q_const)) {
        const SrcDesc& d = v.Q.src[q_var];
        cuuint64_t vd[2] = {(cuuint64_t)d.ld, (cuuint64_t)d.mod[0]};
        cuuint64_t vs[1] = {(cuuint64_t)d.ld * 2};
        cuuint32_t vb[2] = {(cuuint32_t)v.bond_pad, (cuuint32_t)tc::TN};
        cuuint32_t ves[2] = {1, 1};
        const CUtensorMapSwizzle sw = v.bond_pad == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                      : (v.bond_pad == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
        r = enc(vmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(d.ptr), vd, vs, vb, ves,
                CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        if (q_const >= 0) {
            const SrcDesc& c = v.Q.src[q_const];
            cuuint64_t cd[2] = {(cuuint64_t)c.ld, (cuuint64_t)c.mod[0]};
            cuuint64_t cstr[1] = {(cuuint64_t)c.ld * 2};
            cuuint32_t cb[2] = {(cuuint32_t)v.bond_pad, 1};
            r = enc(cmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(c.ptr), cd, cstr, cb, ves,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        }
        p->qmode = 1;
        p->q_var = q_var;
        p->q_const = q_const;
    }
    p->mbits = mbits;
    p->v = v;
    p->w = w;
    p->trans = trans ? 1 : 0;
    p->n_cib = trans ? 1 : (v.c_in + tc::TN - 1) / tc::TN;
    p->n_tiles = trans ? (v.c_out + tc::TN - 1) / tc::TN : v.c_out * p->n_cib;
    p->tiles_per_split = (p->n_tiles + n_split - 1) / n_split;
    p->s_num = s_num;
    p->s_den = s_den;
    p->err = err_flag;
    p->trace = trace;
    p->loss_part = nullptr;
    p->L = LossSpec{};
    p->wait_cycles = tc::kWaitCycles;
    *n_rb_out = (int)((v.rows + tc::TM - 1) / tc::TM);
    return cudaSuccess;
}

}  // namespace

cudaError_t launch_view_tc(const float* y, const uint32_t* mbits, const ViewDesc& v, const WeightSpec& w,
                           int need_den, int n_split, float* s_num, float* s_den, int* err_flag,
                           cudaStream_t st, TcLaunchInfo* info, unsigned long long* trace, const LossSpec* loss,
                           double* loss_part, long long wait_cycles, const TcTileConfig* cfg) {
    if (!tc_view_supported(v, need_den)) return cudaErrorNotSupported;
    if (mbits && !need_den) return cudaErrorInvalidValue;  // mask code lives in the DEN instances only
    CUtensorMap map, vmap, cmap;
    tc::Params p;
    int n_rb = 0;
    cudaError_t e = make_params(y, mbits, v, w, n_split, s_num, s_den, err_flag, trace, &map, &vmap, &cmap, &p,
                                &n_rb, cfg && cfg->gather);
    if (e != cudaSuccess) return e;
    if (loss) {
        p.loss_part = loss_part;
        p.L = *loss;
    }
    if (wait_cycles > 0) p.wait_cycles = wait_cycles;
    const int grid = n_rb * n_split;
    if (info) {
        info->n_ctas = grid;
        info->smem_bytes = 0;
        info->staged = p.qmode ? 1 : 0;
    }
    const int wk = weight_kind(w);
    using LaunchFn = cudaError_t (*)(const CUtensorMap&, const CUtensorMap&, const CUtensorMap&, const tc::Params&,
                                     int, int, int, cudaStream_t);
    // [loss][staged rows][bond 16/32/64]
    static const LaunchFn table[2][2][3] = {
        {{tc::launch_bp16_g, tc::launch_bp32_g, tc::launch_bp64_g}, {tc::launch_bp16, tc::launch_bp32, tc::launch_bp64}},
        {{tc::launch_bp16_g_loss, tc::launch_bp32_g_loss, tc::launch_bp64_g_loss},
         {tc::launch_bp16_loss, tc::launch_bp32_loss, tc::launch_bp64_loss}}};
    // reverse KL and the likelihood families have their own instances for staged Q
    // rows; with gathered rows they run through the generic weight kind
    static const LaunchFn lik_table[2][3] = {
        {tc::launch_bp16_lik, tc::launch_bp32_lik, tc::launch_bp64_lik},
        {tc::launch_bp16_lik_loss, tc::launch_bp32_lik_loss, tc::launch_bp64_lik_loss}};
    const int bi = v.bond_pad == 16 ? 0 : (v.bond_pad == 32 ? 1 : 2);
    if (info) info->ring = 0;
    if (cfg && cfg->ring == 1 && p.qmode && !p.loss_part && wk < tc::WK_NB) {
        // the alternative ring depths exist for the staged instances of the sweep's passes
        static const LaunchFn r1[3] = {tc::launch_bp16_r1, tc::launch_bp32_r1, tc::launch_bp64_r1};
        if (info) info->ring = 1;
        return r1[bi](map, vmap, cmap, p, need_den, wk, grid, st);
    }
    if (wk >= tc::WK_NB && p.qmode)
        return lik_table[p.loss_part ? 1 : 0][bi](map, vmap, cmap, p, need_den, wk, grid, st);
    return table[p.loss_part ? 1 : 0][p.qmode ? 1 : 0][bi](map, vmap, cmap, p, need_den, wk >= tc::WK_NB ? tc::WK_GEN : wk,
                                                          grid, st);
}

static_assert(sizeof(tc::Params) <= sizeof(TcUnit::prm), "TcUnit parameter area too small");
static_assert(tc::TN == kTcTileN, "planner and kernel disagree on the tile width");

bool tc_make_unit(const float* y, const uint32_t* mbits, const ViewDesc& v, const WeightSpec& w, int n_split,
                  float* s_num, float* s_den, int* err_flag, TcUnit* unit, int* n_rb) {
    if (!tc_view_supported(v, 1)) return false;
    tc::Params p;
    if (make_params(y, mbits, v, w, n_split, s_num, s_den, err_flag, nullptr, &unit->ymap, &unit->vmap, &unit->cmap, &p,
                    n_rb) != cudaSuccess)
        return false;
    memset(unit->prm, 0, sizeof(unit->prm));
    memcpy(unit->prm, &p, sizeof(p));
    return true;
}


}  // namespace nef
