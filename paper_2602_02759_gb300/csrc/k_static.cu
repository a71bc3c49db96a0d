// k_static.cu -- a factor update for 3-way CP models that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a framework's
// caching allocator owns all device memory, real-time loops that forbid any
// allocation after start-up, or plugins whose host application reserves the
// whole device.  nef_cp3_update_static serves them: it runs the CUDA-core fused
// pass (the same kernel as NEF_FP32 plans), the split reduction and the update
// of Eq. 3.4, with every intermediate in one file-scope device array of fixed
// size instead of a plan workspace.
//
// The array belongs to the library: every GPU that loads it keeps the array
// until the process exits.  All calls share it, so calls that may overlap on
// the GPU (different streams, or different host threads) race on it and must be
// serialised by the caller.  Each call overwrites every element it later reads,
// so no clearing is needed between calls.
#include <algorithm>
#include <cmath>

#include "../../include/nef.h"
#include "nef_internal.h"

namespace {

// 16 MiB of scratch: per-split partial numerators and denominators plus the
// reduced numerator and denominator of the updated factor.
constexpr int64_t kStaticScratchFloats = (int64_t)4 << 20;
static __device__ __align__(256) float g_nef_static_scratch[kStaticScratchFloats];

// Device address of the scratch array on the current device.  In host code the
// array's name only stands for the host-side shadow symbol, so the address is
// looked up with the device current, on every call: after a device reset the
// module is loaded again and the array may move, so no address is kept.
cudaError_t scratch_on_current_device(float** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_nef_static_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<float*>(p);
    return cudaSuccess;
}

nef_status static_fail(nef_status s, const char* msg) {
    nef::set_last_error(msg);
    return s;
}

}  // namespace

extern "C" nef_status nef_cp3_update_static(const float* Y, const int64_t* shape, int rank,
                                            float* const* factors, int l, double alpha, double beta,
                                            double eps, void* stream) {
    using namespace nef;
    set_last_error("");
    if (!Y || !shape || !factors || !factors[0] || !factors[1] || !factors[2])
        return static_fail(NEF_EINVAL, "NULL argument");
    if (l < 0 || l > 2) return static_fail(NEF_EINVAL, "factor index must be 0, 1 or 2");
    if (rank != 16 && rank != 32 && rank != 64) return static_fail(NEF_EINVAL, "rank must be 16, 32 or 64");
    if (!(eps >= 0.0) || !std::isfinite(eps)) return static_fail(NEF_EINVAL, "eps must be finite and >= 0");
    {
        bool unsupported = false;
        const char* msg = loss_args_error(LIK_NONE, alpha, beta, 0.0, &unsupported);
        if (msg) return static_fail(unsupported ? NEF_EUNSUPPORTED : NEF_EINVAL, msg);
    }
    const int64_t I = shape[0], J = shape[1], K = shape[2];
    if (I < 1 || J < 1 || K < 1) return static_fail(NEF_EINVAL, "dimensions must be >= 1");
    const int64_t dims[3] = {I, J, K};
    const int64_t rows = dims[l];
    const int64_t n_el = rows * rank;
    // one split needs its partials (num, den) plus the reduced num and den
    if (4 * n_el > kStaticScratchFloats)
        return static_fail(NEF_EINVAL,
                           "factor too large for the static scratch (rows x rank must be <= 1048576)");

    ViewDesc v{};
    v.rows = rows;
    v.bond = rank;
    v.bond_pad = rank;
    v.P.nsrc = 1;
    v.P.src[0].ptr = factors[l];
    v.P.src[0].ld = rank;
    v.P.src[0].nterm = 1;
    v.P.src[0].div[0] = 1;
    v.P.src[0].mod[0] = rows;
    v.P.src[0].mul[0] = 1;
    // columns are the two other modes, in Y's order; each gathers its factor's row
    int other[2], k = 0;
    for (int m = 0; m < 3; ++m)
        if (m != l) other[k++] = m;
    const int64_t inner = dims[other[1]];
    v.c_out = (l == 0) ? 1 : (l == 1 ? I : I * J);
    v.c_in = (l == 0) ? J * K : (l == 1 ? K : 1);
    v.Q.nsrc = 2;
    for (int s = 0; s < 2; ++s) {
        SrcDesc& d = v.Q.src[s];
        d.ptr = factors[other[s]];
        d.ld = rank;
        d.nterm = 1;
        d.div[0] = (s == 0) ? inner : 1;
        d.mod[0] = dims[other[s]];
        d.mul[0] = 1;
    }

    float* scratch = nullptr;
    cudaError_t e = scratch_on_current_device(&scratch);
    if (e != cudaSuccess) return static_fail(NEF_ECUDA, cudaGetErrorString(e));
    // four CTAs of the CUDA-core pass per SM of the current device
    int dev = 0, n_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return static_fail(NEF_ECUDA, cudaGetErrorString(e));
    const int64_t ncols = v.c_out * v.c_in;
    const int64_t n_rb = (rows + 63) / 64;
    const int64_t tiles = (ncols + 63) / 64;
    int64_t n_split = std::max<int64_t>(1, (int64_t)4 * std::max(1, n_sm) / n_rb);
    n_split = std::min<int64_t>(n_split, tiles);
    n_split = std::min<int64_t>(n_split, (kStaticScratchFloats / n_el - 2) / 2);
    n_split = std::max<int64_t>(n_split, 1);
    float* part_num = scratch;
    float* part_den = part_num + n_split * n_el;
    float* num = part_den + n_split * n_el;
    float* den = num + n_el;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const WeightSpec w = weight_spec(alpha, beta);
    const UpdateSpec u = update_spec(alpha, beta, eps);
    int n_ctas = 0;
    if ((e = launch_view_simt<float>(Y, nullptr, v, w, 1, (int)n_split, part_num, part_den, nullptr,
                                     nullptr, st, &n_ctas)) != cudaSuccess ||
        (e = launch_reduce_splits<float>(part_num, (int)n_split, n_el, num, st)) != cudaSuccess ||
        (e = launch_reduce_splits<float>(part_den, (int)n_split, n_el, den, st)) != cudaSuccess ||
        (e = launch_update<float>(factors[l], num, den, n_el, u, st)) != cudaSuccess)
        return static_fail(NEF_ECUDA, cudaGetErrorString(e));
    return NEF_OK;
}
