// batched.cpp -- many independent CP factorizations 'ir,jr,kr->ijk', each with
// several random restarts, fitted together by the multiplicative update.
//
// Every (problem, restart) pair is a unit.  Y is copied once per call into a
// zero-padded layout (dimensions rounded up to multiples of 4, padding
// unobserved) so that every unit's views satisfy the TMA stride rule.  A sweep
// is three mode phases (Gauss-Seidel order of Algorithm 1 within every unit);
// each phase is one batched tensor-core launch per bond width plus one batched
// finish.  The whole iteration loop is captured in a CUDA graph and launched
// once.  Restarts of a problem read the same Y tiles: their work items are
// adjacent, so a tile is read from HBM once and from L2 by the other restarts.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/nef.h"
#include "nef_batched.h"
#include "nef_internal.h"

using namespace nef;

namespace {

struct DevBuf {
    void* p = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
    cudaError_t alloc(size_t n) { return cudaMalloc(&p, n ? n : 16); }
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};

nef_status bfail(nef_status s, const char* msg) {
    set_last_error(msg);
    return s;
}

#define B_CUDA(call)                                                     \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) {                                         \
            cudaGetLastError();                                          \
            return bfail(NEF_ECUDA, cudaGetErrorString(e_));             \
        }                                                                \
    } while (0)

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

#ifndef NEF_BATCH_TILES
#define NEF_BATCH_TILES 64
#endif
constexpr int64_t kTilesPerCta = NEF_BATCH_TILES;  // column tiles per CTA of one unit

struct Prob {
    int64_t d[3], pd[3];
    int R, bp;
    int64_t y_off, b_off;  // offsets (elements / words) into the padded buffers
};

}  // namespace

extern "C" nef_status nef_fit_batched(int n, const int64_t* shapes, const int64_t* ranks, const float* const* Y,
                                      const uint8_t* const* masks, float* const* factors, int restarts,
                                      double alpha, double beta, int iters, const nef_options* opt_in,
                                      double* losses) {
    set_last_error("");
    if (n < 1 || !shapes || !ranks || !Y || !factors) return bfail(NEF_EINVAL, "NULL argument or n < 1");
    if (restarts < 1 || restarts > kMaxRestarts) return bfail(NEF_EINVAL, "restarts must be in [1, 16]");
    if (iters < 0) return bfail(NEF_EINVAL, "iters must be >= 0");
    if (alpha == 0.0 && beta != 1.0)
        return bfail(NEF_EUNSUPPORTED, "alpha == 0 with beta != 1 has no decomposition (App. B)");
    nef_options opt;
    if (opt_in) opt = *opt_in;
    else nef_default_options(&opt);
    if (opt.precision != NEF_BF16)
        return bfail(NEF_EUNSUPPORTED, "the batched engine runs on the tensor cores: use NEF_BF16");
    cudaStream_t st = static_cast<cudaStream_t>(opt.stream);
    const WeightSpec w = weight_spec(alpha, beta);
    const UpdateSpec u = update_spec(alpha, beta, opt.eps);
    const LossSpec L = loss_spec(alpha, beta);

    // ---- problems and padded layouts
    std::vector<Prob> pr(n);
    int64_t y_tot = 0, b_tot = 0;
    for (int p = 0; p < n; ++p) {
        Prob& q = pr[p];
        for (int m = 0; m < 3; ++m) {
            q.d[m] = shapes[3 * p + m];
            if (q.d[m] < 1) return bfail(NEF_EINVAL, "dimensions must be >= 1");
            q.pd[m] = rup(q.d[m], 4);
        }
        q.R = (int)ranks[p];
        if (q.R < 1 || q.R > 32) return bfail(NEF_EINVAL, "batched ranks must be in [1, 32]");
        q.bp = q.R <= 16 ? 16 : 32;
        if (!Y[p]) return bfail(NEF_EINVAL, "Y[p] is NULL");
        for (int k = 0; k < restarts; ++k)
            for (int m = 0; m < 3; ++m)
                if (!factors[((int64_t)p * restarts + k) * 3 + m]) return bfail(NEF_EINVAL, "factor pointer is NULL");
        const int64_t np = q.pd[0] * q.pd[1] * q.pd[2];
        q.y_off = y_tot;
        y_tot += rup(np, 64);
        q.b_off = b_tot;
        b_tot += rup((np + 31) / 32 + 2, 64);
    }
    DevBuf ypad, bits;
    B_CUDA(ypad.alloc((size_t)y_tot * 4));
    B_CUDA(bits.alloc((size_t)b_tot * 4));
    for (int p = 0; p < n; ++p)
        B_CUDA(launch_pad_problem(Y[p], masks ? masks[p] : nullptr, pr[p].d, pr[p].pd,
                                  ypad.as<float>() + pr[p].y_off, bits.as<uint32_t>() + pr[p].b_off, st));

    // ---- units: canonical factor copies and partial buffers
    const int nu = n * restarts;
    std::vector<int64_t> canon_off((size_t)nu * 3);
    int64_t canon_tot = 0;
    for (int p = 0; p < n; ++p)
        for (int k = 0; k < restarts; ++k)
            for (int m = 0; m < 3; ++m) {
                canon_off[((size_t)p * restarts + k) * 3 + m] = canon_tot;
                canon_tot += rup(pr[p].pd[m] * pr[p].bp, 64);
            }
    DevBuf c32, c16;
    B_CUDA(c32.alloc((size_t)canon_tot * 4));
    B_CUDA(c16.alloc((size_t)canon_tot * 2));
    B_CUDA(cudaMemsetAsync(c32.p, 0, (size_t)canon_tot * 4, st));
    B_CUDA(cudaMemsetAsync(c16.p, 0, (size_t)canon_tot * 2, st));
    // column tiles of the view of mode l (64 columns per tile)
    auto view_of = [&](int p, int l, ViewDesc& v) {
        const Prob& q = pr[p];
        const int64_t I = q.pd[0], J = q.pd[1], K = q.pd[2];
        v = ViewDesc{};
        v.rows = q.pd[l];
        v.c_out = (l == 0) ? 1 : (l == 1 ? I : I * J);
        v.c_in = (l == 0) ? J * K : (l == 1 ? K : 1);
        v.bond = q.R;
        v.bond_pad = q.bp;
    };
    auto n_tiles_of = [&](const ViewDesc& v) {
        return v.c_in == 1 ? (v.c_out + 63) / 64 : v.c_out * ((v.c_in + 63) / 64);
    };
    std::vector<int64_t> part_off(nu), part_sz(nu, 0);
    int64_t part_tot = 0;
    for (int p = 0; p < n; ++p)
        for (int l = 0; l < 3; ++l) {
            ViewDesc v;
            view_of(p, l, v);
            const int64_t ns = std::max<int64_t>(1, (n_tiles_of(v) + kTilesPerCta - 1) / kTilesPerCta);
            for (int k = 0; k < restarts; ++k) {
                const int uu = p * restarts + k;
                part_sz[uu] = std::max(part_sz[uu], ns * v.rows * pr[p].bp);
            }
        }
    for (int uu = 0; uu < nu; ++uu) {
        part_off[uu] = part_tot;
        part_tot += rup(part_sz[uu], 64);
    }
    DevBuf pnum, pden, errf;
    B_CUDA(pnum.alloc((size_t)part_tot * 4));
    B_CUDA(pden.alloc((size_t)part_tot * 4));
    B_CUDA(errf.alloc(sizeof(int)));
    B_CUDA(cudaMemsetAsync(errf.p, 0, sizeof(int), st));

    // ---- per-mode launch descriptors
    std::vector<TcUnit> units((size_t)nu * 3);
    std::vector<TcWork> work[3][2];  // [mode][bond width 16/32]
    std::vector<BatchFinish> fin((size_t)nu * 3);
    std::vector<int64_t> prefix((size_t)(nu + 1) * 3);
    for (int l = 0; l < 3; ++l) {
        int64_t acc = 0;
        for (int p = 0; p < n; ++p) {
            const Prob& q = pr[p];
            ViewDesc v0;
            view_of(p, l, v0);
            const int64_t ns = std::max<int64_t>(1, (n_tiles_of(v0) + kTilesPerCta - 1) / kTilesPerCta);
            int other[2], oc = 0;
            for (int m = 0; m < 3; ++m)
                if (m != l) other[oc++] = m;
            int n_rb = 1;
            for (int k = 0; k < restarts; ++k) {
                const int uu = p * restarts + k;
                ViewDesc v = v0;
                v.P.nsrc = 1;
                SrcDesc& ps = v.P.src[0];
                ps.ptr = c16.as<uint16_t>() + canon_off[(size_t)uu * 3 + l];
                ps.ld = q.bp;
                ps.nterm = 1;
                ps.div[0] = 1;
                ps.mod[0] = q.pd[l];
                ps.mul[0] = 1;
                v.Q.nsrc = 2;
                for (int s = 0; s < 2; ++s) {
                    SrcDesc& d = v.Q.src[s];
                    d.ptr = c16.as<uint16_t>() + canon_off[(size_t)uu * 3 + other[s]];
                    d.ld = q.bp;
                    d.nterm = 1;
                    d.div[0] = (s == 0) ? q.pd[other[1]] : 1;
                    d.mod[0] = q.pd[other[s]];
                    d.mul[0] = 1;
                }
                float* sn = pnum.as<float>() + part_off[uu];
                float* sd = pden.as<float>() + part_off[uu];
                if (!tc_make_unit(ypad.as<float>() + q.y_off, bits.as<uint32_t>() + q.b_off, v, w, (int)ns, sn, sd,
                                  errf.as<int>(), &units[(size_t)l * nu + uu], &n_rb))
                    return bfail(NEF_EUNSUPPORTED, "a batched view cannot run on the tensor cores");
                BatchFinish& f = fin[(size_t)l * nu + uu];
                f.theta = factors[(size_t)uu * 3 + l];
                f.canon32 = c32.as<float>() + canon_off[(size_t)uu * 3 + l];
                f.canon16 = c16.as<uint16_t>() + canon_off[(size_t)uu * 3 + l];
                f.part_num = sn;
                f.part_den = sd;
                f.rank = q.R;
                f.bp = q.bp;
                f.s_size = v.rows * q.bp;
                f.n_split = (int)ns;
                prefix[(size_t)l * (nu + 1) + uu] = acc;
                acc += q.d[l] * q.R;
            }
            // restarts of one (row block, split) are adjacent: they share Y tiles in L2
            const int g = q.bp == 16 ? 0 : 1;
            for (int rb = 0; rb < n_rb; ++rb)
                for (int sp = 0; sp < ns; ++sp)
                    for (int k = 0; k < restarts; ++k) work[l][g].push_back({p * restarts + k, rb, (int)sp, 0});
        }
        prefix[(size_t)l * (nu + 1) + nu] = acc;
    }
    DevBuf d_units, d_fin, d_prefix, d_work[3][2];
    B_CUDA(d_units.alloc(units.size() * sizeof(TcUnit)));
    B_CUDA(cudaMemcpyAsync(d_units.p, units.data(), units.size() * sizeof(TcUnit), cudaMemcpyHostToDevice, st));
    B_CUDA(d_fin.alloc(fin.size() * sizeof(BatchFinish)));
    B_CUDA(cudaMemcpyAsync(d_fin.p, fin.data(), fin.size() * sizeof(BatchFinish), cudaMemcpyHostToDevice, st));
    B_CUDA(d_prefix.alloc(prefix.size() * sizeof(int64_t)));
    B_CUDA(cudaMemcpyAsync(d_prefix.p, prefix.data(), prefix.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    for (int l = 0; l < 3; ++l)
        for (int g = 0; g < 2; ++g)
            if (!work[l][g].empty()) {
                B_CUDA(d_work[l][g].alloc(work[l][g].size() * sizeof(TcWork)));
                B_CUDA(cudaMemcpyAsync(d_work[l][g].p, work[l][g].data(), work[l][g].size() * sizeof(TcWork),
                                       cudaMemcpyHostToDevice, st));
            }
    const TcUnit* du = d_units.as<TcUnit>();
    const BatchFinish* df = d_fin.as<BatchFinish>();
    const int64_t* dp = d_prefix.as<int64_t>();

    // ---- canonical copies of the starting factors
    for (int l = 0; l < 3; ++l)
        B_CUDA(launch_mirror_batched(df + (size_t)l * nu, dp + (size_t)l * (nu + 1), nu,
                                     prefix[(size_t)l * (nu + 1) + nu], st));

    // ---- the sweep loop, captured in one graph
    if (iters > 0) {
        // the caller's stream may be the legacy stream, which cannot be captured: capture
        // and launch on a private stream that starts after the work queued so far
        cudaStream_t cs = nullptr;
        B_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        struct StreamGuard {
            cudaStream_t s;
            ~StreamGuard() { cudaStreamDestroy(s); }
        } guard{cs};
        B_CUDA(cudaStreamSynchronize(st));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        B_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
        cudaError_t cap = cudaSuccess;
        for (int it = 0; it < iters && cap == cudaSuccess; ++it)
            for (int l = 0; l < 3 && cap == cudaSuccess; ++l) {
                for (int g = 0; g < 2 && cap == cudaSuccess; ++g)
                    if (!work[l][g].empty())
                        cap = launch_view_tc_batched(du + (size_t)l * nu, d_work[l][g].as<TcWork>(),
                                                     (int)work[l][g].size(), 16 << g, 1, w, cs);
                if (cap == cudaSuccess)
                    cap = launch_finish_batched(df + (size_t)l * nu, dp + (size_t)l * (nu + 1), nu,
                                                prefix[(size_t)l * (nu + 1) + nu], u, cs);
            }
        cudaError_t end = cudaStreamEndCapture(cs, &graph);
        if (cap != cudaSuccess || end != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return bfail(NEF_ECUDA, cudaGetErrorString(cap != cudaSuccess ? cap : end));
        }
        cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, cs);
        if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
        if (exec) cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return bfail(NEF_ECUDA, cudaGetErrorString(e));
    }

    // ---- losses of every restart
    if (losses) {
        DevBuf lpart, lout;
        const int nb = 152 * 4;
        B_CUDA(lpart.alloc((size_t)nb * restarts * sizeof(double)));
        B_CUDA(lout.alloc((size_t)nu * sizeof(double)));
        for (int p = 0; p < n; ++p) {
            BatchFactors bf{};
            for (int k = 0; k < restarts; ++k)
                for (int m = 0; m < 3; ++m) bf.f[k][m] = factors[((size_t)p * restarts + k) * 3 + m];
            B_CUDA(launch_loss_batched(Y[p], masks ? masks[p] : nullptr, pr[p].d, pr[p].R, restarts, bf, L,
                                       lpart.as<double>(), nb, lout.as<double>() + (size_t)p * restarts, st));
        }
        B_CUDA(cudaMemcpyAsync(losses, lout.p, (size_t)nu * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    int herr = 0;
    B_CUDA(cudaMemcpyAsync(&herr, errf.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    B_CUDA(cudaStreamSynchronize(st));
    if (herr) return bfail(NEF_ETIMEOUT, "a bounded wait in the batched tensor-core pass gave up");
    return NEF_OK;
}
