// batched.cpp -- many independent CP factorizations 'ir,jr,kr->ijk', each with
// several random restarts, fitted together by the multiplicative update.
//
// Every (problem, restart) pair is a unit.  The whole fit is one persistent
// launch (k_batched_persistent, one CTA per SM): CTAs take work items -- the
// fused pass of one (row block, column split) of one unit in one mode -- from a
// device queue ordered sweep by sweep and mode by mode; a per-unit stage counter,
// waited on with a bound, keeps Algorithm 1's Gauss-Seidel order within every
// unit, and the CTA that completes a stage's last item applies its update.  The
// launch, its counter resets and the final losses form one CUDA graph.  Items of
// the restarts of one problem are adjacent in the queue, so a Y tile read from
// HBM by one restart is read from L2 by the others.  Y is used in place when its
// innermost dimension is a multiple of 4 (the TMA stride rule); other problems
// are copied once per call into a zero-padded layout (dimensions rounded up to
// multiples of 4, padding unobserved).
#include <algorithm>
#include <chrono>
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

constexpr int64_t kDefaultTiles = 64;  // column tiles per work item unless opt->batch_tiles says

struct Prob {
    int64_t d[3], pd[3];
    int R, bp;
    bool padded;           // Y copied into the zero-padded layout
    int64_t y_off, b_off;  // offsets (elements / words) into the padded / bit buffers
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
    if (opt.batch_tiles < 0 || opt.batch_tiles > 4096) return bfail(NEF_EINVAL, "batch_tiles must be in [0, 4096]");
    const int64_t kTilesPerCta = opt.batch_tiles > 0 ? opt.batch_tiles : kDefaultTiles;
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
        }
        // the views' TMA strides are K and J*K elements: whole 16-byte units iff K % 4 == 0
        q.padded = q.d[2] % 4 != 0;
        for (int m = 0; m < 3; ++m) q.pd[m] = q.padded ? rup(q.d[m], 4) : q.d[m];
        q.R = (int)ranks[p];
        if (q.R < 1 || q.R > 32) return bfail(NEF_EINVAL, "batched ranks must be in [1, 32]");
        q.bp = q.R <= 16 ? 16 : 32;
        if (!Y[p]) return bfail(NEF_EINVAL, "Y[p] is NULL");
        for (int k = 0; k < restarts; ++k)
            for (int m = 0; m < 3; ++m)
                if (!factors[((int64_t)p * restarts + k) * 3 + m]) return bfail(NEF_EINVAL, "factor pointer is NULL");
        const int64_t np = q.pd[0] * q.pd[1] * q.pd[2];
        q.y_off = y_tot;
        if (q.padded) y_tot += rup(np, 64);
        q.b_off = b_tot;
        if (q.padded || masks) b_tot += rup((np + 31) / 32 + 2, 64);
    }
    DevBuf ypad, bits;
    B_CUDA(ypad.alloc((size_t)std::max<int64_t>(y_tot, 1) * 4));
    B_CUDA(bits.alloc((size_t)std::max<int64_t>(b_tot, 1) * 4));
    std::vector<const float*> yv(n);
    std::vector<const uint32_t*> bv(n);
    for (int p = 0; p < n; ++p) {
        const Prob& q = pr[p];
        if (q.padded) {
            B_CUDA(launch_pad_problem(Y[p], masks ? masks[p] : nullptr, q.d, q.pd, ypad.as<float>() + q.y_off,
                                      bits.as<uint32_t>() + q.b_off, st));
            yv[p] = ypad.as<float>() + q.y_off;
            bv[p] = bits.as<uint32_t>() + q.b_off;
        } else {
            yv[p] = Y[p];
            bv[p] = nullptr;
            if (masks) {
                B_CUDA(launch_pack_mask(masks[p], q.d[0] * q.d[1] * q.d[2], bits.as<uint32_t>() + q.b_off, st));
                bv[p] = bits.as<uint32_t>() + q.b_off;
            }
        }
    }

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

    // ---- units (one per (problem, restart) and mode), their finishes and the work items
    std::vector<TcUnit> units((size_t)nu * 3);
    std::vector<BatchFinish> fin((size_t)nu * 3);
    std::vector<int64_t> prefix((size_t)(nu + 1) * 3);
    std::vector<int> stage_items((size_t)nu * 3, 0), prefix_items((size_t)nu * 3, 0), sweep_items((size_t)nu, 0);
    std::vector<PersistItem> items[2];  // one sweep, per bond width 16 / 32, mode-major
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
                for (int s2 = 0; s2 < 2; ++s2) {
                    SrcDesc& d = v.Q.src[s2];
                    d.ptr = c16.as<uint16_t>() + canon_off[(size_t)uu * 3 + other[s2]];
                    d.ld = q.bp;
                    d.nterm = 1;
                    d.div[0] = (s2 == 0) ? q.pd[other[1]] : 1;
                    d.mod[0] = q.pd[other[s2]];
                    d.mul[0] = 1;
                }
                float* sn = pnum.as<float>() + part_off[uu];
                float* sd = pden.as<float>() + part_off[uu];
                if (!tc_make_unit(yv[p], bv[p], v, w, (int)ns, sn, sd, errf.as<int>(), &units[(size_t)l * nu + uu],
                                  &n_rb))
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
                f.rows = q.d[l];
                prefix[(size_t)l * (nu + 1) + uu] = acc;
                acc += q.d[l] * q.R;
                const size_t um = (size_t)l * nu + uu;
                stage_items[um] = n_rb * (int)ns;
                prefix_items[um] = sweep_items[uu];
                sweep_items[uu] += stage_items[um];
            }
            // restarts of one (row block, split) are adjacent: they share Y tiles in L2
            const int g = q.bp == 16 ? 0 : 1;
            for (int rb = 0; rb < n_rb; ++rb)
                for (int sp = 0; sp < ns; ++sp)
                    for (int k = 0; k < restarts; ++k)
                        items[g].push_back({l * nu + p * restarts + k, rb, (int)sp, 0});
        }
        prefix[(size_t)l * (nu + 1) + nu] = acc;
    }
    DevBuf d_units, d_fin, d_prefix, d_items[2], d_tab, d_cnt;
    B_CUDA(d_units.alloc(units.size() * sizeof(TcUnit)));
    B_CUDA(cudaMemcpyAsync(d_units.p, units.data(), units.size() * sizeof(TcUnit), cudaMemcpyHostToDevice, st));
    B_CUDA(d_fin.alloc(fin.size() * sizeof(BatchFinish)));
    B_CUDA(cudaMemcpyAsync(d_fin.p, fin.data(), fin.size() * sizeof(BatchFinish), cudaMemcpyHostToDevice, st));
    B_CUDA(d_prefix.alloc(prefix.size() * sizeof(int64_t)));
    B_CUDA(cudaMemcpyAsync(d_prefix.p, prefix.data(), prefix.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    for (int g = 0; g < 2; ++g)
        if (!items[g].empty()) {
            B_CUDA(d_items[g].alloc(items[g].size() * sizeof(PersistItem)));
            B_CUDA(cudaMemcpyAsync(d_items[g].p, items[g].data(), items[g].size() * sizeof(PersistItem),
                                   cudaMemcpyHostToDevice, st));
        }
    // stage tables: [stage_items | prefix_items | sweep_items]
    std::vector<int> tab;
    tab.insert(tab.end(), stage_items.begin(), stage_items.end());
    tab.insert(tab.end(), prefix_items.begin(), prefix_items.end());
    tab.insert(tab.end(), sweep_items.begin(), sweep_items.end());
    B_CUDA(d_tab.alloc(tab.size() * sizeof(int)));
    B_CUDA(cudaMemcpyAsync(d_tab.p, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    // counters: queue[2], abort, pad, done[nu], stage[nu]
    const size_t n_cnt = 4 + 2 * (size_t)nu;
    B_CUDA(d_cnt.alloc(n_cnt * sizeof(unsigned int)));
    unsigned int* cnt = d_cnt.as<unsigned int>();
    const TcUnit* du = d_units.as<TcUnit>();
    const BatchFinish* df = d_fin.as<BatchFinish>();
    const int64_t* dp = d_prefix.as<int64_t>();

    // ---- canonical copies of the starting factors
    for (int l = 0; l < 3; ++l)
        B_CUDA(launch_mirror_batched(df + (size_t)l * nu, dp + (size_t)l * (nu + 1), nu,
                                     prefix[(size_t)l * (nu + 1) + nu], st));

    // ---- the fit: counter resets and one persistent launch per bond width (per chunk of
    // sweeps when the queue of a whole fit would exceed 2^31 items), captured in one graph
    if (iters > 0) {
        int n_sm = 152;
        {
            int dev = 0, v = 0;
            if (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
                n_sm = v;
            cudaGetLastError();
        }
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
        cudaError_t cap = cudaMemsetAsync(cnt, 0, n_cnt * sizeof(unsigned int), cs);
        for (int g = 0; g < 2 && cap == cudaSuccess; ++g) {
            if (items[g].empty()) continue;
            const int64_t n_it = (int64_t)items[g].size();
            const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(iters, ((int64_t)1 << 31) / n_it));
            for (int s0 = 0; s0 < iters && cap == cudaSuccess; s0 += chunk) {
                if (s0 > 0) cap = cudaMemsetAsync(cnt + g, 0, sizeof(unsigned int), cs);  // queue of this chunk
                PersistDesc d{};
                d.units = du;
                d.fin = df;
                d.items = d_items[g].as<PersistItem>();
                d.stage_items = d_tab.as<int>();
                d.prefix_items = d_tab.as<int>() + 3 * (size_t)nu;
                d.sweep_items = d_tab.as<int>() + 6 * (size_t)nu;
                d.n_items = (int)n_it;
                d.n_sweeps = std::min(chunk, iters - s0);
                d.sweep0 = s0;
                d.n_units = nu;
                d.bp = g == 0 ? 16 : 32;
                d.queue = cnt + g;
                d.abort = reinterpret_cast<int*>(cnt + 2);
                d.done = cnt + 4;
                d.stage = cnt + 4 + nu;
                d.err = errf.as<int>();
                d.u = u;
                d.wait_cycles = opt.wait_cycles > 0 ? (long long)opt.wait_cycles : 4000000000LL;
                if (cap == cudaSuccess) cap = launch_batched_persistent(d, w, n_sm, cs);
            }
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

extern "C" nef_status nef_fit_batched_tune(int n, const int64_t* shapes, const int64_t* ranks,
                                           const float* const* Y, const uint8_t* const* masks,
                                           float* const* factors, int restarts, double alpha, double beta,
                                           const nef_options* opt_in, int* tiles, double* ms) {
    set_last_error("");
    if (n < 1 || !shapes || !ranks || !factors || !tiles) return bfail(NEF_EINVAL, "NULL argument or n < 1");
    if (restarts < 1 || restarts > kMaxRestarts) return bfail(NEF_EINVAL, "restarts must be in [1, 16]");
    nef_options opt;
    if (opt_in) opt = *opt_in;
    else nef_default_options(&opt);
    cudaStream_t st = static_cast<cudaStream_t>(opt.stream);
    // copies of every factor: each candidate fits from the caller's starting point
    const size_t nf = (size_t)n * restarts * 3;
    std::vector<size_t> off(nf + 1, 0);
    for (int p = 0; p < n; ++p)
        for (int k = 0; k < restarts; ++k)
            for (int m = 0; m < 3; ++m) {
                const size_t f = ((size_t)p * restarts + k) * 3 + m;
                off[f + 1] = off[f] + (size_t)rup(shapes[3 * p + m] * ranks[p], 4);
            }
    DevBuf work;
    B_CUDA(work.alloc(off[nf] * sizeof(float)));
    std::vector<float*> copies(nf);
    for (size_t f = 0; f < nf; ++f) copies[f] = work.as<float>() + off[f];
    static const int kCand[5] = {16, 32, 64, 128, 256};
    double best = 1e300;
    int best_t = (int)kDefaultTiles;
    for (int c = 0; c < 5; ++c) {
        for (size_t f = 0; f < nf; ++f) {
            const int p = (int)(f / (3 * (size_t)restarts)), m = (int)(f % 3);
            if (!factors[f]) return bfail(NEF_EINVAL, "factor pointer is NULL");
            B_CUDA(cudaMemcpyAsync(copies[f], factors[f], (size_t)shapes[3 * p + m] * ranks[p] * sizeof(float),
                                   cudaMemcpyDeviceToDevice, st));
        }
        B_CUDA(cudaStreamSynchronize(st));
        opt.batch_tiles = kCand[c];
        const auto t0 = std::chrono::steady_clock::now();
        const nef_status rc = nef_fit_batched(n, shapes, ranks, Y, masks, copies.data(), restarts, alpha, beta, 2,
                                              &opt, nullptr);
        const double t = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (rc != NEF_OK) return rc;
        if (ms) ms[c] = t;
        if (t < best) {
            best = t;
            best_t = kCand[c];
        }
    }
    *tiles = best_t;
    return NEF_OK;
}
