// plan.cpp -- einsum contraction planner, workspace, sweep driver and C ABI.
//
// Parsing follows the model-string grammar of Eq. 2.2; swap(model_str, l) of
// Eq. 3.8 is represented by the per-factor pass plan below.  For every factor
// l the planner looks for a "view" of Y (rows = a contiguous run of observed
// letters holding l's observed letters, columns = the other observed letters)
// through which the reconstruction factorises over a small set of latent bond
// letters (Eq. 2.1):  yhat[row, col] = sum_b P[row, b] Q[col, b].
// The numerator/denominator of Eq. 3.6-3.8 then become
//     S[row, b] = sum_col W[row, col] Q[col, b]            (fused pass kernel)
//     num_l = einsum(S, the other row-side factors -> l)   (small epilogue)
// If no view exists (a factor straddles rows and columns, e.g. the many-body
// model), the pass falls back to Algorithm 1 as written: materialise yhat,
// a(Y,Yhat), b(Y,Yhat) and contract with einstr_l.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <vector>

#include "../../include/nef.h"
#include "nef_internal.h"

using namespace nef;

namespace {

thread_local std::string g_err;

nef_status fail(nef_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define NEF_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(NEF_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                \
    } while (0)

// ------------------------------------------------------------------ model
struct Model {
    int M = 0, K = 0, L = 0;                 // observed, latent letters; factors
    std::vector<char> letter;                 // id -> char
    std::vector<int64_t> dim;                 // id -> size
    std::vector<std::vector<int>> term;       // factor -> letter ids in term order
    int64_t N = 1;                            // entries of Y
    bool is_obs(int x) const { return x < M; }
    int64_t fac_size(int f) const {
        int64_t n = 1;
        for (int x : term[f]) n *= dim[x];
        return n;
    }
    bool fac_has(int f, int x) const {
        return std::find(term[f].begin(), term[f].end(), x) != term[f].end();
    }
    int64_t fac_stride(int f, int x) const {  // stride of letter x in factor f (0 if absent)
        int64_t s = 1;
        for (int p = (int)term[f].size() - 1; p >= 0; --p) {
            if (term[f][p] == x) return s;
            s *= dim[term[f][p]];
        }
        return 0;
    }
    int64_t y_stride(int x) const {
        if (x >= M) return 0;
        int64_t s = 1;
        for (int m = M - 1; m > x; --m) s *= dim[m];
        return s;
    }
};

nef_status parse_model(const char* str, const int64_t* shapes, int n_obs, const int64_t* ranks,
                       int n_lat, Model& md) {
    if (!str) return fail(NEF_EINVAL, "model string is NULL");
    std::string s;
    for (const char* p = str; *p; ++p)
        if (*p != ' ') s.push_back(*p);
    size_t arrow = s.find("->");
    if (arrow == std::string::npos || s.find("->", arrow + 2) != std::string::npos)
        return fail(NEF_EPARSE, "model string needs exactly one '->'");
    std::string lhs = s.substr(0, arrow), rhs = s.substr(arrow + 2);
    std::vector<std::string> terms;
    size_t start = 0;
    while (true) {
        size_t c = lhs.find(',', start);
        terms.push_back(lhs.substr(start, c == std::string::npos ? std::string::npos : c - start));
        if (c == std::string::npos) break;
        start = c + 1;
    }
    auto ok_letter = [](char ch) { return ch >= 'a' && ch <= 'z'; };
    int id_of[128];
    for (int& v : id_of) v = -1;
    for (char ch : rhs) {
        if (!ok_letter(ch)) return fail(NEF_EPARSE, "bad output letter '%c'", ch);
        if (id_of[(int)ch] >= 0) return fail(NEF_EPARSE, "repeated output letter '%c'", ch);
        id_of[(int)ch] = (int)md.letter.size();
        md.letter.push_back(ch);
    }
    md.M = (int)md.letter.size();
    if (md.M == 0) return fail(NEF_EPARSE, "no observed letters");
    if ((int)terms.size() > kMaxFac) return fail(NEF_EPARSE, "too many factors (max %d)", kMaxFac);
    for (auto& t : terms) {
        std::vector<int> ids;
        for (char ch : t) {
            if (!ok_letter(ch)) return fail(NEF_EPARSE, "bad letter '%c' in term '%s'", ch, t.c_str());
            if (id_of[(int)ch] < 0) {
                id_of[(int)ch] = (int)md.letter.size();
                md.letter.push_back(ch);
            }
            int id = id_of[(int)ch];
            if (std::find(ids.begin(), ids.end(), id) != ids.end())
                return fail(NEF_EPARSE, "repeated letter '%c' in term '%s'", ch, t.c_str());
            ids.push_back(id);
        }
        md.term.push_back(ids);
    }
    md.L = (int)md.term.size();
    md.K = (int)md.letter.size() - md.M;
    if ((int)md.letter.size() > kMaxLet) return fail(NEF_EPARSE, "too many letters");
    for (int m = 0; m < md.M; ++m) {
        bool seen = false;
        for (auto& t : md.term)
            if (std::find(t.begin(), t.end(), m) != t.end()) seen = true;
        if (!seen) return fail(NEF_EPARSE, "output letter '%c' appears in no term", md.letter[m]);
    }
    if (n_obs != md.M) return fail(NEF_EINVAL, "model has %d observed letters, got %d shapes", md.M, n_obs);
    if (n_lat != md.K) return fail(NEF_EINVAL, "model has %d latent letters, got %d ranks", md.K, n_lat);
    if (md.M > 0 && !shapes) return fail(NEF_EINVAL, "shapes is NULL");
    if (md.K > 0 && !ranks) return fail(NEF_EINVAL, "ranks is NULL");
    md.dim.resize(md.letter.size());
    for (int m = 0; m < md.M; ++m) md.dim[m] = shapes[m];
    for (int k = 0; k < md.K; ++k) md.dim[md.M + k] = ranks[k];
    for (size_t x = 0; x < md.dim.size(); ++x)
        if (md.dim[x] < 1) return fail(NEF_EINVAL, "dimension of '%c' must be >= 1", md.letter[x]);
    md.N = 1;
    for (int m = 0; m < md.M; ++m) md.N *= md.dim[m];
    return NEF_OK;
}

// -------------------------------------------------------------- the plan
// An einsum recipe over global letter ids; pointers are bound at run time.
struct EinOpRef {
    int kind;        // 0 factor f, 1 workspace buffer
    int index;       // factor index or buffer id
    std::vector<int64_t> st;  // per global letter stride (size n_letters)
};

struct EinRecipe {
    std::vector<int> out_let, free_let;   // global ids
    std::vector<int64_t> out_st;          // destination strides (aligned with out_let)
    std::vector<EinOpRef> ops;
    int out_kind = 1, out_index = 0;      // destination: 0 factor, 1 buffer
    int64_t n_out_el = 1, n_free_el = 1;
};

// Recipes that compute the same tensor into the same layout (destinations aside).
bool same_recipe(const EinRecipe& a, const EinRecipe& b) {
    if (a.out_let != b.out_let || a.free_let != b.free_let || a.out_st != b.out_st || a.out_kind != b.out_kind ||
        a.n_out_el != b.n_out_el || a.n_free_el != b.n_free_el || a.ops.size() != b.ops.size())
        return false;
    for (size_t k = 0; k < a.ops.size(); ++k)
        if (a.ops[k].kind != b.ops[k].kind || a.ops[k].index != b.ops[k].index || a.ops[k].st != b.ops[k].st)
            return false;
    return true;
}

// Recipes of one contraction over two different buffers in operand 0 (numerator and
// denominator epilogues): one dual launch computes both.
bool dual_pair(const EinRecipe& a, const EinRecipe& b) {
    if (a.out_let != b.out_let || a.free_let != b.free_let || a.out_st != b.out_st || a.out_kind != b.out_kind ||
        a.ops.empty() || a.ops.size() != b.ops.size() || a.ops[0].kind != 1 || b.ops[0].kind != 1 ||
        a.ops[0].st != b.ops[0].st)
        return false;
    for (size_t k = 1; k < a.ops.size(); ++k)
        if (a.ops[k].kind != b.ops[k].kind || a.ops[k].index != b.ops[k].index || a.ops[k].st != b.ops[k].st)
            return false;
    return true;
}

enum BufId { B_NUM = 0, B_DEN, B_SNUM, B_SDEN, B_SPART_N, B_SPART_D, B_DENVEC, B_COLSUM0,
             B_WA = 20, B_WB, B_SRC0 = 32, B_CS0 = 4096 };

struct SourcePlan {
    EinRecipe build;       // writes the canonical [n x ld] matrix into buffer src_buf
    int buf;               // buffer id (>= B_SRC0)
    int64_t n_rows;        // rows of the canonical matrix
    SrcDesc desc;          // index terms (ptr bound at run time)
    int copy_of = -1;      // factor whose relabelled copy this is (kept current by its update)
    std::vector<int> deps;             // factors the build reads
    int cs_buf = -1;       // column sums of this operand (closed-form denominators), or -1
    bool shared = false;   // same recipe as an earlier pass's operand: reads that pass's buffer
};

struct PassPlan {
    int l = 0;
    bool generic = false;
    // view
    int run_s = 0, run_e = 0;
    std::vector<int> bond;            // global latent ids
    ViewDesc view{};
    SourcePlan P;
    std::vector<SourcePlan> Q;
    bool q_gathered = false;
    EinRecipe epi_num, epi_den;       // S -> num_l, den_l
    bool den_closed = false;          // b == 1 and no mask: den via column sums of Q
    std::vector<EinRecipe> colsum;    // per Q source: [ld] column sums into B_COLSUM0+k
    EinRecipe den_prod;               // product of the column sums -> B_DENVEC
    EinRecipe epi_den_closed;         // den_l from the broadcast den vector
    int n_split = 1;
    TcTileConfig tc{0, false};        // ring-depth configuration and Q path of the tensor-core pass
    int64_t cost = 0;
    std::string desc;
    bool finish_identity = false;     // epilogue is a relabelling of S: fused finish kernel
    bool dual_epi = false;            // epi_num and epi_den differ only in the S they read
    bool epi_s_once = false;          // the epilogue reads every element of S once
    // generic
    EinRecipe gen_num, gen_den;
};

struct Buffer {
    void* ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct nef_plan_s {
    Model md;
    nef_options opt{};
    int prec = NEF_FP32;
    size_t esz = 4;
    std::vector<PassPlan> pass;
    std::vector<Buffer> buf;          // indexed by BufId
    // fixed workspace
    void* ein_partial = nullptr;
    int64_t ein_partial_cap = 0;      // elements
    uint32_t* mask_bits = nullptr;
    double* loss_part = nullptr;
    int loss_part_cap = 0;
    double* loss_out = nullptr;
    int* flag = nullptr;
    int* tc_err = nullptr;
    unsigned long long* tc_trace = nullptr;  // wait-cycle counters of the tensor-core pass (profiling)
    std::vector<uint16_t*> src_bf16;  // per buffer id >= B_SRC0 (BF16 plans)
    std::string info;
    // profiling: event pairs around fused-pass launches, per kernel family
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    size_t ev_next = 0;
    // canonical operand copies kept current by each factor's update
    std::vector<std::vector<std::pair<int, int>>> mirrors_of;   // factor -> (pass, source: -1 = P)
    std::vector<int64_t> fac_version;
    int64_t version_counter = 0;
    // per source buffer: versions of the factors its build read when it was last built
    // (empty = stale); buffers are shared by passes whose operands have one recipe
    std::vector<std::vector<int64_t>> src_built;
    int sweep_launches[2] = {0, 0};   // kernels of one sweep without / with a mask, as last counted
    int64_t max_ld = 16;
    int64_t n_sm = 152;               // SMs of the plan's device (grid sizing)
    // per-sweep loss and graph replay of sweeps
    int* loss_count = nullptr;        // device: entries appended to the loss trace
    // stopping rules on the device: state, validation-loss outputs, packed validation mask
    FitCtlState* ctl = nullptr;
    double* val_out = nullptr;
    int* val_count = nullptr;
    uint32_t* val_bits = nullptr;
    bool sweeps_on_device = false;    // last_sweeps still to be read from ctl->done
    cudaStream_t cap_stream = nullptr;
    cudaStream_t body_stream = nullptr;  // captures the body of a conditional loop
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // captured sweeps, most recently used last: a fit replays the one recorded with
    // its arguments (data, mask, factors, loss trace, alpha, beta) or captures anew
    struct SweepGraph {
        std::vector<const void*> key;
        double ab[2];
        cudaGraphExec_t exec;
    };
    std::vector<SweepGraph> graphs;
    static constexpr size_t kMaxGraphs = 4;
    int last_sweeps = 0;
};

namespace nef {

void set_last_error(const char* msg) { g_err = msg ? msg : ""; }

WeightSpec weight_spec(double al, double be, int lik, double par) {
    WeightSpec w{};
    w.alpha = al;
    w.beta = be;
    if (lik != LIK_NONE) {
        // the likelihood families of App. B: b == 1 only for Jensen-Shannon
        w.lik = lik;
        w.par = par;
        w.y_code = POW_ONE;
        w.a_code = POW_GENERAL;
        w.b_code = lik == LIK_JS ? POW_ONE : POW_GENERAL;
        return w;
    }
    auto code = [](double e) {
        if (e == 0.0) return (int)POW_ONE;
        if (e == 1.0) return (int)POW_ID;
        if (e == -1.0) return (int)POW_RCP;
        if (e == -0.5) return (int)POW_RSQRT;
        if (e == 0.5) return (int)POW_SQRT;
        if (e == 2.0) return (int)POW_SQ;
        if (e == -1.5) return (int)POW_RSQRT3;
        if (e == -2.0) return (int)POW_RCP2;
        return (int)POW_GENERAL;
    };
    if (al == 0.0) {
        w.log_case = 1;
        w.y_code = POW_ONE;
        w.a_code = POW_ONE;
        w.b_code = POW_ONE;
        return w;
    }
    w.e_y = al;
    w.e_a = be - 1.0;
    w.e_b = al + be - 1.0;
    w.y_code = code(w.e_y);
    w.a_code = code(w.e_a);
    w.b_code = code(w.e_b);
    return w;
}

LossSpec loss_spec(double al, double be, int lik, double par) {
    LossSpec L{};
    L.alpha = al;
    L.beta = be;
    L.lik = lik;
    L.par = par;
    if (lik != LIK_NONE) return L;
    if (al != 0.0 && be != 0.0 && al + be != 0.0) L.kase = 0;
    else if (be == 0.0 && al != 0.0) L.kase = 1;
    else if (al == -be && al != 0.0) L.kase = 2;
    else if (al == 0.0 && be != 0.0) L.kase = 3;
    else L.kase = 4;
    return L;
}

UpdateSpec update_spec(double al, double be, double eps, int lik) {
    UpdateSpec u{};
    u.eps = eps;
    if (lik != LIK_NONE) {
        // g(lambda) = lambda (negative binomial, binomial) or log(lambda) (Jensen-Shannon)
        if (lik == LIK_JS) {
            u.log_case = 1;
        } else {
            u.eta = 1.0;
            u.eta_code = POW_ID;
        }
        return u;
    }
    if (al == 0.0 && be == 1.0) {
        u.log_case = 1;
        return u;
    }
    double q = 1.0 / al - be / al;
    double pexp = q > 1.0 ? 1.0 - be : (q < 0.0 ? al + be - 1.0 : al);
    u.eta = 1.0 / pexp;
    if (u.eta == 1.0) u.eta_code = POW_ID;
    else if (u.eta == 2.0) u.eta_code = POW_SQ;
    else if (u.eta == 0.5) u.eta_code = POW_SQRT;
    else if (u.eta == -1.0) u.eta_code = POW_RCP;
    else u.eta_code = POW_GENERAL;
    return u;
}

const char* loss_args_error(int lik, double al, double be, double par, bool* unsupported) {
    if (unsupported) *unsupported = false;
    switch (lik) {
        case LIK_NONE:
            if (!std::isfinite(al) || !std::isfinite(be)) return "alpha/beta must be finite";
            if (al == 0.0 && be != 1.0) {
                if (unsupported) *unsupported = true;
                return "alpha == 0 with beta != 1 has no decomposition (App. B)";
            }
            return nullptr;
        case LIK_NEGBIN:
            return (std::isfinite(par) && par > 0.0) ? nullptr : "negative binomial dispersion phi must be finite and > 0";
        case LIK_BINOMIAL:
            return (std::isfinite(par) && par > 0.0) ? nullptr : "binomial trial count n must be finite and > 0";
        case LIK_JS:
            return nullptr;
        default:
            return "unknown loss family";
    }
}

}  // namespace nef

namespace {

// ------------------------------------------------------------- planning
int64_t prod_dims(const Model& md, const std::vector<int>& ids) {
    int64_t n = 1;
    for (int x : ids) n *= md.dim[x];
    return n;
}

std::string letters_of(const Model& md, const std::vector<int>& ids) {
    std::string s;
    for (int x : ids) s.push_back(md.letter[x]);
    return s;
}

// Strides of a row-major layout over `ids` with an extra trailing block of `ld`
// elements for the bond letters (bond letters row-major inside the block).
void canon_strides(const Model& md, const std::vector<int>& rows, const std::vector<int>& bond,
                   int64_t ld, std::vector<int64_t>& st_of_letter) {
    st_of_letter.assign(md.letter.size(), 0);
    int64_t s = 1;
    for (int p = (int)bond.size() - 1; p >= 0; --p) {
        st_of_letter[bond[p]] = s;
        s *= md.dim[bond[p]];
    }
    s = ld;
    for (int p = (int)rows.size() - 1; p >= 0; --p) {
        st_of_letter[rows[p]] = s;
        s *= md.dim[rows[p]];
    }
}

EinOpRef factor_op(const Model& md, int f) {
    EinOpRef o;
    o.kind = 0;
    o.index = f;
    o.st.assign(md.letter.size(), 0);
    for (int x : md.term[f]) o.st[x] = md.fac_stride(f, x);
    return o;
}

void finish_recipe(const Model& md, EinRecipe& r) {
    r.n_out_el = prod_dims(md, r.out_let);
    r.n_free_el = prod_dims(md, r.free_let);
}

// Letters used by a set of factors.
std::vector<int> letters_used(const Model& md, const std::vector<int>& facs) {
    std::vector<int> used;
    for (int f : facs)
        for (int x : md.term[f])
            if (std::find(used.begin(), used.end(), x) == used.end()) used.push_back(x);
    std::sort(used.begin(), used.end());
    return used;
}

bool plan_view(const nef_plan_s& p, int l, int s, int e, int assign, int qform, PassPlan& out,
               int& next_buf) {
    const Model& md = p.md;
    std::vector<int> run, cols;
    for (int m = 0; m < md.M; ++m) (m >= s && m < e ? run : cols).push_back(m);
    if (cols.empty() || run.empty()) return false;
    auto in_run = [&](int x) { return x >= s && x < e; };
    // classify factors
    std::vector<int> cls(md.L);  // 0 row, 1 col, 2 latent-only
    for (int f = 0; f < md.L; ++f) {
        int nr = 0, nc = 0;
        for (int x : md.term[f])
            if (md.is_obs(x)) (in_run(x) ? nr : nc)++;
        if (nr && nc) return false;  // straddles the split
        cls[f] = nr ? 0 : (nc ? 1 : 2);
    }
    if (cls[l] == 1) return false;
    std::vector<int> lat_only;
    for (int f = 0; f < md.L; ++f)
        if (cls[f] == 2 && f != l) lat_only.push_back(f);
    if (lat_only.size() > 6) return false;
    if (assign >= (1 << lat_only.size())) return false;
    int64_t best_bond = -1;
    std::vector<int> best_row, best_col, best_bondv;
    {
        const int mask = assign;
        std::vector<int> rowf, colf;
        for (int f = 0; f < md.L; ++f) {
            if (cls[f] == 0 || f == l) rowf.push_back(f);
            else if (cls[f] == 1) colf.push_back(f);
        }
        for (size_t q = 0; q < lat_only.size(); ++q)
            ((mask >> q) & 1 ? colf : rowf).push_back(lat_only[q]);
        if (colf.empty()) return false;
        std::vector<int> rl, cl, bond;
        for (int x : letters_used(md, rowf)) if (!md.is_obs(x)) rl.push_back(x);
        for (int x : letters_used(md, colf)) if (!md.is_obs(x)) cl.push_back(x);
        for (int x : rl)
            if (std::find(cl.begin(), cl.end(), x) != cl.end()) bond.push_back(x);
        best_bond = prod_dims(md, bond);
        best_row = rowf;
        best_col = colf;
        best_bondv = bond;
    }
    const std::vector<int>& rowf = best_row;
    const std::vector<int>& colf = best_col;
    const std::vector<int>& bond = best_bondv;
    const int64_t bsz = best_bond;
    int64_t bond_pad;
    if (p.prec == NEF_FP64) bond_pad = bsz <= 32 ? 32 : (bsz <= 64 ? 64 : -1);
    else if (p.prec == NEF_BF16) bond_pad = bsz <= 16 ? 16 : (bsz <= 32 ? 32 : (bsz <= 64 ? 64 : (bsz <= 128 ? 128 : -1)));
    else bond_pad = bsz <= 16 ? 16 : (bsz <= 32 ? 32 : (bsz <= 64 ? 64 : -1));
    if (bond_pad < 0) return false;
    if (p.prec == NEF_BF16 && bond_pad > 64) return false;  // SIMT fallback must cover it too

    PassPlan pp;
    pp.l = l;
    pp.run_s = s;
    pp.run_e = e;
    pp.bond = bond;
    const int64_t rows = prod_dims(md, run);
    const int64_t ncols = prod_dims(md, cols);
    int64_t c_out = 1, c_in = 1;
    for (int m = 0; m < s; ++m) c_out *= md.dim[m];
    for (int m = e; m < md.M; ++m) c_in *= md.dim[m];
    pp.view.c_out = c_out;
    pp.view.rows = rows;
    pp.view.c_in = c_in;
    pp.view.bond = (int)bsz;
    pp.view.bond_pad = (int)bond_pad;

    // ---- P: canonical [rows x bond_pad] over the run letters, summing row-private latents
    {
        SourcePlan sp;
        sp.buf = next_buf++;
        sp.n_rows = rows;
        EinRecipe& r = sp.build;
        std::vector<int64_t> cst;
        canon_strides(md, run, bond, bond_pad, cst);
        r.out_let = run;
        for (int x : bond) r.out_let.push_back(x);
        for (int x : r.out_let) r.out_st.push_back(cst[x]);
        for (int x : letters_used(md, rowf))
            if (std::find(r.out_let.begin(), r.out_let.end(), x) == r.out_let.end())
                r.free_let.push_back(x);
        for (int f : rowf) r.ops.push_back(factor_op(md, f));
        r.out_kind = 1;
        r.out_index = sp.buf;
        finish_recipe(md, r);
        sp.desc = SrcDesc{};
        sp.desc.ld = bond_pad;
        sp.desc.nterm = 1;
        sp.desc.div[0] = 1;
        sp.desc.mod[0] = rows;
        sp.desc.mul[0] = 1;
        pp.P = sp;
        // a row letter without any row-side factor cannot happen: every observed letter is in a term
    }
    // ---- Q: gathered sources, or one dense operand over every column letter.
    // Each source is a group of column factors contracted over the latents private
    // to the group, indexed by the group's observed letters (RHS order) and the
    // bond; Q is the elementwise product of the sources, so every group must carry
    // every bond letter and no two groups may share a letter outside the bond.
    // qform 0 takes each column factor as its own group (it must carry exactly the
    // bond latents) and falls back to the dense operand; qform 1 joins factors that
    // share a letter outside the bond, and is tried only where qform 0 would not
    // gather; qform 2 takes the dense operand where qform 0 would gather (a small
    // dense operand is one TMA-staged source where the gathered form needs three or
    // four per tile), and the cost decides.
    std::vector<std::vector<int>> groups;
    auto is_bond = [&](int x) { return std::find(bond.begin(), bond.end(), x) != bond.end(); };
    bool gather = (int)colf.size() <= kMaxSrc;
    {
        std::vector<int> seen_obs;
        for (int f : colf) {
            std::vector<int> sb = bond, sf;
            for (int x : md.term[f]) if (!md.is_obs(x)) sf.push_back(x);
            std::sort(sb.begin(), sb.end());
            std::sort(sf.begin(), sf.end());
            int nobs = 0;
            for (int x : md.term[f])
                if (md.is_obs(x)) {
                    ++nobs;
                    if (std::find(seen_obs.begin(), seen_obs.end(), x) != seen_obs.end()) gather = false;
                    seen_obs.push_back(x);
                }
            if (sb != sf || nobs == 0) gather = false;
        }
        if ((int)seen_obs.size() != (int)cols.size()) gather = false;
    }
    if (qform == 2) {
        if (!gather) return false;  // qform 0 already builds the dense operand
    } else if (qform == 0) {
        if (gather)
            for (int f : colf) groups.push_back({f});
    } else {
        if (gather) return false;  // qform 0 already gathers this view
        std::vector<int> comp(colf.size());
        for (size_t a = 0; a < colf.size(); ++a) comp[a] = (int)a;
        auto root = [&](int a) {
            while (comp[a] != a) a = comp[a];
            return a;
        };
        for (size_t a = 0; a < colf.size(); ++a)
            for (size_t b = a + 1; b < colf.size(); ++b)
                for (int x : md.term[colf[a]])
                    if (!is_bond(x) && md.fac_has(colf[b], x)) comp[root((int)b)] = root((int)a);
        std::vector<int> rep;
        for (size_t a = 0; a < colf.size(); ++a) {
            const int r = root((int)a);
            auto it = std::find(rep.begin(), rep.end(), r);
            if (it == rep.end()) {
                rep.push_back(r);
                groups.push_back({colf[a]});
            } else {
                groups[it - rep.begin()].push_back(colf[a]);
            }
        }
        // a group without observed letters is a vector over the bond: fold it into
        // the first group that has some
        int host = -1;
        for (size_t g = 0; g < groups.size(); ++g)
            for (int x : letters_used(md, groups[g]))
                if (md.is_obs(x) && host < 0) host = (int)g;
        if (host < 0) return false;
        for (size_t g = 0; g < groups.size();) {
            bool has_obs = false;
            for (int x : letters_used(md, groups[g])) has_obs = has_obs || md.is_obs(x);
            if (has_obs) {
                ++g;
                continue;
            }
            for (int f : groups[g]) groups[host].push_back(f);
            groups.erase(groups.begin() + g);
            if ((int)g < host) --host;
        }
        if ((int)groups.size() > kMaxSrc) return false;
        for (auto& g : groups) {
            const std::vector<int> used = letters_used(md, g);
            for (int x : bond)
                if (std::find(used.begin(), used.end(), x) == used.end()) return false;
        }
    }
    // column index digits: col = mixed radix over `cols` (RHS order)
    auto col_div = [&](int x) {
        int64_t d = 1;
        bool after = false;
        for (int c : cols) {
            if (after) d *= md.dim[c];
            if (c == x) after = true;
        }
        return d;
    };
    // index terms of a source over its observed letters: one per letter, and
    // neighbours in both the column order and the source's row order merge
    struct Terms {
        std::vector<int64_t> div, mod, mul;
    };
    auto index_terms = [&](const std::vector<int>& fobs, const std::vector<int64_t>& cst) {
        Terms t;
        for (int x : fobs) {
            const int64_t d = col_div(x), m = md.dim[x], u = cst[x] / bond_pad;
            if (!t.div.empty() && t.div.back() == d * m && t.mul.back() == u * m) {
                t.div.back() = d;
                t.mod.back() *= m;
                t.mul.back() = u;
            } else {
                t.div.push_back(d);
                t.mod.push_back(m);
                t.mul.push_back(u);
            }
        }
        return t;
    };
    auto group_obs = [&](const std::vector<int>& g) {
        std::vector<int> fobs;
        for (int x : letters_used(md, g))
            if (md.is_obs(x)) fobs.push_back(x);  // ascending = RHS order
        return fobs;
    };
    for (auto& g : groups) {
        const std::vector<int> fobs = group_obs(g);
        std::vector<int64_t> cst;
        canon_strides(md, fobs, bond, bond_pad, cst);
        const bool too_big = g.size() > 1 && prod_dims(md, fobs) * bond_pad > md.N / 4;
        if (too_big || (int)index_terms(fobs, cst).div.size() > kMaxTerm) {
            if (qform != 0) return false;
            groups.clear();  // qform 0: dense operand instead
            break;
        }
    }
    int64_t prep_elems = rows * bond_pad;
    for (auto& g : groups) {
        SourcePlan sp;
        sp.buf = next_buf++;
        const std::vector<int> fobs = group_obs(g);
        sp.n_rows = prod_dims(md, fobs);
        std::vector<int64_t> cst;
        canon_strides(md, fobs, bond, bond_pad, cst);
        EinRecipe& r = sp.build;
        r.out_let = fobs;
        for (int x : bond) r.out_let.push_back(x);
        for (int x : r.out_let) r.out_st.push_back(cst[x]);
        for (int x : letters_used(md, g))
            if (std::find(r.out_let.begin(), r.out_let.end(), x) == r.out_let.end()) r.free_let.push_back(x);
        for (int f : g) r.ops.push_back(factor_op(md, f));
        r.out_kind = 1;
        r.out_index = sp.buf;
        finish_recipe(md, r);
        sp.desc = SrcDesc{};
        sp.desc.ld = bond_pad;
        const Terms t = index_terms(fobs, cst);
        sp.desc.nterm = (int)t.div.size();
        for (size_t k = 0; k < t.div.size(); ++k) {
            sp.desc.div[k] = t.div[k];
            sp.desc.mod[k] = t.mod[k];
            sp.desc.mul[k] = t.mul[k];
        }
        prep_elems += sp.n_rows * bond_pad;
        pp.Q.push_back(sp);
    }
    gather = !groups.empty();
    if (gather) {
        pp.q_gathered = true;
    } else {
        if (ncols * bond_pad > md.N / 4) return false;
        SourcePlan sp;
        sp.buf = next_buf++;
        sp.n_rows = ncols;
        std::vector<int64_t> cst;
        canon_strides(md, cols, bond, bond_pad, cst);
        EinRecipe& r = sp.build;
        r.out_let = cols;
        for (int x : bond) r.out_let.push_back(x);
        for (int x : r.out_let) r.out_st.push_back(cst[x]);
        for (int x : letters_used(md, colf))
            if (std::find(r.out_let.begin(), r.out_let.end(), x) == r.out_let.end())
                r.free_let.push_back(x);
        for (int f : colf) r.ops.push_back(factor_op(md, f));
        r.out_kind = 1;
        r.out_index = sp.buf;
        finish_recipe(md, r);
        sp.desc = SrcDesc{};
        sp.desc.ld = bond_pad;
        sp.desc.nterm = 1;
        sp.desc.div[0] = 1;
        sp.desc.mod[0] = ncols;
        sp.desc.mul[0] = 1;
        prep_elems += ncols * bond_pad;
        pp.Q.push_back(sp);
    }
    // ---- epilogue: num_l = einsum(S[run, bond], other row-side factors -> l)
    auto make_epi = [&](int s_buf, bool broadcast_rows) {
        EinRecipe r;
        r.out_let = md.term[l];
        for (int x : md.term[l]) r.out_st.push_back(md.fac_stride(l, x));
        EinOpRef sop;
        sop.kind = 1;
        sop.index = s_buf;
        sop.st.assign(md.letter.size(), 0);
        std::vector<int64_t> cst;
        canon_strides(md, run, bond, bond_pad, cst);
        for (int x : run) sop.st[x] = broadcast_rows ? 0 : cst[x];
        for (int x : bond) sop.st[x] = cst[x];
        r.ops.push_back(sop);
        std::vector<int> used = run;
        for (int x : bond) used.push_back(x);
        for (int f : rowf) {
            if (f == l) continue;
            r.ops.push_back(factor_op(md, f));
            for (int x : md.term[f]) used.push_back(x);
        }
        std::sort(used.begin(), used.end());
        used.erase(std::unique(used.begin(), used.end()), used.end());
        for (int x : used)
            if (!md.fac_has(l, x)) r.free_let.push_back(x);
        r.out_kind = 1;
        r.out_index = -1;  // bound later (B_NUM / B_DEN)
        finish_recipe(md, r);
        return r;
    };
    pp.epi_num = make_epi(B_SNUM, false);
    pp.epi_num.out_index = B_NUM;
    pp.epi_den = make_epi(B_SDEN, false);
    pp.epi_den.out_index = B_DEN;
    // closed-form denominator (used when b == 1 and there is no mask)
    pp.den_closed = pp.q_gathered;
    if (pp.den_closed) {
        for (size_t k = 0; k < pp.Q.size(); ++k) {
            const SourcePlan& sp = pp.Q[k];
            EinRecipe r;
            // sum over the canonical rows of source k: treat it as a [n_rows x ld] matrix with
            // pseudo letters: we reuse the source's own out letters
            r.out_let = bond;
            std::vector<int64_t> bst;
            canon_strides(md, {}, bond, bond_pad, bst);
            for (int x : bond) r.out_st.push_back(bst[x]);
            EinOpRef o;
            o.kind = 1;
            o.index = sp.buf;
            o.st.assign(md.letter.size(), 0);
            for (size_t q = 0; q < sp.build.out_let.size(); ++q) o.st[sp.build.out_let[q]] = sp.build.out_st[q];
            r.ops.push_back(o);
            for (int x : sp.build.out_let)
                if (std::find(bond.begin(), bond.end(), x) == bond.end()) r.free_let.push_back(x);
            r.out_kind = 1;
            r.out_index = B_COLSUM0 + (int)k;
            finish_recipe(md, r);
            pp.colsum.push_back(r);
        }
        EinRecipe pr;
        pr.out_let = bond;
        std::vector<int64_t> bst;
        canon_strides(md, {}, bond, bond_pad, bst);
        for (int x : bond) pr.out_st.push_back(bst[x]);
        for (size_t k = 0; k < pp.Q.size(); ++k) {
            EinOpRef o;
            o.kind = 1;
            o.index = B_COLSUM0 + (int)k;
            o.st.assign(md.letter.size(), 0);
            for (int x : bond) o.st[x] = bst[x];
            pr.ops.push_back(o);
        }
        pr.out_kind = 1;
        pr.out_index = B_DENVEC;
        finish_recipe(md, pr);
        pp.den_prod = pr;
        pp.epi_den_closed = make_epi(B_DENVEC, true);
        pp.epi_den_closed.out_index = B_DEN;
    }
    // ---- split of the columns across CTAs
    const int tm = (p.prec == NEF_FP64) ? 32 : (p.prec == NEF_BF16 ? 128 : 64);
    const int tn = (p.prec == NEF_FP64) ? 32 : (p.prec == NEF_BF16 ? 128 : 64);
    const int64_t n_rb = (rows + tm - 1) / tm;
    const int64_t tiles = (ncols + tn - 1) / tn;
    // one wave: one tensor-core CTA per SM (its shared memory fills the SM), four
    // CUDA-core CTAs per SM
    // CUDA-core CTAs per SM; the split count fills the waves of CTAs best (the
    // fraction of the last wave in use), preferring fewer splits on a tie, among
    // up to four times one wave's worth
    const int64_t target = (p.prec == NEF_BF16) ? p.n_sm : p.n_sm * 4;
    int64_t ns = 1;
    {
        // the fewest waves of CTAs that keep >= 90 % of the SMs busy (a CTA has a fixed
        // start-up and drain, so one long CTA per SM beats several short ones), else the
        // best-filled split over up to four waves
        const int64_t rbs = std::max<int64_t>(1, n_rb);
        const int64_t hi = std::max<int64_t>(1, std::min<int64_t>(tiles, 4 * ((target + rbs - 1) / rbs)));
        double best = -1.0;
        int64_t best_waves = 0;
        for (int64_t c = 1; c <= hi; ++c) {
            const int64_t ctas = rbs * c;
            const int64_t waves = (ctas + target - 1) / target;
            const double eff = (double)ctas / (double)(waves * target);
            const bool settled = best >= 0.9 && waves > best_waves;  // a fuller, earlier wave count won
            if (!settled && eff > best + 1e-9) {
                best = eff;
                best_waves = waves;
                ns = c;
            }
        }
    }
    pp.n_split = (int)ns;
    pp.view.P.nsrc = 1;
    pp.view.Q.nsrc = (int)pp.Q.size();
    // ---- cost: bytes moved per pass
    int64_t epi_cost = pp.epi_num.n_out_el * pp.epi_num.n_free_el;
    pp.cost = md.N * 4 + prep_elems * 8 + ns * rows * bond_pad * 8 + epi_cost / 4 +
              (gather ? 0 : ncols * bond_pad * 4 * 4);
    // rows past the last full tile of tm rows are computed and discarded
    pp.cost += (int64_t)((double)md.N * 4.0 * ((double)(n_rb * tm) / (double)rows - 1.0));
    // small kernels per pass (a few microseconds each): every operand that is not a
    // relabelled copy of one factor is rebuilt, and an epilogue that contracts runs
    // its own reduction, contractions and update
    {
        auto is_copy = [&](const EinRecipe& r) {
            if (r.ops.size() != 1 || r.ops[0].kind != 0 || !r.free_let.empty()) return false;
            const int f = r.ops[0].index;
            if (r.out_let.size() < md.term[f].size()) return false;
            for (int x : md.term[f])
                if (std::find(r.out_let.begin(), r.out_let.end(), x) == r.out_let.end()) return false;
            return true;
        };
        int launches = is_copy(pp.P.build) ? 0 : 1;
        for (auto& q : pp.Q) launches += is_copy(q.build) ? 0 : 1;
        if (pp.epi_num.ops.size() != 1 || !pp.epi_num.free_let.empty()) launches += 4;
        constexpr int64_t kLaunchBytes = (int64_t)16 << 20;
        pp.cost += launches * kLaunchBytes;
    }
    if (p.prec == NEF_BF16) {
        // the tensor-core pass gathers Q rows per tile where it cannot stage them
        // with TMA, which is slower: weigh that as half a read of Y
        ViewDesc vv = pp.view;
        vv.Q.nsrc = (int)pp.Q.size();
        for (size_t k = 0; k < pp.Q.size() && k < (size_t)kMaxSrc; ++k) vv.Q.src[k] = pp.Q[k].desc;
        int q_var, q_const;
        if (!q_rows_staged(vv, kTcTileN, &q_var, &q_const)) pp.cost += md.N * 2;
    }
    char d[512];
    snprintf(d, sizeof(d),
             "factor %d '%s': view rows='%s' (%lld) cols=%lld [c_out=%lld c_in=%lld] bond='%s' "
             "(%lld->%lld) Q=%s(%d) splits=%d epilogue=%lldx%lld",
             l, letters_of(md, md.term[l]).c_str(), letters_of(md, run).c_str(), (long long)rows,
             (long long)ncols, (long long)c_out, (long long)c_in, letters_of(md, bond).c_str(),
             (long long)bsz, (long long)bond_pad, gather ? "gather" : "dense", (int)pp.Q.size(),
             pp.n_split, (long long)pp.epi_num.n_out_el, (long long)pp.epi_num.n_free_el);
    pp.desc = d;
    out = pp;
    return true;
}

void plan_generic(const nef_plan_s& p, int l, PassPlan& pp) {
    const Model& md = p.md;
    pp.l = l;
    pp.generic = true;
    auto mk = [&](int wbuf, int obuf) {
        EinRecipe r;
        r.out_let = md.term[l];
        for (int x : md.term[l]) r.out_st.push_back(md.fac_stride(l, x));
        EinOpRef w;
        w.kind = 1;
        w.index = wbuf;
        w.st.assign(md.letter.size(), 0);
        for (int m = 0; m < md.M; ++m) w.st[m] = md.y_stride(m);
        r.ops.push_back(w);
        for (int f = 0; f < md.L; ++f)
            if (f != l) r.ops.push_back(factor_op(md, f));
        for (int x = 0; x < (int)md.letter.size(); ++x)
            if (!md.fac_has(l, x)) r.free_let.push_back(x);
        r.out_kind = 1;
        r.out_index = obuf;
        finish_recipe(md, r);
        return r;
    };
    pp.gen_num = mk(B_WA, B_NUM);
    pp.gen_den = mk(B_WB, B_DEN);
    char d[256];
    snprintf(d, sizeof(d), "factor %d '%s': generic (yhat, a, b materialised; einstr contraction)",
             l, letters_of(md, md.term[l]).c_str());
    pp.desc = d;
}

// ------------------------------------------------------------- run time
void* buf_ptr(nef_plan_t p, int id) { return p->buf[id].ptr; }

EinDesc bind(nef_plan_t p, const EinRecipe& r, void* const* factors) {
    EinDesc d{};
    const int nl = (int)(r.out_let.size() + r.free_let.size());
    d.n_ops = (int)r.ops.size();
    d.n_out = (int)r.out_let.size();
    d.n_free = (int)r.free_let.size();
    std::vector<int> lets = r.out_let;
    lets.insert(lets.end(), r.free_let.begin(), r.free_let.end());
    for (int q = 0; q < nl; ++q) d.dim[q] = p->md.dim[lets[q]];
    for (int k = 0; k < d.n_ops; ++k) {
        const EinOpRef& o = r.ops[k];
        d.op[k] = o.kind == 0 ? factors[o.index] : buf_ptr(p, o.index);
        for (int q = 0; q < nl; ++q) d.ost[k][q] = o.st[lets[q]];
    }
    for (int q = 0; q < d.n_out; ++q) d.out_st[q] = r.out_st[q];
    d.n_out_el = r.n_out_el;
    d.n_free_el = r.n_free_el;
    d.out = r.out_kind == 0 ? factors[r.out_index] : buf_ptr(p, r.out_index);
    d.accumulate = 0;
    return d;
}

bool recipe_fits(const EinRecipe& r) {
    return r.ops.size() <= (size_t)kMaxEinOps && r.out_let.size() + r.free_let.size() <= (size_t)kMaxEinLet;
}

template <typename T>
nef_status run_ein(nef_plan_t p, const EinRecipe& r, void* const* factors, cudaStream_t st) {
    EinDesc d = bind(p, r, factors);
    NEF_CUDA(launch_einsum<T>(d, static_cast<T*>(p->ein_partial), p->ein_partial_cap, st));
    return NEF_OK;
}

#define NEF_TRY(x)                     \
    do {                               \
        nef_status s_ = (x);           \
        if (s_ != NEF_OK) return s_;   \
    } while (0)

ViewDesc bind_view(nef_plan_t p, const PassPlan& pp, bool bf16) {
    ViewDesc v = pp.view;
    v.P.nsrc = 1;
    v.P.src[0] = pp.P.desc;
    v.P.src[0].ptr = bf16 ? (const void*)p->src_bf16[pp.P.buf] : buf_ptr(p, pp.P.buf);
    v.Q.nsrc = (int)pp.Q.size();
    for (size_t k = 0; k < pp.Q.size(); ++k) {
        v.Q.src[k] = pp.Q[k].desc;
        v.Q.src[k].ptr = bf16 ? (const void*)p->src_bf16[pp.Q[k].buf] : buf_ptr(p, pp.Q[k].buf);
    }
    return v;
}

SourcePlan& source_ref(PassPlan& pp, int k) { return k < 0 ? pp.P : pp.Q[k]; }

// The canonical copies of factor f that its update writes (FP32/FP64 and BF16).
MirrorDesc mirror_desc(nef_plan_t p, int f) {
    MirrorDesc m{};
    const Model& md = p->md;
    for (auto& ps : p->mirrors_of[f]) {
        SourcePlan& sp = source_ref(p->pass[ps.first], ps.second);
        const int k = m.n++;
        m.p32[k] = buf_ptr(p, sp.buf);
        m.p16[k] = (p->prec == NEF_BF16) ? p->src_bf16[sp.buf] : nullptr;
        for (size_t q = 0; q < md.term[f].size(); ++q) {
            const int x = md.term[f][q];
            const auto it = std::find(sp.build.out_let.begin(), sp.build.out_let.end(), x);
            m.st[k][q] = sp.build.out_st[it - sp.build.out_let.begin()];
        }
    }
    return m;
}

// Column-sum jobs for the closed-form denominators that read copies of factor f
// (f < 0: every factor).
ColsumDesc colsum_jobs(nef_plan_t p, int f) {
    ColsumDesc d{};
    for (int g = 0; g < p->md.L; ++g) {
        if (f >= 0 && g != f) continue;
        for (auto& ps : p->mirrors_of[g]) {
            SourcePlan& sp = source_ref(p->pass[ps.first], ps.second);
            if (sp.cs_buf < 0 || d.n >= kMaxColsumJobs) continue;
            ColsumJob& j = d.job[d.n++];
            j.src = buf_ptr(p, sp.buf);
            j.n_rows = sp.n_rows;
            j.ld = sp.desc.ld;
            j.out = buf_ptr(p, sp.cs_buf);
        }
    }
    return d;
}

bool source_stale(nef_plan_t p, const SourcePlan& sp) {
    if (sp.copy_of >= 0) return false;
    const std::vector<int64_t>& built = p->src_built[sp.buf];
    if (built.size() != sp.deps.size()) return true;
    for (size_t k = 0; k < sp.deps.size(); ++k)
        if (built[k] != p->fac_version[sp.deps[k]]) return true;
    return false;
}

// Start of every call: the caller may have changed the factors, so rebuild every
// kept copy from them and mark the contracted operands stale.
template <typename T>
nef_status init_sources(nef_plan_t p, void* const* factors, cudaStream_t st) {
    const Model& md = p->md;
    for (int f = 0; f < md.L; ++f) {
        p->fac_version[f] = ++p->version_counter;
        if (p->mirrors_of[f].empty()) continue;
        MirrorDesc m = mirror_desc(p, f);
        std::vector<int64_t> dims;
        for (int x : md.term[f]) dims.push_back(md.dim[x]);
        NEF_CUDA(launch_mirror_init<T>(static_cast<const T*>(factors[f]), md.fac_size(f), (int)dims.size(),
                                       dims.data(), m, st));
    }
    ColsumDesc cs = colsum_jobs(p, -1);
    NEF_CUDA(launch_colsums<T>(cs, p->max_ld, st));
    return NEF_OK;
}

// Rebuild the contracted operands of a pass whose factors changed since their last build.
template <typename T>
nef_status refresh_sources(nef_plan_t p, PassPlan& pp, void* const* factors, cudaStream_t st, bool bf16) {
    for (int k = -1; k < (int)pp.Q.size(); ++k) {
        SourcePlan& sp = source_ref(pp, k);
        if (!source_stale(p, sp)) continue;
        // the build also writes the BF16 copy the tensor-core pass reads (and rounds the
        // FP32 values to it); the copy's padding columns stay zero from allocation
        EinDesc d = bind(p, sp.build, factors);
        if constexpr (sizeof(T) == 4) {
            if (bf16) d.out16 = p->src_bf16[sp.buf];
        }
        NEF_CUDA(launch_einsum<T>(d, static_cast<T*>(p->ein_partial), p->ein_partial_cap, st));
        std::vector<int64_t>& built = p->src_built[sp.buf];
        built.clear();
        for (int g : sp.deps) built.push_back(p->fac_version[g]);
    }
    return NEF_OK;
}

// After factor l changed: its copies were written by the update; refresh the
// column sums that read them and bump its version.
template <typename T>
nef_status after_update(nef_plan_t p, int l, cudaStream_t st) {
    ColsumDesc cs = colsum_jobs(p, l);
    NEF_CUDA(launch_colsums<T>(cs, p->max_ld, st));
    p->fac_version[l] = ++p->version_counter;
    return NEF_OK;
}

// Event pair for one profiled launch (pool grows on demand, reused after reset).
nef_status prof_begin(nef_plan_t p, cudaStream_t st, cudaEvent_t* a, cudaEvent_t* b) {
    while (p->ev_next + 2 > p->ev_pool.size()) {
        cudaEvent_t e;
        NEF_CUDA(cudaEventCreate(&e));
        p->ev_pool.push_back(e);
    }
    *a = p->ev_pool[p->ev_next++];
    *b = p->ev_pool[p->ev_next++];
    NEF_CUDA(cudaEventRecord(*a, st));
    return NEF_OK;
}

// One factor update (Algorithm 1's inner step).  With export_num/export_den the
// pass stops after forming num and den (Eq. 3.6-3.8), copies them there and
// leaves the factor unchanged (the caller sums them over shards of Y first).
template <typename T>
nef_status run_pass(nef_plan_t p, PassPlan& pp, const T* y, const uint32_t* mbits,
                    void* const* factors, const WeightSpec& w, const UpdateSpec& u, cudaStream_t st,
                    const LossSpec* loss = nullptr, int* n_part = nullptr, T* export_num = nullptr,
                    T* export_den = nullptr) {
    const Model& md = p->md;
    const int64_t nl = md.fac_size(pp.l);
    T* num = static_cast<T*>(buf_ptr(p, B_NUM));
    T* den = static_cast<T*>(buf_ptr(p, B_DEN));
    std::vector<int64_t> ldims;
    for (int x : md.term[pp.l]) ldims.push_back(md.dim[x]);
    const MirrorDesc mir = mirror_desc(p, pp.l);
    if (pp.generic) {
        GenericRecon g{};
        g.n_obs = md.M;
        g.n_let = (int)md.letter.size();
        g.n_fac = md.L;
        for (int x = 0; x < g.n_let; ++x) g.dim[x] = md.dim[x];
        for (int f = 0; f < md.L; ++f) {
            for (int x = 0; x < g.n_let; ++x) g.fst[f][x] = md.fac_stride(f, x);
            g.fac[f] = factors[f];
        }
        g.n = md.N;
        g.n_lat_el = 1;
        for (int x = md.M; x < g.n_let; ++x) g.n_lat_el *= md.dim[x];
        const int np = loss ? (int)std::min<int64_t>((md.N + 255) / 256, p->loss_part_cap / 2) : 0;
        if (n_part) *n_part = np;
        NEF_CUDA(launch_generic_weights<T>(g, y, mbits, w, static_cast<T*>(buf_ptr(p, B_WA)),
                                           static_cast<T*>(buf_ptr(p, B_WB)), loss, loss ? p->loss_part : nullptr,
                                           np, st));
        NEF_TRY(run_ein<T>(p, pp.gen_num, factors, st));
        NEF_TRY(run_ein<T>(p, pp.gen_den, factors, st));
        if (export_num) {
            NEF_CUDA(cudaMemcpyAsync(export_num, num, nl * sizeof(T), cudaMemcpyDeviceToDevice, st));
            NEF_CUDA(cudaMemcpyAsync(export_den, den, nl * sizeof(T), cudaMemcpyDeviceToDevice, st));
            return NEF_OK;
        }
        NEF_CUDA(launch_update_mirror<T>(static_cast<T*>(factors[pp.l]), num, den, nl, u, (int)ldims.size(),
                                         ldims.data(), mir, st));
        return after_update<T>(p, pp.l, st);
    }
    const bool closed = pp.den_closed && weights_b_is_one(w) && mbits == nullptr;
    const int need_den = closed ? 0 : 1;
    bool use_tc = false;
    if constexpr (sizeof(T) == 4) use_tc = p->prec == NEF_BF16 && tc_view_supported(bind_view(p, pp, true), need_den);
    NEF_TRY(refresh_sources<T>(p, pp, factors, st, use_tc));
    const int64_t sz = pp.view.rows * pp.view.bond_pad;
    T* spn = static_cast<T*>(buf_ptr(p, B_SPART_N));
    T* spd = static_cast<T*>(buf_ptr(p, B_SPART_D));
    const int n_split = pp.n_split;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (p->opt.profile) NEF_TRY(prof_begin(p, st, &e0, &e1));
    if (use_tc) {
        if constexpr (sizeof(T) == 4) {
            ViewDesc v = bind_view(p, pp, true);
            TcLaunchInfo info{};
            NEF_CUDA(launch_view_tc(reinterpret_cast<const float*>(y), mbits, v, w, need_den, n_split,
                                    reinterpret_cast<float*>(spn), reinterpret_cast<float*>(spd),
                                    p->tc_err, st, &info, p->tc_trace, loss, loss ? p->loss_part : nullptr,
                                    p->opt.wait_cycles, &pp.tc));
            if (n_part) *n_part = info.n_ctas;
        }
    } else {
        ViewDesc v = bind_view(p, pp, false);
        int n_ctas = 0;
        NEF_CUDA(launch_view_simt<T>(y, mbits, v, w, need_den, n_split, spn, need_den ? spd : nullptr,
                                     loss, loss ? p->loss_part : nullptr, st, &n_ctas));
        if (n_part) *n_part = n_ctas;
    }
    if (p->opt.profile) {
        NEF_CUDA(cudaEventRecord(e1, st));
        p->ev_used.push_back({use_tc ? 0 : 1, {e0, e1}});
    }
    if (pp.finish_identity && !export_num) {
        // split reduction, denominator, update and the factor's copies in one kernel
        FinishDesc d{};
        d.nlet = (int)ldims.size();
        for (int q = 0; q < d.nlet; ++q) {
            const int x = md.term[pp.l][q];
            d.dim[q] = ldims[q];
            d.s_st[q] = pp.epi_num.ops[0].st[x];
            d.b_st[q] = closed ? pp.epi_den_closed.ops[0].st[x] : 0;
        }
        d.part_num = spn;
        d.part_den = closed ? nullptr : spd;
        d.n_split = n_split;
        d.s_size = sz;
        d.n_cs = closed ? (int)pp.Q.size() : 0;
        if (closed)
            for (size_t k = 0; k < pp.Q.size(); ++k) d.cs[k] = buf_ptr(p, pp.Q[k].cs_buf);
        d.theta = factors[pp.l];
        d.n = nl;
        d.mir = mir;
        NEF_CUDA(launch_finish<T>(d, u, st));
        return after_update<T>(p, pp.l, st);
    }
    // S = the sum of the split partials (one split: the partials are S); numerator and
    // denominator reduced in one launch, and contracted by one dual epilogue where
    // their recipes differ only in which S they read
    // (an epilogue that reads each element of S once sums the partials as it reads them)
    const bool in_place = n_split == 1 || (pp.epi_s_once && (!need_den || pp.dual_epi));
    T* snum = in_place ? spn : static_cast<T*>(buf_ptr(p, B_SNUM));
    T* sden = in_place ? spd : static_cast<T*>(buf_ptr(p, B_SDEN));
    if (!in_place) {
        if (need_den) NEF_CUDA(launch_reduce_splits2<T>(spn, spd, n_split, sz, snum, sden, st));
        else NEF_CUDA(launch_reduce_splits<T>(spn, n_split, sz, snum, st));
    }
    EinDesc en = bind(p, pp.epi_num, factors);
    en.op[0] = snum;
    if (in_place && n_split > 1) {
        en.op0_splits = n_split;
        en.op0_split_stride = sz;
    }
    // the epilogue's last contraction also applies Eq. 3.4 to its outputs (the factor's
    // elements) and writes the factor's copies, unless num and den are exported
    EinUpdate up{};
    up.theta = factors[pp.l];
    up.nlet = (int)ldims.size();
    for (int q = 0; q < up.nlet; ++q) up.dim[q] = ldims[q];
    up.mir = mir;
    up.u = u;
    auto last = [&](const EinDesc& d, const void* num_in) -> cudaError_t {
        if (export_num) return launch_einsum<T>(d, static_cast<T*>(p->ein_partial), p->ein_partial_cap, st);
        EinUpdate uu = up;
        uu.num = num_in;
        return launch_einsum_update<T>(d, uu, static_cast<T*>(p->ein_partial), p->ein_partial_cap, st);
    };
    if (need_den && pp.dual_epi) {
        en.op0b = sden;
        en.outb = buf_ptr(p, B_DEN);
        NEF_CUDA(last(en, nullptr));
    } else if (need_den) {
        NEF_CUDA(launch_einsum<T>(en, static_cast<T*>(p->ein_partial), p->ein_partial_cap, st));
        EinDesc ed = bind(p, pp.epi_den, factors);
        ed.op[0] = sden;
        NEF_CUDA(last(ed, num));
    } else {
        NEF_CUDA(launch_einsum<T>(en, static_cast<T*>(p->ein_partial), p->ein_partial_cap, st));
        for (auto& r : pp.colsum) NEF_TRY(run_ein<T>(p, r, factors, st));
        NEF_TRY(run_ein<T>(p, pp.den_prod, factors, st));
        NEF_CUDA(last(bind(p, pp.epi_den_closed, factors), num));
    }
    if (export_num) {
        NEF_CUDA(cudaMemcpyAsync(export_num, num, nl * sizeof(T), cudaMemcpyDeviceToDevice, st));
        NEF_CUDA(cudaMemcpyAsync(export_den, den, nl * sizeof(T), cudaMemcpyDeviceToDevice, st));
        return NEF_OK;
    }
    return after_update<T>(p, pp.l, st);
}


// The plan's loss family with the call's (alpha, beta) (ignored by the likelihood families).
nef_status check_ab(nef_plan_t p, double al, double be) {
    bool unsup = false;
    const char* msg = loss_args_error(p->opt.loss, al, be, p->opt.loss_par, &unsup);
    if (msg) return fail(unsup ? NEF_EUNSUPPORTED : NEF_EINVAL, "%s", msg);
    return NEF_OK;
}

struct Specs {
    WeightSpec w;
    UpdateSpec u;
    LossSpec L;
};

Specs specs_of(nef_plan_t p, double al, double be) {
    const int lik = p->opt.loss;
    const double par = p->opt.loss_par;
    return Specs{weight_spec(al, be, lik, par), update_spec(al, be, p->opt.eps, lik), loss_spec(al, be, lik, par)};
}

template <typename T>
nef_status prologue(nef_plan_t p, const void* Y, const uint8_t* mask, void* const* factors,
                    cudaStream_t st, const uint32_t** mbits) {
    if (!Y) return fail(NEF_EINVAL, "Y is NULL");
    if (!factors) return fail(NEF_EINVAL, "factors is NULL");
    for (int f = 0; f < p->md.L; ++f)
        if (!factors[f]) return fail(NEF_EINVAL, "factor %d is NULL", f);
    *mbits = nullptr;
    if (mask) {
        NEF_CUDA(launch_pack_mask(mask, p->md.N, p->mask_bits, st));
        *mbits = p->mask_bits;
    }
    if (p->opt.check_data) {
        NEF_CUDA(cudaMemsetAsync(p->flag, 0, sizeof(int), st));
        NEF_CUDA(launch_check_data<T>(static_cast<const T*>(Y), p->md.N, p->flag, st));
        int h = 0;
        NEF_CUDA(cudaMemcpyAsync(&h, p->flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        NEF_CUDA(cudaStreamSynchronize(st));
        if (h) return fail(NEF_EDATA, "Y holds a negative or non-finite entry");
    }
    return NEF_OK;
}

// num and den of factor l at the caller's factors (nef_numden), or the update of
// factor l from given num and den (nef_apply_update: num_in set).
template <typename T>
nef_status numden_impl(nef_plan_t p, int l, const void* Y, const uint8_t* mask, void* const* factors, double al,
                       double be, T* num, T* den, const T* num_in = nullptr, const T* den_in = nullptr) {
    cudaStream_t st = static_cast<cudaStream_t>(p->opt.stream);
    if (p->opt.loss != NEF_LOSS_AB) al = be = 0.0;
    const Specs sp = specs_of(p, al, be);
    if (num_in) {
        if (!factors) return fail(NEF_EINVAL, "factors is NULL");
        for (int f = 0; f < p->md.L; ++f)
            if (!factors[f]) return fail(NEF_EINVAL, "factor %d is NULL", f);
        NEF_TRY(init_sources<T>(p, factors, st));
        const Model& md = p->md;
        std::vector<int64_t> ldims;
        for (int x : md.term[l]) ldims.push_back(md.dim[x]);
        NEF_CUDA(launch_update_mirror<T>(static_cast<T*>(factors[l]), num_in, den_in, md.fac_size(l), sp.u,
                                         (int)ldims.size(), ldims.data(), mirror_desc(p, l), st));
        return after_update<T>(p, l, st);
    }
    const uint32_t* mbits = nullptr;
    NEF_TRY(prologue<T>(p, Y, mask, factors, st, &mbits));
    NEF_TRY(init_sources<T>(p, factors, st));
    return run_pass<T>(p, p->pass[l], static_cast<const T*>(Y), mbits, factors, sp.w, sp.u, st, nullptr, nullptr,
                       num, den);
}

// One sweep of Algorithm 1 (or the single update only_l).  With `loss`, the
// first pass also sums the loss of the factors it starts from, and the sum is
// appended to the loss trace.
template <typename T>
nef_status sweep_once(nef_plan_t p, const T* y, const uint32_t* mbits, void* const* factors, const WeightSpec& w,
                      const UpdateSpec& u, const LossSpec* loss, double* trace, int only_l, cudaStream_t st) {
    bool first = true;
    const long long c0 = kernel_launches();
    for (int l = 0; l < p->md.L; ++l) {
        if (only_l >= 0 && l != only_l) continue;
        const LossSpec* lp = first ? loss : nullptr;
        first = false;
        int n_part = 0;
        NEF_TRY(run_pass<T>(p, p->pass[l], y, mbits, factors, w, u, st, lp, &n_part));
        if (lp) NEF_CUDA(launch_loss_append(p->loss_part, n_part, trace, p->loss_count, p->loss_out, st));
    }
    if (only_l < 0 && !loss) p->sweep_launches[mbits ? 1 : 0] = (int)(kernel_launches() - c0);
    return NEF_OK;
}

// Loss of the current factors without an update: the fused kernel of the first
// viewable pass with its partial products discarded (or the unfused weights).
template <typename T>
nef_status loss_pass(nef_plan_t p, const T* y, const uint32_t* mbits, void* const* factors, const WeightSpec& w,
                     const LossSpec& L, cudaStream_t st, int* n_part);

nef_status ensure_capture_stream(nef_plan_t p) {
    if (p->cap_stream) return NEF_OK;
    NEF_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    NEF_CUDA(cudaStreamCreateWithFlags(&p->body_stream, cudaStreamNonBlocking));
    NEF_CUDA(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    NEF_CUDA(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    return NEF_OK;
}

// A fit of Algorithm 1: `iters` sweeps (or the single update only_l), with the
// optional stopping rules of App. B evaluated on the device (tol on the training
// loss, val_patience on the loss over the validation mask).
template <typename T>
nef_status fit_impl(nef_plan_t p, const void* Y, const uint8_t* mask, void* const* factors,
                    double al, double be, int iters, int only_l, double tol = 0.0, double* trace = nullptr,
                    const uint8_t* val_mask = nullptr, int patience = 0, double* val_trace = nullptr) {
    cudaStream_t st = static_cast<cudaStream_t>(p->opt.stream);
    const uint32_t* mbits = nullptr;
    p->last_sweeps = 0;
    p->sweeps_on_device = false;
    if (p->opt.loss != NEF_LOSS_AB) al = be = 0.0;  // ignored by the likelihood families
    NEF_TRY(prologue<T>(p, Y, mask, factors, st, &mbits));
    const Specs sp = specs_of(p, al, be);
    const WeightSpec& w = sp.w;
    const UpdateSpec& u = sp.u;
    const LossSpec& L = sp.L;
    const bool want_val = only_l < 0 && val_mask != nullptr && (patience > 0 || val_trace != nullptr);
    const bool ctl = only_l < 0 && (tol > 0.0 || (want_val && patience > 0));
    const bool want_loss = only_l < 0 && (trace != nullptr || tol > 0.0);
    const LossSpec* lp = want_loss ? &L : nullptr;
    const T* y = static_cast<const T*>(Y);
    if (iters <= 0) return NEF_OK;
    NEF_TRY(init_sources<T>(p, factors, st));
    if (want_loss) NEF_CUDA(cudaMemsetAsync(p->loss_count, 0, sizeof(int), st));
    // V[k]: the loss over the validation entries after k sweeps
    auto val_pass = [&](cudaStream_t s) -> nef_status {
        int n_part = 0;
        NEF_TRY(loss_pass<T>(p, y, p->val_bits, factors, w, L, s, &n_part));
        NEF_CUDA(launch_loss_append(p->loss_part, n_part, val_trace, p->val_count, p->val_out, s));
        return NEF_OK;
    };
    if (want_val) {
        if (!p->val_bits) NEF_CUDA(cudaMalloc(&p->val_bits, ((p->md.N + 31) / 32 + 1) * sizeof(uint32_t)));
        NEF_CUDA(launch_pack_mask(val_mask, p->md.N, p->val_bits, st));
        NEF_CUDA(cudaMemsetAsync(p->val_count, 0, sizeof(int), st));
        NEF_TRY(val_pass(st));
    }
    if (ctl) {
        FitCtlState h{};
        h.iters = iters;
        h.cont = 1;
        h.patience = want_val ? patience : 0;
        h.tol = tol;
        NEF_CUDA(cudaMemcpyAsync(p->ctl, &h, sizeof(h), cudaMemcpyHostToDevice, st));
        if (want_val) NEF_CUDA(launch_fit_check(p->ctl, nullptr, p->val_out, 0, 0, 1, st));
    }
    // one sweep, the validation loss after it and the stopping rules (set_handle:
    // the loop's conditional handle, inside the graph body)
    auto iteration = [&](cudaStream_t s, bool in_graph, cudaGraphConditionalHandle hnd) -> nef_status {
        NEF_TRY(sweep_once<T>(p, y, mbits, factors, w, u, lp, trace, in_graph ? -1 : only_l, s));
        if (want_val) NEF_TRY(val_pass(s));
        if (ctl)
            NEF_CUDA(launch_fit_check(p->ctl, want_loss ? p->loss_out : nullptr, want_val ? p->val_out : nullptr,
                                      hnd, in_graph ? 1 : 0, 0, s));
        return NEF_OK;
    };
    // sweep 1 runs directly (it also settles which contracted operands each pass rebuilds)
    NEF_TRY(iteration(st, false, 0));
    int done = 1;
    const bool graph = !p->opt.eager && !p->opt.profile && only_l < 0 && iters >= (ctl ? 2 : 3);
    if (done < iters) {
        if (graph) {
            // sweeps 2.. replay a captured sweep on the plan's capture stream: a plain
            // fit launches it iters - 1 times; a fit with stopping rules launches once a
            // graph whose conditional (while) node repeats it until the rules end the loop
            NEF_TRY(ensure_capture_stream(p));
            std::vector<const void*> key = {Y, mbits, trace, reinterpret_cast<const void*>((intptr_t)want_loss),
                                            reinterpret_cast<const void*>((intptr_t)ctl),
                                            want_val ? p->val_bits : nullptr, val_trace};
            for (int f = 0; f < p->md.L; ++f) key.push_back(factors[f]);
            cudaGraphExec_t exec = nullptr;
            for (size_t gi = 0; gi < p->graphs.size(); ++gi) {
                const auto& ge = p->graphs[gi];
                if (ge.key == key && ge.ab[0] == al && ge.ab[1] == be) {
                    exec = ge.exec;
                    std::rotate(p->graphs.begin() + gi, p->graphs.begin() + gi + 1, p->graphs.end());
                    break;
                }
            }
            if (!exec) {
                if (p->graphs.size() >= nef_plan_s::kMaxGraphs) {
                    cudaGraphExecDestroy(p->graphs.front().exec);
                    p->graphs.erase(p->graphs.begin());
                }
                cudaGraph_t g = nullptr;
                NEF_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed));
                nef_status rs = NEF_OK;
                if (!ctl) {
                    rs = iteration(p->cap_stream, true, 0);
                } else {
                    rs = [&]() -> nef_status {
                        cudaStreamCaptureStatus cs;
                        cudaGraph_t cg = nullptr;
                        NEF_CUDA(cudaStreamGetCaptureInfo(p->cap_stream, &cs, nullptr, &cg, nullptr, nullptr, nullptr));
                        cudaGraphConditionalHandle hnd = 0;
                        NEF_CUDA(cudaGraphConditionalHandleCreate(&hnd, cg, 0, cudaGraphCondAssignDefault));
                        NEF_CUDA(launch_fit_set_cond(p->ctl, hnd, p->cap_stream));
                        const cudaGraphNode_t* deps = nullptr;
                        size_t n_deps = 0;
                        NEF_CUDA(cudaStreamGetCaptureInfo(p->cap_stream, &cs, nullptr, &cg, &deps, nullptr, &n_deps));
                        cudaGraphNodeParams np{};
                        np.type = cudaGraphNodeTypeConditional;
                        np.conditional.handle = hnd;
                        np.conditional.type = cudaGraphCondTypeWhile;
                        np.conditional.size = 1;
                        cudaGraphNode_t loop = nullptr;
                        NEF_CUDA(cudaGraphAddNode(&loop, cg, deps, nullptr, n_deps, &np));
                        NEF_CUDA(cudaStreamUpdateCaptureDependencies(p->cap_stream, &loop, nullptr, 1,
                                                                     cudaStreamSetCaptureDependencies));
                        NEF_CUDA(cudaStreamBeginCaptureToGraph(p->body_stream, np.conditional.phGraph_out[0], nullptr,
                                                               nullptr, 0, cudaStreamCaptureModeRelaxed));
                        const nef_status rb = iteration(p->body_stream, true, hnd);
                        cudaGraph_t body = nullptr;
                        const cudaError_t eb = cudaStreamEndCapture(p->body_stream, &body);
                        NEF_TRY(rb);
                        NEF_CUDA(eb);
                        return NEF_OK;
                    }();
                }
                const cudaError_t ec = cudaStreamEndCapture(p->cap_stream, &g);
                if (rs != NEF_OK) {
                    if (g) cudaGraphDestroy(g);
                    return rs;
                }
                NEF_CUDA(ec);
                const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
                cudaGraphDestroy(g);
                NEF_CUDA(ei);
                p->graphs.push_back({key, {al, be}, exec});
            }
            NEF_CUDA(cudaEventRecord(p->ev_fork, st));
            NEF_CUDA(cudaStreamWaitEvent(p->cap_stream, p->ev_fork, 0));
            if (ctl) {
                NEF_CUDA(cudaGraphLaunch(exec, p->cap_stream));
            } else {
                for (; done < iters; ++done) NEF_CUDA(cudaGraphLaunch(exec, p->cap_stream));
            }
            NEF_CUDA(cudaEventRecord(p->ev_join, p->cap_stream));
            NEF_CUDA(cudaStreamWaitEvent(st, p->ev_join, 0));
            // the replays changed every factor behind the host bookkeeping: mark the
            // contracted operands stale
            for (int f = 0; f < p->md.L; ++f) p->fac_version[f] = ++p->version_counter;
        } else {
            while (done < iters) {
                if (ctl) {  // the decision of the last check, read back
                    int c = 0;
                    NEF_CUDA(cudaMemcpyAsync(&c, &p->ctl->cont, sizeof(int), cudaMemcpyDeviceToHost, st));
                    NEF_CUDA(cudaStreamSynchronize(st));
                    if (!c) break;
                }
                NEF_TRY(iteration(st, false, 0));
                ++done;
            }
        }
    }
    p->last_sweeps = done;
    p->sweeps_on_device = ctl;
    if (want_loss) {
        // the loss after the last sweep
        int n_part = 0;
        NEF_TRY(loss_pass<T>(p, y, mbits, factors, w, L, st, &n_part));
        NEF_CUDA(launch_loss_append(p->loss_part, n_part, trace, p->loss_count, p->loss_out, st));
    }
    return NEF_OK;
}

template <typename T>
nef_status loss_pass(nef_plan_t p, const T* y, const uint32_t* mbits, void* const* factors, const WeightSpec& w,
                     const LossSpec& L, cudaStream_t st, int* n_part) {
    int vl = -1;
    for (int l = 0; l < p->md.L; ++l)
        if (!p->pass[l].generic) { vl = l; break; }
    if (vl < 0) {
        GenericRecon g{};
        const Model& md = p->md;
        g.n_obs = md.M;
        g.n_let = (int)md.letter.size();
        g.n_fac = md.L;
        for (int x = 0; x < g.n_let; ++x) g.dim[x] = md.dim[x];
        for (int f = 0; f < md.L; ++f) {
            for (int x = 0; x < g.n_let; ++x) g.fst[f][x] = md.fac_stride(f, x);
            g.fac[f] = factors[f];
        }
        g.n = md.N;
        g.n_lat_el = 1;
        for (int x = md.M; x < g.n_let; ++x) g.n_lat_el *= md.dim[x];
        *n_part = (int)std::min<int64_t>((md.N + 255) / 256, p->loss_part_cap / 2);
        NEF_CUDA(launch_generic_weights<T>(g, y, mbits, w, nullptr, nullptr, &L, p->loss_part, *n_part, st));
        return NEF_OK;
    }
    PassPlan& pp = p->pass[vl];
    // the partial products are discarded: the denominator contraction runs only
    // where the instance needs it (masked views, b != 1)
    const int need_den = (mbits || !weights_b_is_one(w)) ? 1 : 0;
    bool use_tc = false;
    if constexpr (sizeof(T) == 4) use_tc = p->prec == NEF_BF16 && tc_view_supported(bind_view(p, pp, true), need_den);
    NEF_TRY(refresh_sources<T>(p, pp, factors, st, use_tc));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (p->opt.profile) NEF_TRY(prof_begin(p, st, &e0, &e1));
    if (use_tc) {
        if constexpr (sizeof(T) == 4) {
            ViewDesc v = bind_view(p, pp, true);
            TcLaunchInfo info{};
            NEF_CUDA(launch_view_tc(reinterpret_cast<const float*>(y), mbits, v, w, need_den, pp.n_split,
                                    static_cast<float*>(buf_ptr(p, B_SPART_N)),
                                    static_cast<float*>(buf_ptr(p, B_SPART_D)), p->tc_err, st, &info, nullptr, &L,
                                    p->loss_part, p->opt.wait_cycles, &pp.tc));
            *n_part = info.n_ctas;
        }
    } else {
        ViewDesc v = bind_view(p, pp, false);
        const int64_t tm = sizeof(T) == 8 ? 32 : 64;
        const int64_t n_rb = (v.rows + tm - 1) / tm;
        int ns = (int)std::max<int64_t>(1, std::min<int64_t>(pp.n_split, p->loss_part_cap / 2 / n_rb));
        NEF_CUDA(launch_view_simt<T>(y, mbits, v, w, 0, ns, nullptr, nullptr, &L, p->loss_part, st, n_part));
    }
    if (p->opt.profile) {
        NEF_CUDA(cudaEventRecord(e1, st));
        p->ev_used.push_back({use_tc ? 0 : 1, {e0, e1}});
    }
    return NEF_OK;
}

template <typename T>
nef_status loss_impl(nef_plan_t p, const void* Y, const uint8_t* mask, void* const* factors,
                     double al, double be, double* out) {
    cudaStream_t st = static_cast<cudaStream_t>(p->opt.stream);
    const uint32_t* mbits = nullptr;
    NEF_TRY(prologue<T>(p, Y, mask, factors, st, &mbits));
    const Specs sp = specs_of(p, al, be);
    const WeightSpec& w = sp.w;
    const LossSpec& L = sp.L;
    const T* y = static_cast<const T*>(Y);
    int n_part = 0;
    // the first factor with a view serves as the reconstruction route
    int vl = -1;
    for (int l = 0; l < p->md.L; ++l)
        if (!p->pass[l].generic) { vl = l; break; }
    if (vl >= 0) {
        // the fused pass of the first viewable factor with its products discarded:
        // tensor cores for NEF_BF16 plans, CUDA cores otherwise
        NEF_TRY(init_sources<T>(p, factors, st));
        NEF_TRY(loss_pass<T>(p, y, mbits, factors, w, L, st, &n_part));
    } else {
        GenericRecon g{};
        const Model& md = p->md;
        g.n_obs = md.M;
        g.n_let = (int)md.letter.size();
        g.n_fac = md.L;
        for (int x = 0; x < g.n_let; ++x) g.dim[x] = md.dim[x];
        for (int f = 0; f < md.L; ++f) {
            for (int x = 0; x < g.n_let; ++x) g.fst[f][x] = md.fac_stride(f, x);
            g.fac[f] = factors[f];
        }
        g.n = md.N;
        g.n_lat_el = 1;
        for (int x = md.M; x < g.n_let; ++x) g.n_lat_el *= md.dim[x];
        n_part = (int)std::min<int64_t>((md.N + 255) / 256, p->loss_part_cap / 2);
        NEF_CUDA(launch_generic_weights<T>(g, y, mbits, w, nullptr, nullptr, &L, p->loss_part, n_part, st));
    }
    NEF_CUDA(launch_sum_f64(p->loss_part, n_part, p->loss_out, st));
    NEF_CUDA(launch_sum_f64(p->loss_part + n_part, n_part, p->loss_out + 1, st));
    NEF_CUDA(cudaMemcpyAsync(out, p->loss_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    NEF_CUDA(cudaStreamSynchronize(st));
    return NEF_OK;
}

nef_status alloc(nef_plan_t p, int id, size_t bytes);

// Key of one pass's tuned split in the cache file: the pass's view (rows, columns,
// bond), precision, weight kind, denominator mode, mask and the SM count.
std::string tune_key(nef_plan_t p, const PassPlan& pp, const WeightSpec& w, int need_den, bool masked) {
    char k[512];
    snprintf(k, sizeof(k), "view rows=%lld c_out=%lld c_in=%lld bond_pad=%lld nq=%d prec=%d ab=%.17g,%.17g lik=%d,%.17g "
             "den=%d mask=%d sm=%lld",
             (long long)pp.view.rows, (long long)pp.view.c_out, (long long)pp.view.c_in, (long long)pp.view.bond_pad,
             (int)pp.Q.size(), p->prec, w.lik ? 0.0 : w.alpha, w.lik ? 0.0 : w.beta, w.lik, w.par, need_den,
             masked ? 1 : 0, (long long)p->n_sm);
    return k;
}

// Grow the split-partial and loss-partial buffers to what the current splits need.
nef_status ensure_split_buffers(nef_plan_t p) {
    int64_t need = 16, loss_ctas = 0;
    for (auto& pp : p->pass) {
        if (pp.generic) continue;
        need = std::max(need, (int64_t)pp.n_split * pp.view.rows * pp.view.bond_pad);
        loss_ctas = std::max<int64_t>(loss_ctas, ((pp.view.rows + 31) / 32) * std::max<int64_t>(2, pp.n_split));
    }
    const size_t bytes = (size_t)need * p->esz;
    for (int id : {(int)B_SPART_N, (int)B_SPART_D}) {
        if (p->buf[id].bytes >= bytes) continue;
        cudaFree(p->buf[id].ptr);
        p->buf[id].ptr = nullptr;
        NEF_TRY(alloc(p, id, bytes));
    }
    if (2 * loss_ctas > p->loss_part_cap) {
        cudaFree(p->loss_part);
        p->loss_part = nullptr;
        p->loss_part_cap = (int)(2 * loss_ctas);
        NEF_CUDA(cudaMalloc(&p->loss_part, p->loss_part_cap * sizeof(double)));
    }
    return NEF_OK;
}

// The tensor-core pass's tile configuration as it runs: the deeper-ring instances
// exist for staged Q rows only, so a gathered pass runs the default ring.
static TcTileConfig tc_tile_normalise(const ViewDesc& v, TcTileConfig c) {
    int qv = 0, qc = 0;
    const bool staged = !c.gather && q_rows_staged(v, kTcTileN, &qv, &qc);
    if (!staged) c.ring = 0;
    return c;
}

static std::string tc_tile_desc(const ViewDesc& v, const TcTileConfig& c0) {
    const TcTileConfig c = tc_tile_normalise(v, c0);
    int qv = 0, qc = 0;
    const bool staged = !c.gather && q_rows_staged(v, kTcTileN, &qv, &qc);
    return std::string(" tile=128x") + std::to_string(kTcTileN) + " ring=" + std::to_string(c.ring) +
           (staged ? " q=staged" : " q=gathered");
}

template <typename T>
nef_status autotune_impl(nef_plan_t p, const void* Y, const uint8_t* mask, void* const* factors, double al,
                         double be, const char* cache_path, int* splits) {
    cudaStream_t st = static_cast<cudaStream_t>(p->opt.stream);
    const uint32_t* mbits = nullptr;
    NEF_TRY(prologue<T>(p, Y, mask, factors, st, &mbits));
    const WeightSpec w = specs_of(p, al, be).w;
    const T* y = static_cast<const T*>(Y);
    std::map<std::string, std::string> cache;  // key -> "split ring gather" 
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char line[1024];
            while (fgets(line, sizeof(line), f)) {
                char* tab = strrchr(line, '\t');
                if (!tab) continue;
                *tab = 0;
                cache[line] = tab + 1;
            }
            fclose(f);
        }
    }
    NEF_TRY(init_sources<T>(p, factors, st));
    cudaEvent_t e0, e1;
    NEF_CUDA(cudaEventCreate(&e0));
    NEF_CUDA(cudaEventCreate(&e1));
    nef_status rs = NEF_OK;
    for (int l = 0; l < p->md.L && rs == NEF_OK; ++l) {
        PassPlan& pp = p->pass[l];
        if (splits) splits[l] = -1;
        if (pp.generic) continue;
        const bool closed = pp.den_closed && weights_b_is_one(w) && mbits == nullptr;
        const int need_den = closed ? 0 : 1;
        bool use_tc = false;
        if constexpr (sizeof(T) == 4) use_tc = p->prec == NEF_BF16 && tc_view_supported(bind_view(p, pp, true), need_den);
        const int64_t tm = use_tc ? 128 : (sizeof(T) == 8 ? 32 : 64);
        const int64_t tn = sizeof(T) == 8 ? 32 : 64;
        const int64_t n_rb = (pp.view.rows + tm - 1) / tm;
        const int64_t tiles = std::max<int64_t>(1, (pp.view.c_out * pp.view.c_in + tn - 1) / tn);
        const std::string key = tune_key(p, pp, w, need_den, mbits != nullptr);
        auto hit = cache.find(key);
        if (hit != cache.end()) {
            int sv = 1, rv = 0, gv = 0;
            sscanf(hit->second.c_str(), "%d %d %d", &sv, &rv, &gv);
            pp.n_split = (int)std::max<int64_t>(1, std::min<int64_t>(sv, tiles));
            pp.tc = use_tc ? tc_tile_normalise(bind_view(p, pp, true), TcTileConfig{rv == 1 ? 1 : 0, gv != 0})
                           : TcTileConfig{0, false};
            if (splits) splits[l] = pp.n_split;
            continue;
        }
        // candidates: 1..4 waves of CTAs over the SMs, and the current choice
        const int64_t per_sm = use_tc ? 1 : 4;
        std::vector<int> cand = {pp.n_split};
        for (int k = 1; k <= 4; ++k) {
            const int64_t c = std::max<int64_t>(1, std::min<int64_t>(tiles, k * p->n_sm * per_sm / n_rb));
            if (std::find(cand.begin(), cand.end(), (int)c) == cand.end()) cand.push_back((int)c);
        }
        const int keep = pp.n_split;
        pp.n_split = *std::max_element(cand.begin(), cand.end());
        if ((rs = ensure_split_buffers(p)) != NEF_OK) break;
        pp.n_split = keep;
        if ((rs = refresh_sources<T>(p, pp, factors, st, use_tc)) != NEF_OK) break;
        T* spn = static_cast<T*>(buf_ptr(p, B_SPART_N));
        T* spd = static_cast<T*>(buf_ptr(p, B_SPART_D));
        double best_ms = 1e300;
        int best = keep;
        TcTileConfig best_tc{0, false};
        // tensor-core passes: the ring-depth configurations of the staged instances and,
        // where the Q rows can be staged, the gathered path too
        std::vector<TcTileConfig> tcs = {TcTileConfig{0, false}};
        if (use_tc) {
            int qv, qc;
            if (q_rows_staged(bind_view(p, pp, true), kTcTileN, &qv, &qc)) {
                tcs.push_back(TcTileConfig{1, false});
                tcs.push_back(TcTileConfig{0, true});
            }
        }
        for (const TcTileConfig& tcc : tcs)
        for (int c : cand) {
            auto launch = [&]() -> cudaError_t {
                if (use_tc) {
                    if constexpr (sizeof(T) == 4) {
                        TcLaunchInfo info{};
                        return launch_view_tc(reinterpret_cast<const float*>(y), mbits, bind_view(p, pp, true), w,
                                              need_den, c, reinterpret_cast<float*>(spn), reinterpret_cast<float*>(spd),
                                              p->tc_err, st, &info, nullptr, nullptr, nullptr, p->opt.wait_cycles, &tcc);
                    }
                    return cudaErrorNotSupported;
                }
                int n_ctas = 0;
                return launch_view_simt<T>(y, mbits, bind_view(p, pp, false), w, need_den, c, spn,
                                           need_den ? spd : nullptr, nullptr, nullptr, st, &n_ctas);
            };
            std::vector<float> ms;
            cudaError_t ce = launch();  // warm-up
            for (int r = 0; r < 3 && ce == cudaSuccess; ++r) {
                cudaEventRecord(e0, st);
                ce = launch();
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                ms.push_back(t);
            }
            if (ce != cudaSuccess) {
                rs = fail(NEF_ECUDA, "autotune launch failed: %s", cudaGetErrorString(ce));
                break;
            }
            std::sort(ms.begin(), ms.end());
            if (ms[1] < best_ms) {
                best_ms = ms[1];
                best = c;
                best_tc = tcc;
            }
        }
        if (rs != NEF_OK) break;
        pp.n_split = best;
        pp.tc = best_tc;
        char v[64];
        snprintf(v, sizeof(v), "%d %d %d", best, best_tc.ring, best_tc.gather ? 1 : 0);
        cache[key] = v;
        if (splits) splits[l] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    NEF_TRY(rs);
    NEF_TRY(ensure_split_buffers(p));
    // the plan description carries the splits and the tensor-core tile configuration
    std::string info;
    for (auto& pp : p->pass) {
        const size_t at = pp.desc.find("splits=");
        if (at != std::string::npos) {
            const size_t end = pp.desc.find(' ', at);
            pp.desc = pp.desc.substr(0, at) + "splits=" + std::to_string(pp.n_split) +
                      (end == std::string::npos ? std::string() : pp.desc.substr(end));
        }
        if (pp.desc.find("kernel=tcgen05") != std::string::npos) {
            const size_t t = pp.desc.find(" tile=");
            if (t != std::string::npos) pp.desc.resize(t);
            pp.desc += tc_tile_desc(bind_view(p, pp, true), pp.tc);
        }
        info += pp.desc + "\n";
    }
    p->info = info;
    for (auto& ge : p->graphs) cudaGraphExecDestroy(ge.exec);  // recorded with the old splits
    p->graphs.clear();
    if (cache_path) {
        FILE* f = fopen(cache_path, "w");
        if (!f) return fail(NEF_EINVAL, "cannot write the autotune cache %s", cache_path);
        for (auto& kv : cache) fprintf(f, "%s\t%s\n", kv.first.c_str(), kv.second.c_str());
        fclose(f);
    }
    return NEF_OK;
}

nef_status alloc(nef_plan_t p, int id, size_t bytes) {
    if ((int)p->buf.size() <= id) p->buf.resize(id + 1);
    if (bytes == 0) bytes = 16;
    void* ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NEF_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    NEF_CUDA(cudaMemset(ptr, 0, bytes));
    p->buf[id].ptr = ptr;
    p->buf[id].bytes = bytes;
    return NEF_OK;
}

void destroy(nef_plan_t p) {
    if (!p) return;
    for (auto& b : p->buf)
        if (b.ptr) cudaFree(b.ptr);
    for (auto* q : p->src_bf16)
        if (q) cudaFree(q);
    if (p->ein_partial) cudaFree(p->ein_partial);
    if (p->mask_bits) cudaFree(p->mask_bits);
    if (p->loss_part) cudaFree(p->loss_part);
    if (p->loss_out) cudaFree(p->loss_out);
    if (p->flag) cudaFree(p->flag);
    if (p->tc_err) cudaFree(p->tc_err);
    if (p->tc_trace) cudaFree(p->tc_trace);
    if (p->loss_count) cudaFree(p->loss_count);
    if (p->ctl) cudaFree(p->ctl);
    if (p->val_out) cudaFree(p->val_out);
    if (p->val_count) cudaFree(p->val_count);
    if (p->val_bits) cudaFree(p->val_bits);
    if (p->body_stream) cudaStreamDestroy(p->body_stream);
    for (auto& ge : p->graphs) cudaGraphExecDestroy(ge.exec);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    for (auto e : p->ev_pool) cudaEventDestroy(e);
    delete p;
}

nef_status build_plan(nef_plan_t p) {
    const Model& md = p->md;
    int next_buf = B_SRC0;
    std::string info;
    for (int l = 0; l < md.L; ++l) {
        PassPlan best;
        bool found = false;
        if (!p->opt.force_generic) {
            for (int s = 0; s < md.M; ++s)
                for (int e = s + 1; e <= md.M; ++e) {
                    bool ok_run = true;
                    for (int x : md.term[l])
                        if (md.is_obs(x) && !(x >= s && x < e)) ok_run = false;
                    if (!ok_run) continue;
                  for (int assign = 0; assign < 64; ++assign)
                  for (int qform = 0; qform < 3; ++qform) {
                    PassPlan cand;
                    int nb = next_buf;
                    if (!plan_view(*p, l, s, e, assign, qform, cand, nb)) continue;
                    bool fits = recipe_fits(cand.P.build) && recipe_fits(cand.epi_num) &&
                                recipe_fits(cand.epi_den);
                    for (auto& q : cand.Q) fits = fits && recipe_fits(q.build);
                    if (cand.den_closed) {
                        for (auto& r : cand.colsum) fits = fits && recipe_fits(r);
                        fits = fits && recipe_fits(cand.den_prod) && recipe_fits(cand.epi_den_closed);
                    }
                    if (!fits) continue;
                    if (!found || cand.cost < best.cost) {
                        best = cand;
                        found = true;
                    }
                  }
                }
        }
        if (found) {
            // renumber the source buffers of the chosen candidate
            int remap_base = next_buf;
            auto renum = [&](SourcePlan& sp) {
                int nb = remap_base++;
                sp.buf = nb;
                sp.build.out_index = nb;
            };
            std::vector<int> old_ids;
            old_ids.push_back(best.P.buf);
            for (auto& q : best.Q) old_ids.push_back(q.buf);
            renum(best.P);
            for (auto& q : best.Q) renum(q);
            for (size_t k = 0; k < best.colsum.size(); ++k) best.colsum[k].ops[0].index = best.Q[k].buf;
            next_buf = remap_base;
            (void)old_ids;
        } else {
            plan_generic(*p, l, best);
            if (!recipe_fits(best.gen_num))
                return fail(NEF_EUNSUPPORTED, "factor %d: contraction too large for the generic path", l);
        }
        if (!best.generic) {
            bool tc = false;
            ViewDesc vv = best.view;
            if (p->prec == NEF_BF16) {
                vv.P.nsrc = 1;
                vv.P.src[0] = best.P.desc;
                vv.Q.nsrc = (int)best.Q.size();
                for (size_t k = 0; k < best.Q.size(); ++k) vv.Q.src[k] = best.Q[k].desc;
                tc = tc_view_supported(vv, 1);
            }
            best.desc += tc ? " kernel=tcgen05" : (p->prec == NEF_FP64 ? " kernel=simt-fp64" : " kernel=simt-fp32");
            if (tc) best.desc += tc_tile_desc(vv, best.tc);
        }
        info += best.desc + "\n";
        p->pass.push_back(best);
    }
    p->info = info;
    // ---- operand bookkeeping: relabelled copies of one factor are kept current by
    // that factor's update; contracted operands are rebuilt when a factor they read changed
    p->mirrors_of.assign(md.L, {});
    p->fac_version.assign(md.L, 0);
    int next_cs = B_CS0;
    for (int pi = 0; pi < (int)p->pass.size(); ++pi) {
        PassPlan& pp = p->pass[pi];
        if (pp.generic) continue;
        for (int k = -1; k < (int)pp.Q.size(); ++k) {
            SourcePlan& sp = source_ref(pp, k);
            const EinRecipe& r = sp.build;
            sp.deps.clear();
            for (auto& o : r.ops)
                if (o.kind == 0) sp.deps.push_back(o.index);
            sp.copy_of = -1;
            if (r.ops.size() == 1 && r.ops[0].kind == 0 && r.free_let.empty()) {
                const int f = r.ops[0].index;
                bool perm = r.out_let.size() == md.term[f].size();
                for (int x : r.out_let) perm = perm && md.fac_has(f, x);
                if (perm && p->mirrors_of[f].size() < (size_t)kMaxMirror) {
                    sp.copy_of = f;
                    p->mirrors_of[f].push_back({pi, k});
                }
            }
            if (k >= 0 && pp.den_closed && sp.copy_of >= 0) sp.cs_buf = next_cs++;
        }
        // a closed-form denominator needs the column sums of every column-side operand
        if (pp.den_closed)
            for (auto& q : pp.Q)
                if (q.cs_buf < 0) pp.den_closed = false;
        const bool id_num = pp.epi_num.ops.size() == 1 && pp.epi_num.free_let.empty() &&
                            pp.epi_num.out_let.size() <= (size_t)kMaxFacLet;
        const bool id_den = pp.epi_den.ops.size() == 1 && pp.epi_den.free_let.empty();
        const bool id_closed = !pp.den_closed ||
                               (pp.epi_den_closed.ops.size() == 1 && pp.epi_den_closed.free_let.empty());
        pp.finish_identity = id_num && id_den && id_closed && md.term[pp.l].size() <= (size_t)kMaxFacLet;
        pp.dual_epi = dual_pair(pp.epi_num, pp.epi_den);
        // every letter of the epilogue moves its S operand: each S element is read once,
        // so the split partials can be summed where they are read
        pp.epi_s_once = !pp.epi_num.ops.empty() && pp.epi_num.ops[0].kind == 1;
        for (int x : pp.epi_num.out_let) pp.epi_s_once = pp.epi_s_once && pp.epi_num.ops[0].st[x] != 0;
        for (int x : pp.epi_num.free_let) pp.epi_s_once = pp.epi_s_once && pp.epi_num.ops[0].st[x] != 0;
        p->max_ld = std::max<int64_t>(p->max_ld, pp.view.bond_pad);
    }
    // ---- contracted operands with one recipe (the same product of the same factors in
    // the same layout, e.g. the column-side operand of several passes of one view) share
    // the first one's buffer, so a sweep builds each of them once per change of its factors
    for (int pi = 0; pi < (int)p->pass.size(); ++pi) {
        PassPlan& pp = p->pass[pi];
        if (pp.generic) continue;
        for (int k = -1; k < (int)pp.Q.size(); ++k) {
            SourcePlan& sp = source_ref(pp, k);
            if (sp.copy_of >= 0) continue;
            bool done = false;
            for (int pj = 0; pj <= pi && !done; ++pj) {
                PassPlan& po = p->pass[pj];
                if (po.generic || po.view.bond_pad != pp.view.bond_pad) continue;
                for (int k2 = -1; k2 < (int)po.Q.size() && !done; ++k2) {
                    if (pj == pi && k2 >= k) break;
                    const SourcePlan& so = source_ref(po, k2);
                    if (so.copy_of >= 0 || so.shared || so.n_rows != sp.n_rows || so.desc.ld != sp.desc.ld ||
                        !same_recipe(so.build, sp.build))
                        continue;
                    sp.buf = so.buf;
                    sp.build.out_index = so.buf;
                    sp.shared = true;
                    done = true;
                }
            }
        }
    }
    // ---- workspace
    size_t es = p->esz;
    int64_t max_fac = 1, max_s = 16, max_part = 16;
    bool any_generic = false;
    int64_t max_bond_pad = 16;
    for (int l = 0; l < md.L; ++l) max_fac = std::max(max_fac, md.fac_size(l));
    for (auto& pp : p->pass) {
        if (pp.generic) { any_generic = true; continue; }
        max_s = std::max(max_s, pp.view.rows * pp.view.bond_pad);
        max_part = std::max(max_part, (int64_t)pp.n_split * pp.view.rows * pp.view.bond_pad);
        max_bond_pad = std::max<int64_t>(max_bond_pad, pp.view.bond_pad);
    }
    NEF_TRY(alloc(p, B_NUM, max_fac * es));
    NEF_TRY(alloc(p, B_DEN, max_fac * es));
    NEF_TRY(alloc(p, B_SNUM, max_s * es));
    NEF_TRY(alloc(p, B_SDEN, max_s * es));
    NEF_TRY(alloc(p, B_SPART_N, max_part * es));
    NEF_TRY(alloc(p, B_SPART_D, max_part * es));
    NEF_TRY(alloc(p, B_DENVEC, max_bond_pad * es));
    for (int k = 0; k < kMaxSrc; ++k) NEF_TRY(alloc(p, B_COLSUM0 + k, max_bond_pad * es));
    if (any_generic) {
        NEF_TRY(alloc(p, B_WA, md.N * es));
        NEF_TRY(alloc(p, B_WB, md.N * es));
    }
    for (auto& pp : p->pass) {
        if (pp.generic) continue;
        for (auto& q : pp.Q)
            if (q.cs_buf >= 0) NEF_TRY(alloc(p, q.cs_buf, (size_t)pp.view.bond_pad * es));
    }
    p->src_bf16.assign(next_buf + 1, nullptr);
    p->src_built.assign(next_buf + 1, {});
    for (auto& pp : p->pass) {
        if (pp.generic) continue;
        std::vector<SourcePlan*> srcs{&pp.P};
        for (auto& q : pp.Q) srcs.push_back(&q);
        for (auto* sp : srcs) {
            if (sp->shared) continue;  // the buffer of the operand it repeats
            size_t n = (size_t)sp->n_rows * pp.view.bond_pad;
            NEF_TRY(alloc(p, sp->buf, n * es));
            if (p->prec == NEF_BF16) {
                void* q = nullptr;
                if (cudaMalloc(&q, n * 2) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(NEF_ENOMEM, "cudaMalloc of a BF16 operand failed");
                }
                NEF_CUDA(cudaMemset(q, 0, n * 2));
                p->src_bf16[sp->buf] = static_cast<uint16_t*>(q);
            }
        }
    }
    p->ein_partial_cap = 1 << 22;
    NEF_CUDA(cudaMalloc(&p->ein_partial, p->ein_partial_cap * es));
    NEF_CUDA(cudaMalloc(&p->mask_bits, ((md.N + 31) / 32 + 1) * sizeof(uint32_t)));
    // loss partials: two doubles per CTA of the loss pass (view of the first viewable factor)
    // (and the update passes that also sum the loss: one CTA per row block and split)
    int64_t loss_ctas = 152 * 64;
    for (auto& pp : p->pass) {
        if (pp.generic) continue;
        loss_ctas = std::max<int64_t>(loss_ctas, ((pp.view.rows + 31) / 32) * std::max<int64_t>(2, pp.n_split));
    }
    p->loss_part_cap = (int)(2 * loss_ctas);
    NEF_CUDA(cudaMalloc(&p->loss_part, p->loss_part_cap * sizeof(double)));
    NEF_CUDA(cudaMalloc(&p->loss_out, 2 * sizeof(double)));
    NEF_CUDA(cudaMalloc(&p->loss_count, sizeof(int)));
    NEF_CUDA(cudaMemset(p->loss_count, 0, sizeof(int)));
    NEF_CUDA(cudaMalloc(&p->ctl, sizeof(FitCtlState)));
    NEF_CUDA(cudaMalloc(&p->val_out, 2 * sizeof(double)));
    NEF_CUDA(cudaMalloc(&p->val_count, sizeof(int)));
    NEF_CUDA(cudaMalloc(&p->flag, sizeof(int)));
    NEF_CUDA(cudaMalloc(&p->tc_err, sizeof(int)));
    NEF_CUDA(cudaMemset(p->tc_err, 0, sizeof(int)));
    if (p->opt.profile >= 2) {
        NEF_CUDA(cudaMalloc(&p->tc_trace, 32 * sizeof(unsigned long long)));
        NEF_CUDA(cudaMemset(p->tc_trace, 0, 32 * sizeof(unsigned long long)));
    }
    return NEF_OK;
}

}  // namespace

static_assert((int)NEF_LOSS_AB == (int)LIK_NONE && (int)NEF_LOSS_NEGBIN == (int)LIK_NEGBIN &&
                  (int)NEF_LOSS_BINOMIAL == (int)LIK_BINOMIAL && (int)NEF_LOSS_JS == (int)LIK_JS,
              "loss families of the ABI and of the kernels");

// ================================================================== C ABI
extern "C" {

void nef_default_options(nef_options* opt) {
    if (!opt) return;
    opt->precision = NEF_FP32;
    opt->eps = 1e-10;
    opt->check_data = 0;
    opt->force_generic = 0;
    opt->profile = 0;
    opt->stream = nullptr;
    opt->tol = 0.0;
    opt->loss_trace = nullptr;
    opt->eager = 0;
    opt->loss = NEF_LOSS_AB;
    opt->loss_par = 0.0;
    opt->wait_cycles = 0;
    opt->batch_tiles = 0;
}

nef_status nef_plan(const char* model_str, const int64_t* shapes, int n_obs, const int64_t* ranks,
                    int n_lat, const nef_options* opt, nef_plan_t* out) {
    g_err.clear();
    if (!out) return fail(NEF_EINVAL, "out is NULL");
    *out = nullptr;
    nef_plan_t p = new nef_plan_s();
    if (opt) p->opt = *opt;
    else nef_default_options(&p->opt);
    if (p->opt.precision != NEF_FP32 && p->opt.precision != NEF_BF16 && p->opt.precision != NEF_FP64) {
        delete p;
        return fail(NEF_EINVAL, "unknown precision %d", p->opt.precision);
    }
    if (!(p->opt.eps >= 0.0) || !std::isfinite(p->opt.eps)) {
        delete p;
        return fail(NEF_EINVAL, "eps must be finite and >= 0");
    }
    if (p->opt.loss != NEF_LOSS_AB) {
        const char* msg = loss_args_error(p->opt.loss, 1.0, 0.0, p->opt.loss_par, nullptr);
        if (msg) {
            delete p;
            return fail(NEF_EINVAL, "%s", msg);
        }
    }
    if (p->opt.wait_cycles < 0) {
        delete p;
        return fail(NEF_EINVAL, "wait_cycles must be >= 0");
    }
    p->prec = p->opt.precision;
    p->esz = p->prec == NEF_FP64 ? 8 : 4;
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            p->n_sm = nsm;
        cudaGetLastError();
    }
    nef_status s = parse_model(model_str, shapes, n_obs, ranks, n_lat, p->md);
    if (s != NEF_OK) {
        delete p;
        return s;
    }
    s = build_plan(p);
    if (s != NEF_OK) {
        destroy(p);
        return s;
    }
    *out = p;
    return NEF_OK;
}

void nef_plan_destroy(nef_plan_t plan) { destroy(plan); }

nef_status nef_fit_ctl(nef_plan_t plan, const void* Y, const uint8_t* mask, void* const* factors, double alpha,
                       double beta, int iters, const nef_fit_control* ctl, int* sweeps) {
    g_err.clear();
    if (sweeps) *sweeps = 0;
    if (!plan) return fail(NEF_EINVAL, "plan is NULL");
    if (iters < 0) return fail(NEF_EINVAL, "iters must be >= 0");
    nef_fit_control c{};
    if (ctl) c = *ctl;
    if (!(c.tol >= 0.0)) return fail(NEF_EINVAL, "tol must be >= 0");
    if (c.val_patience < 0) return fail(NEF_EINVAL, "val_patience must be >= 0");
    if (!c.val_mask && (c.val_patience > 0 || c.val_trace))
        return fail(NEF_EINVAL, "val_patience and val_trace need val_mask");
    NEF_TRY(check_ab(plan, alpha, beta));
    const nef_status r =
        plan->prec == NEF_FP64
            ? fit_impl<double>(plan, Y, mask, factors, alpha, beta, iters, -1, c.tol, c.loss_trace, c.val_mask,
                               c.val_patience, c.val_trace)
            : fit_impl<float>(plan, Y, mask, factors, alpha, beta, iters, -1, c.tol, c.loss_trace, c.val_mask,
                              c.val_patience, c.val_trace);
    if (sweeps && r == NEF_OK) *sweeps = nef_plan_sweeps(plan);
    return r;
}

nef_status nef_fit_ex(nef_plan_t plan, const void* Y, const uint8_t* mask, void* const* factors, double alpha,
                      double beta, int iters, double tol, double* loss_trace, int* sweeps) {
    nef_fit_control c{};
    c.tol = tol;
    c.loss_trace = loss_trace;
    return nef_fit_ctl(plan, Y, mask, factors, alpha, beta, iters, &c, sweeps);
}

nef_status nef_fit(nef_plan_t plan, const void* Y, const uint8_t* mask, void* const* factors,
                   double alpha, double beta, int iters) {
    if (!plan) {
        g_err = "plan is NULL";
        return NEF_EINVAL;
    }
    return nef_fit_ex(plan, Y, mask, factors, alpha, beta, iters, plan->opt.tol, plan->opt.loss_trace, nullptr);
}

int nef_plan_sweeps(nef_plan_t plan) {
    if (!plan) return 0;
    if (plan->sweeps_on_device) {
        cudaStream_t st = static_cast<cudaStream_t>(plan->opt.stream);
        int d = 0;
        if (cudaMemcpyAsync(&d, &plan->ctl->done, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess) {
            plan->last_sweeps = d;
            plan->sweeps_on_device = false;
        } else {
            cudaGetLastError();
        }
    }
    return plan->last_sweeps;
}

nef_status nef_plan_autotune(nef_plan_t plan, const void* Y, const uint8_t* mask, void* const* factors,
                             double alpha, double beta, const char* cache_path, int* splits) {
    g_err.clear();
    if (!plan) return fail(NEF_EINVAL, "plan is NULL");
    NEF_TRY(check_ab(plan, alpha, beta));
    if (plan->prec == NEF_FP64)
        return autotune_impl<double>(plan, Y, mask, factors, alpha, beta, cache_path, splits);
    return autotune_impl<float>(plan, Y, mask, factors, alpha, beta, cache_path, splits);
}

nef_status nef_update(nef_plan_t plan, int l, const void* Y, const uint8_t* mask, void* const* factors,
                      double alpha, double beta) {
    g_err.clear();
    if (!plan) return fail(NEF_EINVAL, "plan is NULL");
    if (l < 0 || l >= plan->md.L) return fail(NEF_EINVAL, "factor index %d out of range", l);
    NEF_TRY(check_ab(plan, alpha, beta));
    if (plan->prec == NEF_FP64) return fit_impl<double>(plan, Y, mask, factors, alpha, beta, 1, l);
    return fit_impl<float>(plan, Y, mask, factors, alpha, beta, 1, l);
}

nef_status nef_numden(nef_plan_t plan, int l, const void* Y, const uint8_t* mask, void* const* factors,
                      double alpha, double beta, void* num, void* den) {
    g_err.clear();
    if (!plan) return fail(NEF_EINVAL, "plan is NULL");
    if (l < 0 || l >= plan->md.L) return fail(NEF_EINVAL, "factor index %d out of range", l);
    if (!num || !den) return fail(NEF_EINVAL, "num/den is NULL");
    NEF_TRY(check_ab(plan, alpha, beta));
    if (plan->prec == NEF_FP64)
        return numden_impl<double>(plan, l, Y, mask, factors, alpha, beta, static_cast<double*>(num),
                                   static_cast<double*>(den));
    return numden_impl<float>(plan, l, Y, mask, factors, alpha, beta, static_cast<float*>(num),
                              static_cast<float*>(den));
}

nef_status nef_apply_update(nef_plan_t plan, int l, void* const* factors, const void* num, const void* den,
                            double alpha, double beta) {
    g_err.clear();
    if (!plan) return fail(NEF_EINVAL, "plan is NULL");
    if (l < 0 || l >= plan->md.L) return fail(NEF_EINVAL, "factor index %d out of range", l);
    if (!num || !den) return fail(NEF_EINVAL, "num/den is NULL");
    NEF_TRY(check_ab(plan, alpha, beta));
    if (plan->prec == NEF_FP64)
        return numden_impl<double>(plan, l, nullptr, nullptr, factors, alpha, beta, nullptr, nullptr,
                                   static_cast<const double*>(num), static_cast<const double*>(den));
    return numden_impl<float>(plan, l, nullptr, nullptr, factors, alpha, beta, nullptr, nullptr,
                              static_cast<const float*>(num), static_cast<const float*>(den));
}

nef_status nef_loss(nef_plan_t plan, const void* Y, const uint8_t* mask, void* const* factors,
                    double alpha, double beta, double* out) {
    g_err.clear();
    if (!plan) return fail(NEF_EINVAL, "plan is NULL");
    if (!out) return fail(NEF_EINVAL, "out is NULL");
    NEF_TRY(check_ab(plan, alpha, beta));
    if (plan->prec == NEF_FP64) return loss_impl<double>(plan, Y, mask, factors, alpha, beta, out);
    return loss_impl<float>(plan, Y, mask, factors, alpha, beta, out);
}

int nef_plan_info(nef_plan_t plan, char* buf, int cap) {
    if (!plan) return 0;
    int n = (int)plan->info.size();
    if (buf && cap > 0) {
        int c = std::min(n, cap - 1);
        memcpy(buf, plan->info.data(), c);
        buf[c] = 0;
    }
    return n + 1;
}

int nef_plan_launches(nef_plan_t plan, int has_mask) {
    if (!plan) return 0;
    // one sweep inside a nef_fit call (the per-call start-up is not counted): as counted
    // when a sweep was last recorded or run, else the planner's estimate
    if (plan->sweep_launches[has_mask ? 1 : 0] > 0) return plan->sweep_launches[has_mask ? 1 : 0];
    int total = 0;
    for (auto& pp : plan->pass) {
        if (pp.generic) {
            total += 1 + 2 + 2 + 1 + 1;
            continue;
        }
        int n = 0;
        for (int k = -1; k < (int)pp.Q.size(); ++k) {
            const SourcePlan& sp = k < 0 ? pp.P : pp.Q[k];
            if (sp.copy_of < 0) n += 2 + (plan->prec == NEF_BF16 ? 1 : 0);  // rebuild (+ BF16 copy)
        }
        n += 1;  // fused pass
        const bool closed = pp.den_closed && !has_mask;
        if (pp.finish_identity) {
            n += 1;
        } else {
            n += closed ? 1 : 2;                                // split reductions
            n += 2;                                             // epilogue num
            n += closed ? 2 * ((int)pp.colsum.size() + 2) : 2;  // den
            n += 1;                                             // update
        }
        bool any_cs = false;
        for (auto& ps : plan->mirrors_of[pp.l]) {
            const SourcePlan& sp = ps.second < 0 ? plan->pass[ps.first].P : plan->pass[ps.first].Q[ps.second];
            any_cs = any_cs || sp.cs_buf >= 0;
        }
        n += any_cs ? 1 : 0;                                    // column sums
        total += n;
    }
    return total;
}

nef_status nef_plan_profile(nef_plan_t plan, double* ms, int* count, int reset) {
    g_err.clear();
    if (!plan || !ms || !count) return fail(NEF_EINVAL, "NULL argument");
    if (!plan->opt.profile) return fail(NEF_EINVAL, "plan was created without opt.profile");
    cudaStream_t st = static_cast<cudaStream_t>(plan->opt.stream);
    NEF_CUDA(cudaStreamSynchronize(st));
    ms[0] = ms[1] = 0.0;
    count[0] = count[1] = 0;
    for (auto& u : plan->ev_used) {
        float t = 0.f;
        NEF_CUDA(cudaEventElapsedTime(&t, u.second.first, u.second.second));
        ms[u.first] += t;
        count[u.first] += 1;
    }
    if (reset) {
        plan->ev_used.clear();
        plan->ev_next = 0;
    }
    return NEF_OK;
}

int nef_tc_trace(nef_plan_t plan, unsigned long long* out, int reset) {
    if (!plan || !out || !plan->tc_trace) return 1;
    cudaStream_t st = static_cast<cudaStream_t>(plan->opt.stream);
    if (cudaMemcpyAsync(out, plan->tc_trace, 32 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return 5;
    if (reset) {
        if (cudaMemsetAsync(plan->tc_trace, 0, 32 * sizeof(unsigned long long), st) != cudaSuccess) return 5;
    }
    return 0;
}

nef_status nef_check(nef_plan_t plan) {
    g_err.clear();
    if (!plan) return fail(NEF_EINVAL, "plan is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(plan->opt.stream);
    int h = 0;
    NEF_CUDA(cudaMemcpyAsync(&h, plan->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    NEF_CUDA(cudaStreamSynchronize(st));
    if (h) {
        NEF_CUDA(cudaMemsetAsync(plan->tc_err, 0, sizeof(int), st));
        NEF_CUDA(cudaStreamSynchronize(st));
        return fail(NEF_ETIMEOUT, "a bounded wait in the tensor-core pass gave up (site %d)", h);
    }
    return NEF_OK;
}

const char* nef_last_error(void) { return g_err.c_str(); }

}  // extern "C"
