// nef_internal.h -- descriptors shared by the host planner and the CUDA kernels.
//
// A factor update (one inner step of Algorithm 1) runs as a "view pass":
// Y is viewed as a matrix Y[row, col] where the rows are a contiguous run of
// observed letters containing the updated factor's observed letters and the
// columns are the remaining observed letters:
//     element (row, col = co*c_in + ci) lives at  co*rows*c_in + row*c_in + ci.
// The reconstruction factorises through a set of latent "bond" letters,
//     yhat[row, col] = sum_b P[row, b] * Q[col, b]                  (Eq. 2.1)
// and the numerator of Eq. 3.6-3.8 is  S_a[row, b] = sum_col W_a[row,col] Q[col,b]
// followed by a small "epilogue" einsum of S_a with the other row-side factors.
// P and Q are Hadamard products of rows gathered from canonical [n x ld]
// operand matrices ("sources").
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nef {

constexpr int kMaxLet = 26;
constexpr int kMaxFac = 16;
constexpr int kMaxSrc = 4;    // gathered sources per operand side
constexpr int kMaxTerm = 3;   // index terms per source
constexpr int kTcTileN = 64;  // columns per tile of the tensor-core pass
constexpr int kMaxEinOps = 8; // operands of a small einsum
constexpr int kMaxEinLet = 12;

// Specialised evaluation of x^e for the weights of App. B.
enum PowCode : int {
    POW_ONE = 0,      // x^0
    POW_ID = 1,       // x^1
    POW_RCP = 2,      // x^-1
    POW_RSQRT = 3,    // x^-1/2
    POW_SQRT = 4,     // x^1/2
    POW_SQ = 5,       // x^2
    POW_RSQRT3 = 6,   // x^-3/2
    POW_GENERAL = 7,  // exp2(e * log2 x)
    POW_RCP2 = 8      // x^-2
};

// Likelihood families of App. B outside the (alpha,beta) family (nef.h NEF_LOSS_*).
enum LikKind : int { LIK_NONE = 0, LIK_NEGBIN = 1, LIK_BINOMIAL = 2, LIK_JS = 3 };

// Weights of App. B: wa = M * y^alpha * yhat^(beta-1), wb = M * yhat^(alpha+beta-1)
// (alpha != 0), or wa = M * log(y/yhat), wb = M (alpha = 0, beta = 1).  With lik
// set, the likelihood family's a and b instead (negative binomial: y/yhat and
// (par+y)/(par+yhat); binomial on odds: y/yhat and par/(1+yhat); Jensen-Shannon:
// log((y+yhat)/(2 yhat)) and 1), par being phi or the trial count.
struct WeightSpec {
    int log_case;       // 1 for (alpha, beta) = (0, 1)
    int y_code;         // PowCode of y^alpha
    int a_code;         // PowCode of yhat^(beta-1)
    int b_code;         // PowCode of yhat^(alpha+beta-1); POW_ONE whenever b == 1
    double alpha, beta;
    double e_y, e_a, e_b;  // exponents (used by POW_GENERAL)
    int lik;            // LikKind
    double par;         // phi (negative binomial) or trials n (binomial)
};

// Loss cases of App. B.
struct LossSpec {
    int kase;           // 0 generic, 1 beta=0, 2 alpha=-beta, 3 alpha=0, 4 alpha=beta=0
    double alpha, beta;
    int lik;            // LikKind: a likelihood family's D instead of D_{alpha,beta}
    double par;
};

// Update of Eq. 3.4: theta <- max(eps, theta * ginv(num/den)).
struct UpdateSpec {
    int log_case;       // g = log -> exp
    int eta_code;       // PowCode of z^eta
    double eta;
    double eps;
};

struct SrcDesc {
    const void* ptr;              // canonical [n x ld] matrix (operand element type)
    int64_t ld;                   // elements per row (= bond_pad)
    int nterm;
    int64_t div[kMaxTerm], mod[kMaxTerm], mul[kMaxTerm];  // row = sum ((i/div)%mod)*mul
};

struct SideDesc {
    int nsrc;
    SrcDesc src[kMaxSrc];
};

struct ViewDesc {
    int64_t c_out, rows, c_in;    // Y viewed as [c_out][rows][c_in]
    int bond, bond_pad;           // real and padded bond size
    SideDesc P, Q;
};

// Small generic einsum: out[o] = sum over free combos of prod_k op_k[...].
// Letters are compact ids 0..n_let-1: out letters first, then free letters.
struct EinDesc {
    int n_ops;
    const void* op[kMaxEinOps];
    int64_t ost[kMaxEinOps][kMaxEinLet];  // per-letter strides of each operand (0 = absent)
    int n_out, n_free;
    int64_t dim[kMaxEinLet];
    int64_t out_st[kMaxEinLet];           // destination strides for the out letters
    int64_t n_out_el, n_free_el;
    void* out;
    int accumulate;                        // 1: out += result, 0: out = result
    // FP32 only, with accumulate = 0: also write the BF16 copy of the result here (same
    // offsets) and store the FP32 result rounded to it (round to nearest even)
    uint16_t* out16;
    // optional second contraction of the same shape that reads op0b in place of op[0]
    // and writes outb (the two share every other operand read)
    const void* op0b;
    void* outb;
    // op0_splits > 1: operand 0 (and op0b) is the sum of that many partial copies
    // op0_split_stride elements apart (read in split order at every access)
    int op0_splits;
    int64_t op0_split_stride;
};

// ----------------------------------------------------- finishing a pass
constexpr int kMaxMirror = 8;
constexpr int kMaxFacLet = 8;

// Canonical operand copies of one factor that its update writes directly
// (element e of the factor, decoded over the factor's letters in term order,
// goes to offset sum_q idx[q] * st[k][q] of copy k).
struct MirrorDesc {
    int n;
    void* p32[kMaxMirror];          // copy in the plan's element type
    uint16_t* p16[kMaxMirror];      // BF16 copy of the same layout, or null
    int64_t st[kMaxMirror][kMaxFacLet];
};

// Split reduction + denominator + update (Eq. 3.4) + copies, for passes whose
// epilogue is a relabelling of S[rows][bond_pad] onto the factor's layout.
struct FinishDesc {
    int nlet;
    int64_t dim[kMaxFacLet];        // the factor's letter sizes, term order
    int64_t s_st[kMaxFacLet];       // offset into S per letter
    int64_t b_st[kMaxFacLet];       // offset into the bond vector per letter (closed-form den)
    const void* part_num;           // [n_split][s_size]
    const void* part_den;           // [n_split][s_size], or null: closed-form den
    int n_split;
    int64_t s_size;
    int n_cs;                       // closed-form den = product of these column sums
    const void* cs[kMaxSrc];
    void* theta;
    int64_t n;
    MirrorDesc mir;
};

struct ColsumJob {
    const void* src;                // canonical [n_rows x ld] operand
    int64_t n_rows, ld;
    void* out;                      // [ld] column sums
};
constexpr int kMaxColsumJobs = 16;
struct ColsumDesc {
    int n;
    ColsumJob job[kMaxColsumJobs];
};

template <typename T>
cudaError_t launch_finish(const FinishDesc& d, const UpdateSpec& u, cudaStream_t st);

// Eq. 3.4 applied by the contraction that completes a factor's numerator and
// denominator (the epilogue's last einsum, whose outputs are the factor's elements in
// term order): with num set, the contraction computes den and num is read there;
// otherwise it is the dual form computing num (out) and den (outb).  The updated
// element goes to theta and to the factor's canonical copies.
struct EinUpdate {
    void* theta;
    const void* num;
    int nlet;
    int64_t dim[kMaxFacLet];
    MirrorDesc mir;
    UpdateSpec u;
};

template <typename T>
cudaError_t launch_einsum_update(const EinDesc& d, const EinUpdate& up, T* partial, int64_t partial_cap,
                                 cudaStream_t st);

template <typename T>
cudaError_t launch_update_mirror(T* theta, const T* num, const T* den, int64_t n, const UpdateSpec& u,
                                 int nlet, const int64_t* dim, const MirrorDesc& m, cudaStream_t st);

template <typename T>
cudaError_t launch_mirror_init(const T* theta, int64_t n, int nlet, const int64_t* dim,
                               const MirrorDesc& m, cudaStream_t st);

template <typename T>
cudaError_t launch_colsums(const ColsumDesc& d, int64_t max_ld, cudaStream_t st);

// Message returned by nef_last_error() on this thread.
void set_last_error(const char* msg);

// Specialisation of the App. B weights, loss and update for given (alpha, beta)
// (lik = LIK_NONE) or for a likelihood family with parameter par (alpha, beta
// ignored).
WeightSpec weight_spec(double alpha, double beta, int lik = LIK_NONE, double par = 0.0);
LossSpec loss_spec(double alpha, double beta, int lik = LIK_NONE, double par = 0.0);
UpdateSpec update_spec(double alpha, double beta, double eps, int lik = LIK_NONE);

// Argument check shared by every entry point that takes a loss: returns nullptr
// when (lik, alpha, beta, par) is valid, else a message; *unsupported is set for
// alpha == 0 with beta != 1 (no decomposition, App. B).
const char* loss_args_error(int lik, double alpha, double beta, double par, bool* unsupported);

// True when b(x, y) == 1 for these weights (the closed-form denominator applies).
inline bool weights_b_is_one(const WeightSpec& w) {
    return w.lik == LIK_JS || (w.lik == LIK_NONE && (w.log_case || w.b_code == POW_ONE));
}

// ------------------------------------------------------------- launchers
// All launchers return cudaGetLastError() after enqueueing on `st`.

template <typename T>
cudaError_t launch_einsum(const EinDesc& d, T* partial, int64_t partial_cap, cudaStream_t st);

cudaError_t launch_pack_mask(const uint8_t* mask, int64_t n, uint32_t* bits, cudaStream_t st);

template <typename T>
cudaError_t launch_check_data(const T* y, int64_t n, int* flag, cudaStream_t st);

template <typename T>
cudaError_t launch_view_simt(const T* y, const uint32_t* mbits, const ViewDesc& v,
                             const WeightSpec& w, int need_den, int n_split,
                             T* s_num, T* s_den, const LossSpec* loss, double* loss_part,
                             cudaStream_t st, int* n_ctas_out);

// Kernels this library has launched in this process (a counter kept by the launchers).
long long kernel_launches();

// Both split reductions of a pass (numerator and denominator partials) in one launch.
template <typename T>
cudaError_t launch_reduce_splits2(const T* part_a, const T* part_b, int n_split, int64_t n, T* out_a, T* out_b,
                                  cudaStream_t st);
template <typename T>
cudaError_t launch_reduce_splits(const T* part, int n_split, int64_t n, T* out, cudaStream_t st);

template <typename T>
cudaError_t launch_update(T* theta, const T* num, const T* den, int64_t n, const UpdateSpec& u,
                          cudaStream_t st);

template <typename T>
cudaError_t launch_fill(T* p, int64_t n, T v, cudaStream_t st);

cudaError_t launch_sum_f64(const double* part, int n, double* out, cudaStream_t st);

// Generic (unfused) path: materialise yhat, then W_a, W_b and optionally the loss.
struct GenericRecon {
    int n_obs, n_let, n_fac;
    int64_t dim[kMaxLet];
    int64_t y_st[kMaxLet];                   // strides of Y per observed letter
    int64_t fst[kMaxFac][kMaxLet];           // strides of each factor per letter
    const void* fac[kMaxFac];
    int64_t n, n_lat_el;
};

template <typename T>
cudaError_t launch_generic_weights(const GenericRecon& g, const T* y, const uint32_t* mbits,
                                   const WeightSpec& w, T* wa, T* wb, const LossSpec* loss,
                                   double* loss_part, int n_part, cudaStream_t st);

// tcgen05 path (BF16 operands, FP32 accumulators in TMEM).
struct TcLaunchInfo {
    int n_ctas;
    int smem_bytes;
    int staged;   // 1: Q rows staged by TMA, 0: gathered per tile
    int ring;     // ring-depth configuration launched
};

// Per-pass choices of the tensor-core pass beyond the split (the autotuner's):
// ring-depth configuration 0 or 1 of the staged instances, and gathered Q rows
// even where they could be staged.
struct TcTileConfig {
    int ring;
    bool gather;
};

// BF16 copy dst of src; src is replaced by the same rounded values.
cudaError_t launch_convert_bf16(float* src, int64_t n, uint16_t* dst, cudaStream_t st);

// Tensor-core GEMM C[M x N] (=, or += with accumulate) A[M x K] . B[N x K]^T; A and B
// row-major BF16 (pitches lda, ldb elements, multiples of 8; 16-byte aligned bases),
// C row-major FP32 (pitch ldc).  err: device flag set when a bounded wait gives up.
// n_split > 1 splits K over that many CTAs per tile, with partial tiles in ws
// (n_split * M * ldc floats; too small or null: no split) summed in split order.
cudaError_t launch_gemm_nt(const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* C, int64_t ldc,
                           int M, int N, int K, int accumulate, int* err, cudaStream_t st, float* ws = nullptr,
                           int64_t ws_floats = 0, int n_split = 1);

// Split count for an M x N x K product on n_sm SMs (about one wave of CTAs).
int gemm_splits(int M, int N, int K, int n_sm);

// Fold-in encoder kernels (k_foldin.cu).
cudaError_t launch_fi_features(const float* slices, int n, int d, uint16_t* x, uint16_t* xt, int ldt, cudaStream_t st);
cudaError_t launch_fi_bias_act(float* z, const float* b, int n, int h, int act, uint16_t* hb, uint16_t* ht, int ldt,
                               float* out, cudaStream_t st);
cudaError_t launch_fi_out_grad(const float* out, const float* t, const float* z, int64_t n_el, float inv_count,
                               float* g, double* part, int n_part, cudaStream_t st);
cudaError_t launch_fi_relu_grad(float* g, const float* z, int n, int h, uint16_t* gb, uint16_t* gt, int ldt,
                                cudaStream_t st);
cudaError_t launch_fi_convert(const float* src, int n, int d, uint16_t* dst, uint16_t* dst_t, int ldt,
                              cudaStream_t st);
cudaError_t launch_fi_colsum(const float* g, int n, int h, float* out, cudaStream_t st);
cudaError_t launch_fi_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1, float b2,
                           float eps, float bc1, float bc2, cudaStream_t st);
cudaError_t launch_fi_weight_copy(const float* w, int rows, int cols, uint16_t* dst, uint16_t* dst_t,
                                  cudaStream_t st);
// Adam on a [rows x cols] weight block plus its BF16 transposed copy dst_t [cols x rows].
cudaError_t launch_fi_adam_t(float* p, const float* g, float* m, float* v, int rows, int cols, float lr, float b1,
                             float b2, float eps, float bc1, float bc2, uint16_t* dst_t, cudaStream_t st);

// Device state of a fit whose stopping rules (App. B) are evaluated on the device.
struct FitCtlState {
    int iters;          // sweep cap
    int done;           // sweeps run so far
    int cont;           // 1 while the loop goes on
    int rises;          // consecutive sweeps whose validation loss rose
    int patience;       // stop once rises reaches this (0: no validation rule)
    int have_loss;      // prev_loss holds L[done - 1]
    int have_val;       // prev_val holds V[done]
    int pad;
    double tol;         // relative training-loss decrease threshold (0: off)
    double prev_loss, prev_val;
};

// After sweep done+1: done += 1, apply the rules to the training loss out_loss[0]
// (L[done - 1], summed inside that sweep's first pass) and the validation loss
// out_val[0] (V[done], or null), set cont and, when set_handle, the conditional
// handle of the enclosing graph loop.  mode 1 only records out_val[0] as V[0].
cudaError_t launch_fit_check(FitCtlState* s, const double* out_loss, const double* out_val,
                             cudaGraphConditionalHandle handle, int set_handle, int mode, cudaStream_t st);

// Set the loop's conditional handle from s->cont (the first node of the graph).
cudaError_t launch_fit_set_cond(const FitCtlState* s, cudaGraphConditionalHandle handle, cudaStream_t st);

// Sum per-CTA loss partials (part[0..n): loss, part[n..2n): count) into out[0..1];
// also append the loss to trace[*count] when trace is set, and increment *count.
cudaError_t launch_loss_append(const double* part, int n, double* trace, int* count, double* out,
                               cudaStream_t st);

cudaError_t launch_view_tc(const float* y, const uint32_t* mbits, const ViewDesc& v,
                           const WeightSpec& w, int need_den, int n_split, float* s_num,
                           float* s_den, int* err_flag, cudaStream_t st, TcLaunchInfo* info,
                           unsigned long long* trace = nullptr, const LossSpec* loss = nullptr,
                           double* loss_part = nullptr, long long wait_cycles = 0,
                           const TcTileConfig* cfg = nullptr);

bool tc_view_supported(const ViewDesc& v, int need_den);

// The tensor-core pass stages the Q operand's rows with TMA, instead of gathering
// them per tile, when within a tile one source has consecutive rows and the other,
// if any, a single row.  Tiles of tn columns start at multiples of tn when c_in is
// 1 or a multiple of tn: then the consecutive source needs one index term, divisor
// 1 and a modulus that is a multiple of tn, the single-row source a divisor that is
// a multiple of tn.  Otherwise (block form) the tiles restart at every c_in block
// and the last one of a block is partial: the consecutive source's modulus must be
// c_in (its rows are the offsets inside the block; rows past c_in read as zero) and
// the single-row source's divisor a multiple of c_in.  Returns the two sources'
// indices (q_const = -1 when there is one source).  A single source whose rows
// are the columns of a view with c_in == 1 (mod == c_out) is staged too: its rows
// never wrap, and the rows past c_out of the last, partial tile read as zeros.
inline bool q_rows_staged(const ViewDesc& v, int tn, int* q_var, int* q_const) {
    if (v.Q.nsrc < 1 || v.Q.nsrc > 2) return false;
    const bool block = v.c_in != 1 && v.c_in % tn != 0;
    int var = -1, cst = -1;
    for (int s = 0; s < v.Q.nsrc; ++s) {
        const SrcDesc& d = v.Q.src[s];
        if (d.nterm != 1 || d.mul[0] != 1) return false;
        const bool whole = v.Q.nsrc == 1 && v.c_in == 1 && d.mod[0] == v.c_out;
        if (d.div[0] == 1 && (block ? d.mod[0] == v.c_in : (d.mod[0] % tn == 0 || whole))) {
            if (var >= 0) return false;
            var = s;
        } else if (block ? d.div[0] % v.c_in == 0 : d.div[0] % tn == 0) {
            if (cst >= 0) return false;
            cst = s;
        } else {
            return false;
        }
    }
    if (var < 0) return false;
    *q_var = var;
    *q_const = cst;
    return true;
}

}  // namespace nef
