// foldin.cpp -- the fold-in encoder: an MLP from log1p(slice) to the slice's
// nonnegative mode-0 loading row, trained and run on the GPU by this library's
// own kernels (tensor-core products in k_gemm_tc.cu, the rest in k_foldin.cu).
//
//   x   = log1p(slice)                     [n x d]   (BF16)
//   z1  = x W1 + b1,  h1 = relu(z1)        [n x h]
//   z2  = h1 W2 + b2, h2 = relu(z2)        [n x h]
//   z3  = h2 W3 + b3, out = softplus(z3)   [n x o]
//   L   = mean over the n x o outputs of (log1p(out) - log1p(t))^2
//
// Every product is written as C = A . B^T with both operands K-major, using
// BF16 copies of the weights (straight and transposed) that the optimizer step
// refreshes, and BF16 copies of the activations and gradients (row-major and
// transposed) that the elementwise kernels write.  Parameters, gradients and
// the Adam moments are FP32 and packed in the order W1, b1, W2, b2, W3, b3
// (weights [fan_in x fan_out], row-major).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/nef.h"
#include "nef_internal.h"

struct nef_foldin_s {
    int d = 0, h = 0, o = 0, nmax = 0, ldn = 0;
    cudaStream_t st = nullptr;
    int64_t np = 0;
    int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    uint16_t *X = nullptr, *Xt = nullptr;
    uint16_t *W1t = nullptr, *W2t = nullptr, *W2n = nullptr, *W3t = nullptr, *W3n = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *OUT = nullptr;
    uint16_t *H1 = nullptr, *H1t = nullptr, *H2 = nullptr, *H2t = nullptr;
    float *G3 = nullptr, *G2 = nullptr, *G1 = nullptr;
    uint16_t *G3b = nullptr, *G3t = nullptr, *G2b = nullptr, *G2t = nullptr, *G1t = nullptr;
    double* part = nullptr;
    int n_part = 256;
    int* err = nullptr;
    float* ws = nullptr;       // split-K partial tiles of the products
    int64_t ws_floats = 0;
    int n_sm = 152;
    int64_t t = 0;
    int loaded_n = 0;          // slices whose features X, Xt hold (nef_foldin_load_batch), or 0
    std::vector<void*> allocs;
};

namespace {

using nef::set_last_error;

#define FI_TRY(x)                      \
    do {                               \
        const nef_status s_ = (x);     \
        if (s_ != NEF_OK) return s_;   \
    } while (0)

nef_status fi_fail(nef_status s, const char* msg) {
    set_last_error(msg);
    return s;
}

#define FI_CUDA(call)                                                        \
    do {                                                                     \
        cudaError_t e_ = (call);                                             \
        if (e_ != cudaSuccess) return fi_fail(NEF_ECUDA, cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
nef_status fi_alloc(nef_foldin_t f, T** ptr, int64_t count) {
    void* q = nullptr;
    if (cudaMalloc(&q, (size_t)std::max<int64_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return fi_fail(NEF_ENOMEM, "cudaMalloc failed in the fold-in encoder");
    }
    f->allocs.push_back(q);
    FI_CUDA(cudaMemsetAsync(q, 0, (size_t)std::max<int64_t>(count, 1) * sizeof(T), f->st));
    *ptr = static_cast<T*>(q);
    return NEF_OK;
}

void fi_free(nef_foldin_t f) {
    for (void* q : f->allocs) cudaFree(q);
    f->allocs.clear();
}

// BF16 copies of the weights used by the products (with_w1: also W1's, which the
// Adam step otherwise writes itself).
nef_status refresh_weights(nef_foldin_t f, bool with_w1 = true) {
    if (with_w1) FI_CUDA(nef::launch_fi_weight_copy(f->p + f->oW1, f->d, f->h, nullptr, f->W1t, f->st));
    FI_CUDA(nef::launch_fi_weight_copy(f->p + f->oW2, f->h, f->h, f->W2n, f->W2t, f->st));
    FI_CUDA(nef::launch_fi_weight_copy(f->p + f->oW3, f->h, f->o, f->W3n, f->W3t, f->st));
    return NEF_OK;
}

// Products with few output tiles and a long K (the first layer's forward product,
// the weight gradients of the small layers) split K over about one wave of CTAs.
nef_status gemm(nef_foldin_t f, const uint16_t* A, int64_t lda, const uint16_t* B, int64_t ldb, float* C, int64_t ldc,
                int M, int N, int K) {
    const int splits = nef::gemm_splits(M, N, K, f->n_sm);
    FI_CUDA(nef::launch_gemm_nt(A, lda, B, ldb, C, ldc, M, N, K, 0, f->err, f->st, f->ws, f->ws_floats, splits));
    return NEF_OK;
}

// Forward pass of n samples; with `train`, also the transposed copies the backward pass needs.
nef_status forward(nef_foldin_t f, const float* slices, int n, bool train) {
    const int d = f->d, h = f->h, o = f->o, ldn = f->ldn;
    if (slices) {
        FI_CUDA(nef::launch_fi_features(slices, n, d, f->X, train ? f->Xt : nullptr, ldn, f->st));
        f->loaded_n = 0;  // X (and Xt) no longer hold the kept batch
    } else if (f->loaded_n != n) {
        return fi_fail(NEF_EINVAL, "slices is NULL and no batch of this size is kept (nef_foldin_load_batch)");
    }
    FI_TRY(gemm(f, f->X, d, f->W1t, d, f->Z1, h, n, h, d));
    FI_CUDA(nef::launch_fi_bias_act(f->Z1, f->p + f->ob1, n, h, 1, f->H1, train ? f->H1t : nullptr, ldn, nullptr,
                                    f->st));
    FI_TRY(gemm(f, f->H1, h, f->W2t, h, f->Z2, h, n, h, h));
    FI_CUDA(nef::launch_fi_bias_act(f->Z2, f->p + f->ob2, n, h, 1, f->H2, train ? f->H2t : nullptr, ldn, nullptr,
                                    f->st));
    FI_TRY(gemm(f, f->H2, h, f->W3t, h, f->Z3, o, n, o, h));
    FI_CUDA(nef::launch_fi_bias_act(f->Z3, f->p + f->ob3, n, o, 2, nullptr, nullptr, ldn, f->OUT, f->st));
    return NEF_OK;
}

// Loss partials and the gradient of every parameter into f->g.
nef_status backward(nef_foldin_t f, const float* targets, int n) {
    const int h = f->h, o = f->o, ldn = f->ldn;
    const int64_t n_el = (int64_t)n * o;
    FI_CUDA(nef::launch_fi_out_grad(f->OUT, targets, f->Z3, n_el, (float)(1.0 / (double)n_el), f->G3, f->part,
                                    f->n_part, f->st));
    FI_CUDA(nef::launch_fi_convert(f->G3, n, o, f->G3b, f->G3t, ldn, f->st));
    // layer 3: gW3 = h2^T g3, gb3 = colsum g3, g_h2 = g3 W3^T
    FI_TRY(gemm(f, f->H2t, ldn, f->G3t, ldn, f->g + f->oW3, o, h, o, n));
    FI_CUDA(nef::launch_fi_colsum(f->G3, n, o, f->g + f->ob3, f->st));
    FI_TRY(gemm(f, f->G3b, o, f->W3n, o, f->G2, h, n, h, o));
    FI_CUDA(nef::launch_fi_relu_grad(f->G2, f->Z2, n, h, f->G2b, f->G2t, ldn, f->st));
    // layer 2
    FI_TRY(gemm(f, f->H1t, ldn, f->G2t, ldn, f->g + f->oW2, h, h, h, n));
    FI_CUDA(nef::launch_fi_colsum(f->G2, n, h, f->g + f->ob2, f->st));
    FI_TRY(gemm(f, f->G2b, h, f->W2n, h, f->G1, h, n, h, h));
    FI_CUDA(nef::launch_fi_relu_grad(f->G1, f->Z1, n, h, nullptr, f->G1t, ldn, f->st));
    // layer 1
    FI_TRY(gemm(f, f->Xt, ldn, f->G1t, ldn, f->g + f->oW1, h, f->d, h, n));
    FI_CUDA(nef::launch_fi_colsum(f->G1, n, h, f->g + f->ob1, f->st));
    return NEF_OK;
}

nef_status read_loss(nef_foldin_t f, int n, double* loss) {
    std::vector<double> hp(f->n_part);
    int herr = 0;
    FI_CUDA(cudaMemcpyAsync(hp.data(), f->part, f->n_part * sizeof(double), cudaMemcpyDeviceToHost, f->st));
    FI_CUDA(cudaMemcpyAsync(&herr, f->err, sizeof(int), cudaMemcpyDeviceToHost, f->st));
    FI_CUDA(cudaStreamSynchronize(f->st));
    if (herr) return fi_fail(NEF_ETIMEOUT, "a bounded wait in the fold-in products gave up");
    double s = 0.0;
    for (double x : hp) s += x;
    *loss = s / ((double)n * f->o);
    return NEF_OK;
}

nef_status check_batch(nef_foldin_t f, int n) {
    if (!f) return fi_fail(NEF_EINVAL, "encoder is NULL");
    if (n < 1 || n > f->nmax) return fi_fail(NEF_EINVAL, "batch size must be in [1, max_batch]");
    return NEF_OK;
}

}  // namespace

extern "C" {

int64_t nef_foldin_num_params(int d_in, int d_h, int d_out) {
    return (int64_t)d_in * d_h + d_h + (int64_t)d_h * d_h + d_h + (int64_t)d_h * d_out + d_out;
}

nef_status nef_foldin_create(int d_in, int d_h, int d_out, int max_batch, const float* params, void* stream,
                             nef_foldin_t* out) {
    set_last_error("");
    if (!out) return fi_fail(NEF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!params) return fi_fail(NEF_EINVAL, "params is NULL");
    if (d_in < 8 || d_h < 8 || d_out < 8 || d_in % 8 || d_h % 8 || d_out % 8)
        return fi_fail(NEF_EINVAL, "layer widths must be positive multiples of 8");
    if (max_batch < 1) return fi_fail(NEF_EINVAL, "max_batch must be >= 1");
    nef_foldin_t f = new nef_foldin_s;
    f->d = d_in;
    f->h = d_h;
    f->o = d_out;
    f->nmax = max_batch;
    f->ldn = (max_batch + 7) / 8 * 8;
    f->st = static_cast<cudaStream_t>(stream);
    f->oW1 = 0;
    f->ob1 = (int64_t)d_in * d_h;
    f->oW2 = f->ob1 + d_h;
    f->ob2 = f->oW2 + (int64_t)d_h * d_h;
    f->oW3 = f->ob2 + d_h;
    f->ob3 = f->oW3 + (int64_t)d_h * d_out;
    f->np = f->ob3 + d_out;
    const int64_t n = max_batch, d = d_in, h = d_h, o = d_out, ldn = f->ldn;
    nef_status s = NEF_OK;
    auto A = [&](auto** ptr, int64_t cnt) {
        if (s == NEF_OK) s = fi_alloc(f, ptr, cnt);
    };
    A(&f->p, f->np);
    A(&f->g, f->np);
    A(&f->m, f->np);
    A(&f->v, f->np);
    A(&f->X, n * d);
    A(&f->Xt, d * ldn);
    A(&f->W1t, h * d);
    A(&f->W2t, h * h);
    A(&f->W2n, h * h);
    A(&f->W3t, o * h);
    A(&f->W3n, h * o);
    A(&f->Z1, n * h);
    A(&f->Z2, n * h);
    A(&f->Z3, n * o);
    A(&f->OUT, n * o);
    A(&f->H1, n * h);
    A(&f->H1t, h * ldn);
    A(&f->H2, n * h);
    A(&f->H2t, h * ldn);
    A(&f->G3, n * o);
    A(&f->G2, n * h);
    A(&f->G1, n * h);
    A(&f->G3b, n * o);
    A(&f->G3t, o * ldn);
    A(&f->G2b, n * h);
    A(&f->G2t, h * ldn);
    A(&f->G1t, h * ldn);
    A(&f->part, f->n_part);
    A(&f->err, 1);
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && nsm > 0)
            f->n_sm = nsm;
        cudaGetLastError();
        // every product of forward() and backward(): (M, N, K, ldc)
        const int64_t prods[8][4] = {{n, h, d, h}, {n, h, h, h}, {n, o, h, o}, {h, o, n, o},
                                     {n, h, o, h}, {h, h, n, h}, {n, h, h, h}, {d, h, n, h}};
        for (auto& q : prods) {
            const int sp = nef::gemm_splits((int)q[0], (int)q[1], (int)q[2], f->n_sm);
            if (sp > 1) f->ws_floats = std::max<int64_t>(f->ws_floats, sp * q[0] * q[3]);
        }
        if (f->ws_floats > 0) A(&f->ws, f->ws_floats);
    }
    if (s == NEF_OK && cudaMemcpyAsync(f->p, params, f->np * sizeof(float), cudaMemcpyDeviceToDevice, f->st) !=
                           cudaSuccess)
        s = fi_fail(NEF_ECUDA, "parameter copy failed");
    if (s == NEF_OK) s = refresh_weights(f);
    if (s != NEF_OK) {
        fi_free(f);
        delete f;
        return s;
    }
    *out = f;
    return NEF_OK;
}

void nef_foldin_destroy(nef_foldin_t f) {
    if (!f) return;
    fi_free(f);
    delete f;
}

nef_status nef_foldin_grad(nef_foldin_t f, const float* slices, const float* targets, int n, float* grads,
                           double* loss) {
    set_last_error("");
    FI_TRY(check_batch(f, n));
    if (!targets || !grads) return fi_fail(NEF_EINVAL, "NULL argument");
    FI_TRY(forward(f, slices, n, true));
    FI_TRY(backward(f, targets, n));
    FI_CUDA(cudaMemcpyAsync(grads, f->g, f->np * sizeof(float), cudaMemcpyDeviceToDevice, f->st));
    if (loss) FI_TRY(read_loss(f, n, loss));
    return NEF_OK;
}

nef_status nef_foldin_train_step(nef_foldin_t f, const float* slices, const float* targets, int n, double lr,
                                 double beta1, double beta2, double eps, double* loss) {
    set_last_error("");
    FI_TRY(check_batch(f, n));
    if (!targets) return fi_fail(NEF_EINVAL, "NULL argument");
    if (!(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
        return fi_fail(NEF_EINVAL, "Adam hyper-parameters out of range");
    FI_TRY(forward(f, slices, n, true));
    FI_TRY(backward(f, targets, n));
    f->t += 1;
    const double bc1 = 1.0 - std::pow(beta1, (double)f->t), bc2 = 1.0 - std::pow(beta2, (double)f->t);
    // W1 (the bulk of the parameters) in tiles that also write its BF16 transposed
    // copy; the rest of the packed parameters elementwise; then the small copies
    FI_CUDA(nef::launch_fi_adam_t(f->p + f->oW1, f->g + f->oW1, f->m + f->oW1, f->v + f->oW1, f->d, f->h, (float)lr,
                                  (float)beta1, (float)beta2, (float)eps, (float)bc1, (float)bc2, f->W1t, f->st));
    FI_CUDA(nef::launch_fi_adam(f->p + f->ob1, f->g + f->ob1, f->m + f->ob1, f->v + f->ob1, f->np - f->ob1,
                                (float)lr, (float)beta1, (float)beta2, (float)eps, (float)bc1, (float)bc2, f->st));
    FI_TRY(refresh_weights(f, false));
    if (loss) FI_TRY(read_loss(f, n, loss));
    return NEF_OK;
}

nef_status nef_foldin_load_batch(nef_foldin_t f, const float* slices, int n) {
    set_last_error("");
    FI_TRY(check_batch(f, n));
    if (!slices) return fi_fail(NEF_EINVAL, "NULL argument");
    f->loaded_n = 0;  // X and Xt are rewritten: no batch is kept unless this one is
    FI_CUDA(nef::launch_fi_features(slices, n, f->d, f->X, f->Xt, f->ldn, f->st));
    f->loaded_n = n;
    return NEF_OK;
}

nef_status nef_foldin_predict(nef_foldin_t f, const float* slices, int n, float* out) {
    set_last_error("");
    FI_TRY(check_batch(f, n));
    if (!slices || !out) return fi_fail(NEF_EINVAL, "NULL argument");
    FI_TRY(forward(f, slices, n, false));
    FI_CUDA(cudaMemcpyAsync(out, f->OUT, (size_t)n * f->o * sizeof(float), cudaMemcpyDeviceToDevice, f->st));
    return NEF_OK;
}

nef_status nef_foldin_params(nef_foldin_t f, float* out) {
    set_last_error("");
    if (!f || !out) return fi_fail(NEF_EINVAL, "NULL argument");
    FI_CUDA(cudaMemcpyAsync(out, f->p, f->np * sizeof(float), cudaMemcpyDeviceToDevice, f->st));
    return NEF_OK;
}

}  // extern "C"
