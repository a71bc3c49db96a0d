// nef_device.cuh -- device-side helpers: the App. B weights, divergence and
// update in float and double, with specialised powers.
#pragma once

#include <cmath>
#include <cstdint>

#include "nef_internal.h"

namespace nef {

__device__ __forceinline__ float pw_code(float x, int code, double e) {
    switch (code) {
        case POW_ONE: return 1.0f;
        case POW_ID: return x;
        case POW_RCP: return 1.0f / x;
        case POW_RSQRT: return rsqrtf(x);
        case POW_SQRT: return sqrtf(x);
        case POW_SQ: return x * x;
        case POW_RSQRT3: { float r = rsqrtf(x); return r * r * r; }
        case POW_RCP2: { float r = 1.0f / x; return r * r; }
        default: return powf(x, (float)e);
    }
}

__device__ __forceinline__ double pw_code(double x, int code, double e) {
    switch (code) {
        case POW_ONE: return 1.0;
        case POW_ID: return x;
        case POW_RCP: return 1.0 / x;
        case POW_RSQRT: return 1.0 / sqrt(x);
        case POW_SQRT: return sqrt(x);
        case POW_SQ: return x * x;
        case POW_RSQRT3: { double r = 1.0 / sqrt(x); return r * r * r; }
        case POW_RCP2: { double r = 1.0 / x; return r * r; }
        default: return pow(x, e);
    }
}

// x^p with 0^p = 0 for p > 0, 0^0 = 1 (the convention of App. B at x = 0).
template <typename T>
__device__ __forceinline__ T powz(T x, double p) {
    if (x == T(0)) return p > 0.0 ? T(0) : (p == 0.0 ? T(1) : T(INFINITY));
    return pw_code(x, POW_GENERAL, p);
}

// y log z with 0 log z = 0 (the convention of App. B at y = 0).
template <typename T>
__device__ __forceinline__ T xlogy(T y, T z) {
    return y == T(0) ? T(0) : y * log(z);
}

// a and b of the likelihood families of App. B (negative binomial, binomial on
// the odds, Jensen-Shannon); mask handled by the caller.
template <typename T>
__device__ __forceinline__ void lik_weights(T y, T yh, const WeightSpec& w, T& wa, T& wb) {
    const T par = T(w.par);
    switch (w.lik) {
        case LIK_NEGBIN: wa = y / yh; wb = (par + y) / (par + yh); break;
        case LIK_BINOMIAL: wa = y / yh; wb = par / (T(1) + yh); break;
        default: wa = log((y + yh) / (T(2) * yh)); wb = T(1); break;  // LIK_JS
    }
}

// Masked weights of App. B (mask handled by the caller).
template <typename T>
__device__ __forceinline__ void ab_weights(T y, T yh, const WeightSpec& w, T& wa, T& wb) {
    if (w.lik) {
        lik_weights(y, yh, w, wa, wb);
        return;
    }
    if (w.log_case) {
        wa = log(y / yh);
        wb = T(1);
        return;
    }
    T ya;
    if (y == T(0)) ya = (w.e_y > 0.0) ? T(0) : (w.e_y == 0.0 ? T(1) : T(INFINITY));
    else ya = pw_code(y, w.y_code, w.e_y);
    wa = ya * pw_code(yh, w.a_code, w.e_a);
    wb = pw_code(yh, w.b_code, w.e_b);
}

// D(x, y) of a likelihood family of App. B with its constant terms dropped:
// negative binomial (phi + x) log(phi + y) - x log y; binomial on the odds
// n log(1 + y) - x log y; Jensen-Shannon (x log x + y log y)/2 - m log m with
// m = (x + y)/2, evaluated as (x log(x/m) + y log(y/m))/2 (the same value
// without the cancellation of the first form).
template <typename T>
__device__ __forceinline__ T lik_divergence(T x, T y, const LossSpec& L) {
    const T par = T(L.par);
    switch (L.lik) {
        case LIK_NEGBIN: return xlogy(par + x, par + y) - xlogy(x, y);
        case LIK_BINOMIAL: return par * log1p(y) - xlogy(x, y);
        default: {  // LIK_JS
            const T m = T(0.5) * (x + y);
            return T(0.5) * (xlogy(x, x / m) + xlogy(y, y / m));
        }
    }
}

// D_{alpha,beta}(x, y): the five cases of App. B (or a likelihood family's D).
template <typename T>
__device__ __forceinline__ T divergence(T x, T y, const LossSpec& L) {
    if (L.lik) return lik_divergence(x, y, L);
    const double al = L.alpha, be = L.beta;
    switch (L.kase) {
        case 1: {  // beta = 0
            T xa = powz(x, al);
            T t = (x == T(0)) ? T(0) : T(al) * xa * log(x / y);
            return T(1.0 / (al * al)) * (powz(y, al) - xa + t);
        }
        case 2:  // alpha = -beta
            return T(1.0 / (al * al)) * (powz(x, al) / powz(y, al) - T(1) + T(al) * log(y / x));
        case 3:  // alpha = 0
            return T(1.0 / (be * be)) *
                   (T(be) * powz(y, be) * log(y / x) - powz(y, be) + powz(x, be));
        case 4: {  // alpha = beta = 0
            T d = log(x) - log(y);
            return T(0.5) * d * d;
        }
        default: {
            const double ab = al + be;
            return T(1.0 / (al * be)) *
                   (T(al / ab) * powz(x, ab) + T(be / ab) * powz(y, ab) - powz(x, al) * powz(y, be));
        }
    }
}

// The stopping rules of App. B applied after one sweep (mode 0) or recording V[0]
// before the first sweep (mode 1); returns the loop's new condition (1 = go on).
// Training loss: stop once the relative decrease (L[k-2] - L[k-1]) / L[k-2] falls
// below tol; validation loss: stop once it rose `patience` sweeps in a row; and
// the sweep cap.
__host__ __device__ inline int fit_rule_step(FitCtlState* s, const double* out_loss, const double* out_val,
                                             int mode) {
    if (mode == 1) {
        s->prev_val = out_val[0];
        s->have_val = 1;
        return s->cont;
    }
    s->done += 1;
    bool stop = s->done >= s->iters;
    if (out_loss) {
        const double l = out_loss[0];
        if (s->tol > 0.0 && s->have_loss && s->prev_loss != 0.0 && (s->prev_loss - l) / s->prev_loss < s->tol)
            stop = true;
        s->prev_loss = l;
        s->have_loss = 1;
    }
    if (out_val) {
        const double v = out_val[0];
        s->rises = (s->have_val && v > s->prev_val) ? s->rises + 1 : 0;
        if (s->patience > 0 && s->rises >= s->patience) stop = true;
        s->prev_val = v;
        s->have_val = 1;
    }
    s->cont = stop ? 0 : 1;
    return s->cont;
}

// Eq. 3.4 for one element; den == 0 keeps theta.
template <typename T>
__device__ __forceinline__ T mu_update(T theta, T num, T den, const UpdateSpec& u) {
    if (den == T(0)) return theta;
    T z = num / den;
    T g = u.log_case ? exp(z) : pw_code(z, u.eta_code, u.eta);
    T v = theta * g;
    return v > T(u.eps) ? v : T(u.eps);
}

// Bit e of a packed mask (bit e%32 of word e/32).
__device__ __forceinline__ int mask_bit(const uint32_t* bits, int64_t e) {
    return (bits[e >> 5] >> (e & 31)) & 1u;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace nef
