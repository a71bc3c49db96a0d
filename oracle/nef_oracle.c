/*
 * nef_oracle.c -- FP64 CPU oracle for the NNEinFact multiplicative update.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this code.  It shares no
 * code with the CUDA path and must never be called by the product.
 *
 * Every routine is a plain loop nest written from the paper:
 *   - reconstruction  yhat_i = sum_r prod_l theta^(l)_{i_l, r_l}        (Eq. 2.1)
 *   - a(x,y), b(x,y) of the (alpha,beta)-divergence                     (App. B)
 *   - numerator / denominator as einsum(einstr_l, ..., a(Y,Yhat), ...)  (Eq. 3.6-3.8)
 *   - update  theta <- max(eps, theta * g^{-1}(num / den))              (Eq. 3.4)
 *   - g(lambda) case table                                              (App. B)
 *   - D_{alpha,beta}(x,y) five-case definition                          (App. B)
 *   - Algorithm 1: Gauss-Seidel over factors in string order, Yhat
 *     recomputed before every factor update                             (Algorithm 1)
 *   - the likelihood losses of App. B outside the (alpha,beta) family:
 *     negative binomial, binomial / Bernoulli on odds, Jensen-Shannon,
 *     with their a, b and g                                             (App. B)
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - the mask multiplies the weights: W_a = M*a, W_b = M*b (Sec. 6, masked
 *     training loss); a literal M*Y, M*Yhat substitution would leave b(0,0)=1
 *     for KL and count missing entries in the denominator;
 *   - den == 0 leaves theta unchanged (no information about that entry);
 *   - 0 * log 0 = 0 and 0^p = 0 for p > 0 in D and in a(x,y);
 *   - the negative binomial dispersion phi is one value for all entries.
 *
 * Layout: Y and the mask are row-major over the observed letters in RHS order;
 * each factor is row-major over its own letters in term order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXLET 26
#define OR_MAXFAC 16
#define OR_MAXOPS (OR_MAXFAC + 1)

typedef struct {
    int32_t n_obs;                         /* M: observed letters are ids 0..M-1 (RHS order) */
    int32_t n_let;                         /* M + K: latent letters are ids M..M+K-1         */
    int64_t dim[OR_MAXLET];
    int32_t n_fac;                         /* L */
    int32_t fac_nlet[OR_MAXFAC];
    int32_t fac_let[OR_MAXFAC][OR_MAXLET]; /* letter ids of each factor, term order          */
} or_spec;

/* ------------------------------------------------------------------ strides */

static void y_strides(const or_spec* s, int64_t* st) {
    for (int x = 0; x < OR_MAXLET; ++x) st[x] = 0;
    int64_t acc = 1;
    for (int m = s->n_obs - 1; m >= 0; --m) { st[m] = acc; acc *= s->dim[m]; }
}

static void fac_strides(const or_spec* s, int f, int64_t* st) {
    for (int x = 0; x < OR_MAXLET; ++x) st[x] = 0;
    int64_t acc = 1;
    for (int p = s->fac_nlet[f] - 1; p >= 0; --p) {
        int x = s->fac_let[f][p];
        st[x] = acc;
        acc *= s->dim[x];
    }
}

static int64_t fac_size(const or_spec* s, int f) {
    int64_t n = 1;
    for (int p = 0; p < s->fac_nlet[f]; ++p) n *= s->dim[s->fac_let[f][p]];
    return n;
}

static int64_t y_size(const or_spec* s) {
    int64_t n = 1;
    for (int m = 0; m < s->n_obs; ++m) n *= s->dim[m];
    return n;
}

static int in_factor(const or_spec* s, int f, int x) {
    for (int p = 0; p < s->fac_nlet[f]; ++p) if (s->fac_let[f][p] == x) return 1;
    return 0;
}

/* --------------------------------------------------------------- contraction
 * Generic einsum: for every output element (enumerated row-major over
 * out_let), sum over every combination of the free letters the product of the
 * operands, each addressed through its per-letter strides (0 = letter absent).
 * This is the definition of einsum written out; nothing is reordered.
 */
static void or_contract(const or_spec* s, int n_ops, const double* const* ops,
                        int64_t st[][OR_MAXLET], int n_out, const int* out_let,
                        int n_free, const int* free_let, double* out) {
    int64_t n_out_el = 1;
    for (int q = 0; q < n_out; ++q) n_out_el *= s->dim[out_let[q]];
    int64_t n_free_el = 1;
    for (int q = 0; q < n_free; ++q) n_free_el *= s->dim[free_let[q]];

#pragma omp parallel for schedule(static)
    for (int64_t o = 0; o < n_out_el; ++o) {
        int64_t base[OR_MAXOPS];
        for (int k = 0; k < n_ops; ++k) base[k] = 0;
        int64_t rem = o;
        for (int q = n_out - 1; q >= 0; --q) {
            int x = out_let[q];
            int64_t v = rem % s->dim[x];
            rem /= s->dim[x];
            for (int k = 0; k < n_ops; ++k) base[k] += v * st[k][x];
        }
        double acc = 0.0;
        int64_t idx[OR_MAXLET];
        for (int q = 0; q < n_free; ++q) idx[q] = 0;
        int64_t off[OR_MAXOPS];
        for (int k = 0; k < n_ops; ++k) off[k] = base[k];
        for (int64_t c = 0; c < n_free_el; ++c) {
            double p = 1.0;
            for (int k = 0; k < n_ops; ++k) p *= ops[k][off[k]];
            acc += p;
            /* odometer step over the free letters, last letter fastest */
            for (int q = n_free - 1; q >= 0; --q) {
                int x = free_let[q];
                idx[q] += 1;
                for (int k = 0; k < n_ops; ++k) off[k] += st[k][x];
                if (idx[q] < s->dim[x]) break;
                for (int k = 0; k < n_ops; ++k) off[k] -= st[k][x] * s->dim[x];
                idx[q] = 0;
            }
        }
        out[o] = acc;
    }
}

/* Eq. 2.1: Yhat = einsum(model_str, Theta) */
void or_reconstruct(const or_spec* s, const double* const* fac, double* yhat) {
    int64_t st[OR_MAXOPS][OR_MAXLET];
    for (int f = 0; f < s->n_fac; ++f) fac_strides(s, f, st[f]);
    int out_let[OR_MAXLET], free_let[OR_MAXLET];
    for (int m = 0; m < s->n_obs; ++m) out_let[m] = m;
    int nf = 0;
    for (int x = s->n_obs; x < s->n_let; ++x) free_let[nf++] = x;
    or_contract(s, s->n_fac, fac, st, s->n_obs, out_let, nf, free_let, yhat);
}

/* Eq. 3.6-3.8: out = einsum(einstr_l, Theta^(1..l-1), T, Theta^(l+1..L)),
 * i.e. T (a tensor shaped like Y) takes the place of factor l's term and the
 * output is indexed by factor l's letters. */
void or_einstr(const or_spec* s, int l, const double* T, const double* const* fac,
               double* out) {
    const double* ops[OR_MAXOPS];
    int64_t st[OR_MAXOPS][OR_MAXLET];
    int n_ops = 0;
    ops[n_ops] = T;
    y_strides(s, st[n_ops]);
    ++n_ops;
    for (int f = 0; f < s->n_fac; ++f) {
        if (f == l) continue;
        ops[n_ops] = fac[f];
        fac_strides(s, f, st[n_ops]);
        ++n_ops;
    }
    int out_let[OR_MAXLET], free_let[OR_MAXLET];
    int no = s->fac_nlet[l];
    for (int p = 0; p < no; ++p) out_let[p] = s->fac_let[l][p];
    int nf = 0;
    for (int x = 0; x < s->n_let; ++x)
        if (!in_factor(s, l, x)) free_let[nf++] = x;
    or_contract(s, n_ops, ops, st, no, out_let, nf, free_let, out);
}

/* ----------------------------------------------------- loss family (App. B) */

/* x^p with the convention 0^p = 0 for p > 0 (and 0^0 = 1). */
static double powz(double x, double p) {
    if (x == 0.0) return p > 0.0 ? 0.0 : (p == 0.0 ? 1.0 : INFINITY);
    return pow(x, p);
}

/* D_{alpha,beta}(x, y), the five cases of App. B. */
double or_divergence(double x, double y, double al, double be) {
    double ab = al + be;
    if (al != 0.0 && be != 0.0 && ab != 0.0) {
        return (1.0 / (al * be)) *
               ((al / ab) * powz(x, ab) + (be / ab) * powz(y, ab) - powz(x, al) * powz(y, be));
    }
    if (be == 0.0 && al != 0.0) {
        double xa = powz(x, al);
        double t = (x == 0.0) ? 0.0 : al * xa * log(x / y); /* 0 * log 0 = 0 */
        return (1.0 / (al * al)) * (powz(y, al) - xa + t);
    }
    if (al == -be && al != 0.0) {
        return (1.0 / (al * al)) * (powz(x, al) / powz(y, al) - 1.0 + al * log(y / x));
    }
    if (al == 0.0 && be != 0.0) {
        return (1.0 / (be * be)) * (be * powz(y, be) * log(y / x) - powz(y, be) + powz(x, be));
    }
    double d = log(x) - log(y);
    return 0.5 * d * d;
}

/* 0 = ok, 1 = no decomposition known (alpha == 0 and beta != 1, App. B). */
int or_ab_supported(double al, double be) {
    if (al == 0.0 && be != 1.0) return 0;
    return 1;
}

/* a(x,y) and b(x,y): alpha != 0: a = x^alpha y^(beta-1), b = y^(alpha+beta-1);
 * alpha = 0, beta = 1: a = log(x/y), b = 1. */
static void ab_weights(double x, double y, double al, double be, double* a, double* b) {
    if (al != 0.0) {
        *a = powz(x, al) * pow(y, be - 1.0);
        *b = pow(y, al + be - 1.0);
    } else {
        *a = log(x / y);
        *b = 1.0;
    }
}

/* g^{-1}(z) from the App. B case table on q = 1/alpha - beta/alpha. */
double or_ginv(double z, double al, double be) {
    if (al == 0.0 && be == 1.0) return exp(z);
    double q = 1.0 / al - be / al;
    double p;
    if (q > 1.0) p = 1.0 - be;
    else if (q < 0.0) p = al + be - 1.0;
    else p = al;
    return pow(z, 1.0 / p);
}

/* ------------------------------------------------------------ Algorithm 1 */

/* Elementwise weights a(Y,Yhat), b(Y,Yhat), masked. */
void or_weights(int64_t n, const double* y, const uint8_t* mask, const double* yhat,
                double al, double be, double* wa, double* wb) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) {
        if (mask && !mask[e]) { wa[e] = 0.0; wb[e] = 0.0; continue; }
        ab_weights(y[e], yhat[e], al, be, &wa[e], &wb[e]);
    }
}

/* Eq. 3.4: theta <- max(eps, theta * g^{-1}(num/den)); den == 0 keeps theta. */
void or_apply_update(int64_t n, double* theta, const double* num, const double* den,
                     double al, double be, double eps) {
    for (int64_t e = 0; e < n; ++e) {
        if (den[e] == 0.0) continue;
        double v = theta[e] * or_ginv(num[e] / den[e], al, be);
        theta[e] = v > eps ? v : eps;
    }
}

/* One factor update (the body of the inner loop of Algorithm 1).
 * num/den (size of factor l) are returned for inspection when non-NULL. */
int or_update_factor(const or_spec* s, int l, const double* y, const uint8_t* mask,
                     double* const* fac, double al, double be, double eps,
                     double* num_out, double* den_out) {
    if (!or_ab_supported(al, be)) return 1;
    int64_t n = y_size(s);
    int64_t nl = fac_size(s, l);
    double* yhat = (double*)malloc(sizeof(double) * n);
    double* wa = (double*)malloc(sizeof(double) * n);
    double* wb = (double*)malloc(sizeof(double) * n);
    double* num = num_out ? num_out : (double*)malloc(sizeof(double) * nl);
    double* den = den_out ? den_out : (double*)malloc(sizeof(double) * nl);
    if (!yhat || !wa || !wb || !num || !den) return 2;
    or_reconstruct(s, (const double* const*)fac, yhat);
    or_weights(n, y, mask, yhat, al, be, wa, wb);
    or_einstr(s, l, wa, (const double* const*)fac, num);
    or_einstr(s, l, wb, (const double* const*)fac, den);
    or_apply_update(nl, fac[l], num, den, al, be, eps);
    free(yhat); free(wa); free(wb);
    if (!num_out) free(num);
    if (!den_out) free(den);
    return 0;
}

/* Sum over observed entries of D(y, yhat); count of observed entries in *cnt. */
double or_loss(const or_spec* s, const double* y, const uint8_t* mask,
               const double* const* fac, double al, double be, int64_t* cnt) {
    int64_t n = y_size(s);
    double* yhat = (double*)malloc(sizeof(double) * n);
    or_reconstruct(s, fac, yhat);
    double tot = 0.0;
    int64_t c = 0;
    for (int64_t e = 0; e < n; ++e) {
        if (mask && !mask[e]) continue;
        tot += or_divergence(y[e], yhat[e], al, be);
        ++c;
    }
    free(yhat);
    if (cnt) *cnt = c;
    return tot;
}

/* Algorithm 1 for a fixed number of sweeps; trace (iters+1 entries, or NULL)
 * receives the loss before the first sweep and after each sweep. */
int or_fit(const or_spec* s, const double* y, const uint8_t* mask, double* const* fac,
           double al, double be, double eps, int iters, double* trace) {
    if (!or_ab_supported(al, be)) return 1;
    if (trace) trace[0] = or_loss(s, y, mask, (const double* const*)fac, al, be, NULL);
    for (int it = 0; it < iters; ++it) {
        for (int l = 0; l < s->n_fac; ++l) {
            int rc = or_update_factor(s, l, y, mask, fac, al, be, eps, NULL, NULL);
            if (rc) return rc;
        }
        if (trace) trace[it + 1] = or_loss(s, y, mask, (const double* const*)fac, al, be, NULL);
    }
    return 0;
}

/* ---------------------------------------------------- sampled evaluation
 * For parity checks at sizes where a full FP64 pass is too slow: num and den
 * of Eq. 3.6-3.8 for selected elements of factor l only.  The sum over the
 * letters outside factor l is grouped by observed entry (yhat and the weights
 * are evaluated once per entry, then the latent letters outside factor l are
 * summed); this is the same finite sum in a different order. */
int or_numden_sampled(const or_spec* s, int l, int64_t n_samp, const int64_t* elems,
                      const double* y, const uint8_t* mask, const double* const* fac,
                      double al, double be, double* num, double* den) {
    if (!or_ab_supported(al, be)) return 1;
    int64_t yst[OR_MAXLET];
    y_strides(s, yst);
    int64_t fst[OR_MAXFAC][OR_MAXLET];
    for (int f = 0; f < s->n_fac; ++f) fac_strides(s, f, fst[f]);
    int free_obs[OR_MAXLET], free_lat[OR_MAXLET], all_lat[OR_MAXLET];
    int nfo = 0, nfl = 0, nal = 0;
    for (int x = 0; x < s->n_let; ++x) {
        if (x >= s->n_obs) all_lat[nal++] = x;
        if (in_factor(s, l, x)) continue;
        if (x < s->n_obs) free_obs[nfo++] = x; else free_lat[nfl++] = x;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < n_samp; ++q) {
        int64_t idx[OR_MAXLET];
        for (int x = 0; x < OR_MAXLET; ++x) idx[x] = 0;
        int64_t rem = elems[q];
        for (int p = s->fac_nlet[l] - 1; p >= 0; --p) {
            int x = s->fac_let[l][p];
            idx[x] = rem % s->dim[x];
            rem /= s->dim[x];
        }
        double sn = 0.0, sd = 0.0;
        int64_t nobs = 1;
        for (int t = 0; t < nfo; ++t) nobs *= s->dim[free_obs[t]];
        for (int64_t co = 0; co < nobs; ++co) {
            int64_t r2 = co;
            for (int t = nfo - 1; t >= 0; --t) {
                int x = free_obs[t];
                idx[x] = r2 % s->dim[x];
                r2 /= s->dim[x];
            }
            int64_t e = 0;
            for (int m = 0; m < s->n_obs; ++m) e += idx[m] * yst[m];
            if (mask && !mask[e]) continue;
            /* yhat at entry e: all latent letters free */
            int64_t save[OR_MAXLET];
            for (int x = 0; x < OR_MAXLET; ++x) save[x] = idx[x];
            int64_t nlat = 1;
            for (int t = 0; t < nal; ++t) nlat *= s->dim[all_lat[t]];
            double yh = 0.0;
            for (int64_t cl = 0; cl < nlat; ++cl) {
                int64_t r3 = cl;
                for (int t = nal - 1; t >= 0; --t) {
                    int x = all_lat[t];
                    idx[x] = r3 % s->dim[x];
                    r3 /= s->dim[x];
                }
                double p = 1.0;
                for (int f = 0; f < s->n_fac; ++f) {
                    int64_t off = 0;
                    for (int pp = 0; pp < s->fac_nlet[f]; ++pp) {
                        int x = s->fac_let[f][pp];
                        off += idx[x] * fst[f][x];
                    }
                    p *= fac[f][off];
                }
                yh += p;
            }
            for (int x = 0; x < OR_MAXLET; ++x) idx[x] = save[x];
            double wa, wb;
            ab_weights(y[e], yh, al, be, &wa, &wb);
            /* gradient factor: latent letters outside factor l free */
            int64_t ng = 1;
            for (int t = 0; t < nfl; ++t) ng *= s->dim[free_lat[t]];
            double g = 0.0;
            for (int64_t cg = 0; cg < ng; ++cg) {
                int64_t r4 = cg;
                for (int t = nfl - 1; t >= 0; --t) {
                    int x = free_lat[t];
                    idx[x] = r4 % s->dim[x];
                    r4 /= s->dim[x];
                }
                double p = 1.0;
                for (int f = 0; f < s->n_fac; ++f) {
                    if (f == l) continue;
                    int64_t off = 0;
                    for (int pp = 0; pp < s->fac_nlet[f]; ++pp) {
                        int x = s->fac_let[f][pp];
                        off += idx[x] * fst[f][x];
                    }
                    p *= fac[f][off];
                }
                g += p;
            }
            sn += wa * g;
            sd += wb * g;
        }
        num[q] = sn;
        den[q] = sd;
    }
    return 0;
}

/* ---------------------------------------- likelihood losses of App. B
 * Losses outside the (alpha,beta) family that have the same convex-concave
 * structure, each with its a(x,y), b(x,y) and g (App. B):
 *   kind 1, negative binomial with dispersion par = phi (one value for all
 *     entries): D = (phi + x) log(phi + y) - x log y,
 *     a = x / y, b = (phi + x) / (phi + y), g(lambda) = lambda;
 *   kind 2, binomial on the odds y = p / (1 - p) with n trials per entry
 *     (ntr, or 1 everywhere = Bernoulli when ntr is NULL):
 *     D = n log(1 + y) - x log y, a = x / y, b = n / (1 + y), g(lambda) = lambda;
 *   kind 3, Jensen-Shannon: D = (x log x + y log y) / 2 - (x + y)/2 log((x + y)/2),
 *     a = log((x + y) / (2 y)), b = 1, g(lambda) = log(lambda), so the update
 *     multiplies by exp(num / den).
 * The constant terms of the likelihoods are dropped (0 log 0 = 0). */

static double xlogy(double x, double y) { return x == 0.0 ? 0.0 : x * log(y); }

double or_lik_divergence(int kind, double x, double y, double par, double n) {
    switch (kind) {
        case 1: return xlogy(par + x, par + y) - xlogy(x, y);
        case 2: return n * log1p(y) - xlogy(x, y);
        case 3: {
            const double m = 0.5 * (x + y);
            return 0.5 * (xlogy(x, x) + xlogy(y, y)) - xlogy(m, m);
        }
        default: return NAN;
    }
}

static void lik_ab(int kind, double x, double y, double par, double n, double* a, double* b) {
    switch (kind) {
        case 1: *a = x / y; *b = (par + x) / (par + y); break;
        case 2: *a = x / y; *b = n / (1.0 + y); break;
        case 3: *a = log((x + y) / (2.0 * y)); *b = 1.0; break;
        default: *a = NAN; *b = NAN; break;
    }
}

static double lik_ginv(int kind, double z) { return kind == 3 ? exp(z) : z; }

void or_lik_weights(int64_t n, const double* y, const uint8_t* mask, const double* ntr,
                    const double* yhat, int kind, double par, double* wa, double* wb) {
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < n; ++e) {
        if (mask && !mask[e]) { wa[e] = 0.0; wb[e] = 0.0; continue; }
        lik_ab(kind, y[e], yhat[e], par, ntr ? ntr[e] : 1.0, &wa[e], &wb[e]);
    }
}

double or_lik_loss(const or_spec* s, const double* y, const uint8_t* mask, const double* ntr,
                   const double* const* fac, int kind, double par, int64_t* cnt) {
    int64_t n = y_size(s);
    double* yhat = (double*)malloc(sizeof(double) * n);
    or_reconstruct(s, fac, yhat);
    double tot = 0.0;
    int64_t c = 0;
    for (int64_t e = 0; e < n; ++e) {
        if (mask && !mask[e]) continue;
        tot += or_lik_divergence(kind, y[e], yhat[e], par, ntr ? ntr[e] : 1.0);
        ++c;
    }
    free(yhat);
    if (cnt) *cnt = c;
    return tot;
}

/* One factor update under a likelihood loss: the same three steps as
 * or_update_factor with the weights and g of the chosen kind. */
int or_lik_update_factor(const or_spec* s, int l, const double* y, const uint8_t* mask,
                         const double* ntr, double* const* fac, int kind, double par, double eps,
                         double* num_out, double* den_out) {
    if (kind < 1 || kind > 3) return 1;
    int64_t n = y_size(s);
    int64_t nl = fac_size(s, l);
    double* yhat = (double*)malloc(sizeof(double) * n);
    double* wa = (double*)malloc(sizeof(double) * n);
    double* wb = (double*)malloc(sizeof(double) * n);
    double* num = num_out ? num_out : (double*)malloc(sizeof(double) * nl);
    double* den = den_out ? den_out : (double*)malloc(sizeof(double) * nl);
    if (!yhat || !wa || !wb || !num || !den) return 2;
    or_reconstruct(s, (const double* const*)fac, yhat);
    or_lik_weights(n, y, mask, ntr, yhat, kind, par, wa, wb);
    or_einstr(s, l, wa, (const double* const*)fac, num);
    or_einstr(s, l, wb, (const double* const*)fac, den);
    for (int64_t e = 0; e < nl; ++e) {
        if (den[e] == 0.0) continue;
        const double v = fac[l][e] * lik_ginv(kind, num[e] / den[e]);
        fac[l][e] = v > eps ? v : eps;
    }
    free(yhat); free(wa); free(wb);
    if (!num_out) free(num);
    if (!den_out) free(den);
    return 0;
}

/* Algorithm 1 under a likelihood loss; trace as in or_fit. */
int or_lik_fit(const or_spec* s, const double* y, const uint8_t* mask, const double* ntr,
               double* const* fac, int kind, double par, double eps, int iters, double* trace) {
    if (kind < 1 || kind > 3) return 1;
    if (trace) trace[0] = or_lik_loss(s, y, mask, ntr, (const double* const*)fac, kind, par, NULL);
    for (int it = 0; it < iters; ++it) {
        for (int l = 0; l < s->n_fac; ++l) {
            int rc = or_lik_update_factor(s, l, y, mask, ntr, fac, kind, par, eps, NULL, NULL);
            if (rc) return rc;
        }
        if (trace) trace[it + 1] = or_lik_loss(s, y, mask, ntr, (const double* const*)fac, kind, par, NULL);
    }
    return 0;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
