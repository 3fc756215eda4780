/*
 * vrs_oracle.c -- CPU oracle for exact filtered top-k vector search.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or helper with the CUDA library, and the library never
 * calls it.
 *
 * Everything is computed in float64 from the *stored* input values (float32
 * arrays; bf16-stored data is passed in decoded).  Each routine cites the
 * passage of the paper (arXiv 2403.15807, "Efficient Data Access Paths for
 * Mixed Vector-Relational Search") it follows:
 *
 *   Sec. 3, "Brute force similarity search with relational predicate theta":
 *       sigma_{eps,v,theta_R}(R) = sigma_eps(v x sigma_{theta_R}(R))
 *       -> vrs_oracle_predicate (sigma_theta_R), vrs_oracle_compact,
 *          vrs_oracle_query (sigma_eps over the selected rows, top-k form),
 *          vrs_oracle_range (sigma_eps with eps a bound on the score).
 *   Sec. 2.2 / Sec. 5 "Vector Index": results are retrieved as a top-k.
 *   Sec. 3.1: cosine = dot product of normalised vectors -> metric IP.
 *
 * Readings of what the paper leaves open (listed in the design notes too):
 *   - L2 is reported squared, computed in the direct form sum_t (q_t-x_t)^2.
 *   - IP ranks by larger q.x; internally key = -q.x, reported value = q.x.
 *   - ties are broken by the smaller row id; rows are numbered by position.
 *   - predicate terms are half-open ranges lo <= a < hi; 0 terms = all rows.
 *   - fewer than k qualifying rows: pad with id -1 and distance +inf.
 *
 * The number-format helpers (bf16, FP8 E4M3) and the MLP plan model are
 * oracle pieces for the precision and learned-plan parts of the library;
 * they have no counterpart in the paper and say so where they are defined.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Relational predicate theta_R (Sec. 3, eq. "Brute force similarity search  */
/* with relational predicate"; Sec. 3.2 predicate pushdown).                 */
/* ------------------------------------------------------------------------ */

/* Does row i satisfy the conjunction of the n_terms ranges? */
static int row_qualifies(const int32_t *attrs, int64_t n, int64_t i, int32_t n_terms,
                         const int32_t *cols, const int32_t *lo, const int32_t *hi) {
    for (int32_t t = 0; t < n_terms; ++t) {
        int32_t a = attrs[(int64_t)cols[t] * n + i];
        if (!(lo[t] <= a && a < hi[t])) return 0;
    }
    return 1;
}

/* bitmap: uint32 words, row i is bit (i % 32) of word (i / 32); bits past n
 * are zero.  Returns |S|, the number of qualifying rows. */
ORACLE_API int64_t vrs_oracle_predicate(const int32_t *attrs, int64_t n, int32_t n_terms,
                                        const int32_t *cols, const int32_t *lo,
                                        const int32_t *hi, uint32_t *bitmap) {
    int64_t words = (n + 31) / 32, count = 0;
    for (int64_t w = 0; w < words; ++w) bitmap[w] = 0u;
    for (int64_t i = 0; i < n; ++i) {
        if (row_qualifies(attrs, n, i, n_terms, cols, lo, hi)) {
            bitmap[i / 32] |= (uint32_t)1u << (i % 32);
            ++count;
        }
    }
    return count;
}

/* Late materialisation (Sec. 3.2, predicate-first strategy): the positions
 * of the qualifying rows in ascending order.  Returns the count. */
ORACLE_API int64_t vrs_oracle_compact(const uint32_t *bitmap, int64_t n, int32_t *ids) {
    int64_t c = 0;
    for (int64_t i = 0; i < n; ++i)
        if ((bitmap[i / 32] >> (i % 32)) & 1u) ids[c++] = (int32_t)i;
    return c;
}

/* ------------------------------------------------------------------------ */
/* Distance and exact top-k (Sec. 3 eqs., Sec. 3.1)                         */
/* ------------------------------------------------------------------------ */

typedef struct { double key; int64_t id; } pair_t;

static int pair_cmp(const void *a, const void *b) {
    const pair_t *x = (const pair_t *)a, *y = (const pair_t *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* metric 0: squared L2, direct form; metric 1: inner product, key = -q.x */
static double key_of(const float *q, const float *x, int32_t d, int metric) {
    double s = 0.0;
    if (metric == 0) {
        for (int32_t t = 0; t < d; ++t) {
            double diff = (double)q[t] - (double)x[t];
            s += diff * diff;
        }
        return s;
    }
    for (int32_t t = 0; t < d; ++t) s += (double)q[t] * (double)x[t];
    return -s;
}

typedef struct {
    const float *x; int64_t n; int32_t d;
    const int32_t *attrs;
    const float *q; int32_t b;
    const int32_t *poff, *pcols, *plo, *phi; int32_t n_preds;
    const int32_t *k; int32_t n_k; int32_t k_max;
    int metric;
    int64_t *out_ids; double *out_dist; int64_t *out_count;
    int32_t next;              /* next query to take (under mu) */
    pthread_mutex_t mu;
} job_t;

static void one_query(job_t *J, int32_t qi, pair_t *buf) {
    int32_t p = J->n_preds == 1 ? 0 : qi;
    int32_t t0 = J->poff[p], nt = J->poff[p + 1] - t0;
    const float *q = J->q + (int64_t)qi * J->d;
    int64_t m = 0;
    /* S = sigma_theta(R), then eps evaluated on v x S */
    for (int64_t i = 0; i < J->n; ++i) {
        if (!row_qualifies(J->attrs, J->n, i, nt, J->pcols + t0, J->plo + t0, J->phi + t0))
            continue;
        buf[m].key = key_of(q, J->x + i * J->d, J->d, J->metric);
        buf[m].id = i;
        ++m;
    }
    qsort(buf, (size_t)m, sizeof(pair_t), pair_cmp);
    int32_t k = J->n_k == 1 ? J->k[0] : J->k[qi];
    if (J->out_count) J->out_count[qi] = m;
    for (int32_t j = 0; j < J->k_max; ++j) {
        int64_t o = (int64_t)qi * J->k_max + j;
        if (j < k && j < m) {
            J->out_ids[o] = buf[j].id;
            J->out_dist[o] = J->metric == 0 ? buf[j].key : -buf[j].key;
        } else {
            J->out_ids[o] = -1;
            J->out_dist[o] = INFINITY;
        }
    }
}

static void *worker(void *arg) {
    job_t *J = (job_t *)arg;
    pair_t *buf = (pair_t *)malloc(sizeof(pair_t) * (size_t)(J->n > 0 ? J->n : 1));
    if (!buf) return (void *)1;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int32_t qi = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (qi >= J->b) break;
        one_query(J, qi, buf);
    }
    free(buf);
    return NULL;
}

/*
 * Exact filtered top-k for a batch of queries.
 *   x      [n x d] float32 stored values, row-major; attrs [n_cols x n] int32
 *   q      [b x d] float32
 *   predicates in CSR form: terms of predicate p are poff[p] .. poff[p+1]-1;
 *          n_preds == 1: every query uses predicate 0; else n_preds == b
 *   k      per-query k (n_k == 1: shared), every k <= k_max
 *   out_ids [b x k_max] int64, out_dist [b x k_max] float64 (L2: squared
 *          distance; IP: q.x), out_count[b] = |S| per query (may be NULL)
 *   n_threads: worker threads across queries (>= 1)
 * Returns 0, or -1 if a thread could not allocate.
 */
ORACLE_API int vrs_oracle_query(const float *x, int64_t n, int32_t d, const int32_t *attrs,
                                const float *q, int32_t b, const int32_t *poff,
                                const int32_t *pcols, const int32_t *plo, const int32_t *phi,
                                int32_t n_preds, const int32_t *k, int32_t n_k, int32_t k_max,
                                int32_t metric, int64_t *out_ids, double *out_dist,
                                int64_t *out_count, int32_t n_threads) {
    job_t J = {x, n, d, attrs, q, b, poff, pcols, plo, phi, n_preds, k, n_k, k_max,
               metric, out_ids, out_dist, out_count, 0, PTHREAD_MUTEX_INITIALIZER};
    if (n_threads < 1) n_threads = 1;
    if (n_threads > b) n_threads = b > 0 ? b : 1;
    pthread_t th[256];
    if (n_threads > 256) n_threads = 256;
    int rc = 0;
    for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, worker, &J);
    for (int t = 0; t < n_threads; ++t) {
        void *r = NULL;
        pthread_join(th[t], &r);
        if (r) rc = -1;
    }
    return rc;
}

/*
 * Exact filtered range selection: sigma_eps applied with eps as a bound on the
 * score (Sec. 3, eq. "Brute force similarity search with relational predicate
 * theta": sigma_{eps,v,theta_R}(R) = sigma_eps(v x sigma_{theta_R}(R))), one
 * shared predicate.  Query qi keeps every selected row with squared L2
 * distance <= eps (metric 0) or q.x >= eps (metric 1).
 *   off[b+1]: CSR offsets of the results (always written); query qi's rows
 *             are ids/dist[off[qi] .. off[qi+1]), in (score, id) order:
 *             ascending distance for L2, descending q.x for IP, then id
 *   ids, dist: written only when the total fits cap (else may be NULL)
 * Returns the total number of results, or -1 if memory ran out.
 */
ORACLE_API int64_t vrs_oracle_range(const float *x, int64_t n, int32_t d, const int32_t *attrs,
                                    const float *q, int32_t b, int32_t n_terms,
                                    const int32_t *cols, const int32_t *lo, const int32_t *hi,
                                    double eps, int32_t metric, int64_t *off, int64_t *ids,
                                    double *dist, int64_t cap) {
    pair_t *buf = (pair_t *)malloc(sizeof(pair_t) * (size_t)(n > 0 ? n : 1));
    if (!buf) return -1;
    /* in key order (key = distance, or -q.x), a row passes when key <= ekey */
    const double ekey = metric == 0 ? eps : -eps;
    off[0] = 0;
    for (int32_t qi = 0; qi < b; ++qi) {
        const float *qv = q + (int64_t)qi * d;
        int64_t m = 0;
        for (int64_t i = 0; i < n; ++i) {
            if (!row_qualifies(attrs, n, i, n_terms, cols, lo, hi)) continue;
            double key = key_of(qv, x + i * d, d, metric);
            if (!(key <= ekey)) continue;
            buf[m].key = key;
            buf[m].id = i;
            ++m;
        }
        qsort(buf, (size_t)m, sizeof(pair_t), pair_cmp);
        off[qi + 1] = off[qi] + m;
        if (off[qi + 1] <= cap && ids && dist)
            for (int64_t j = 0; j < m; ++j) {
                ids[off[qi] + j] = buf[j].id;
                dist[off[qi] + j] = metric == 0 ? buf[j].key : -buf[j].key;
            }
    }
    free(buf);
    return off[b];
}

/* Exact score of given (query, row) pairs: the key_of() value reported the
 * way vrs_oracle_query reports it.  For sampled checks at sizes where the
 * full sort is too slow. */
ORACLE_API void vrs_oracle_pair_dist(const float *x, int32_t d, const float *q,
                                     const int64_t *qi, const int64_t *xi, int64_t m,
                                     int32_t metric, double *out) {
    for (int64_t j = 0; j < m; ++j) {
        double v = key_of(q + qi[j] * d, x + xi[j] * d, d, metric);
        out[j] = metric == 0 ? v : -v;
    }
}

/* ||x_i||^2 in float64, the definition the library's compensated float32
 * norms are held to (used in the L2 expansion ||q||^2 - 2 q.x + ||x||^2). */
ORACLE_API void vrs_oracle_sqnorm(const float *x, int64_t n, int32_t d, double *out) {
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int32_t t = 0; t < d; ++t) s += (double)x[i * d + t] * (double)x[i * d + t];
        out[i] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Number formats (no counterpart in the paper; used by the reduced-precision */
/* scan).  Written from the format definitions, not from any library.        */
/* ------------------------------------------------------------------------ */

/* bfloat16: 1 sign, 8 exponent (bias 127), 7 fraction bits.  Round to
 * nearest, ties to even, at 8 significant bits; the subnormal quantum is
 * 2^-133; overflow rounds to infinity; NaN maps to a quiet NaN. */
ORACLE_API uint16_t vrs_oracle_bf16_encode(float v) {
    if (isnan(v)) return 0x7FC0;
    double a = fabs((double)v);
    uint16_t sign = signbit(v) ? 0x8000 : 0;
    if (a == 0.0) return sign;
    if (isinf(v)) return sign | 0x7F80;
    int e;
    frexp(a, &e);                   /* a = f * 2^e, f in [0.5, 1) */
    int ex = e - 1;                 /* a in [2^ex, 2^(ex+1)) */
    if (ex < -126) ex = -126;
    double quantum = ldexp(1.0, ex - 7);
    double r = nearbyint(a / quantum) * quantum;   /* ties to even */
    if (r >= ldexp(1.0, 128)) return sign | 0x7F80;
    /* r is exactly representable as float; take its upper 16 bits */
    float rf = (float)r;
    uint32_t bits;
    memcpy(&bits, &rf, 4);
    return sign | (uint16_t)(bits >> 16);
}

ORACLE_API float vrs_oracle_bf16_decode(uint16_t h) {
    uint32_t bits = (uint32_t)h << 16;
    float f;
    memcpy(&f, &bits, 4);
    return f;
}

/* FP8 E4M3 (OCP 8-bit floating point, "E4M3FN"): 1 sign, 4 exponent (bias
 * 7), 3 mantissa bits; no infinities; S.1111.111 is NaN; largest finite
 * 448 = 1.75 * 2^8; smallest normal 2^-6; subnormals m/8 * 2^-6.
 * Encoding: round to nearest, ties to even, saturating to +-448 ("satfinite":
 * finite overflow and infinities clamp to the largest finite). */
ORACLE_API uint8_t vrs_oracle_e4m3_encode(float v) {
    if (isnan(v)) return 0x7F;
    uint8_t sign = signbit(v) ? 0x80 : 0;
    double a = fabs((double)v);
    if (a >= 448.0) return sign | 0x7E;
    if (a < ldexp(1.0, -6)) {                  /* subnormal range, quantum 2^-9 */
        double m = nearbyint(a / ldexp(1.0, -9));   /* 0 .. 8 */
        return sign | (uint8_t)m;               /* m == 8 is the smallest normal */
    }
    int e;
    frexp(a, &e);
    int ex = e - 1;                             /* -6 .. 8 */
    double m = nearbyint(a / ldexp(1.0, ex - 3));   /* 8 .. 16 */
    if (m >= 16.0) { m = 8.0; ex += 1; }
    if (ex > 8 || (ex == 8 && m > 14.0)) return sign | 0x7E;
    return sign | (uint8_t)(((ex + 7) << 3) | ((int)m - 8));
}

ORACLE_API double vrs_oracle_e4m3_decode(uint8_t c) {
    int s = c >> 7, e = (c >> 3) & 15, m = c & 7;
    double v;
    if (e == 15 && m == 7) return NAN;
    if (e == 0) v = ldexp((double)m, -9);
    else v = ldexp(1.0 + m / 8.0, e - 7);
    return s ? -v : v;
}

/* Per-vector scaled E4M3 copy: scale_i = max_t |x_it| / 448 (float32; 1 if
 * the row is all zero), code_it = E4M3(x_it / scale_i) with the quotient
 * rounded to float32 first.  Decoded value = decode(code) * scale. */
ORACLE_API void vrs_oracle_e4m3_rows(const float *x, int64_t n, int32_t d, uint8_t *codes,
                                     float *scale) {
    for (int64_t i = 0; i < n; ++i) {
        float amax = 0.0f;
        for (int32_t t = 0; t < d; ++t) {
            float a = fabsf(x[i * d + t]);
            if (a > amax) amax = a;
        }
        float s = amax > 0.0f ? amax / 448.0f : 1.0f;
        scale[i] = s;
        for (int32_t t = 0; t < d; ++t) {
            volatile float qv = x[i * d + t] / s;   /* float32 quotient */
            codes[i * d + t] = vrs_oracle_e4m3_encode(qv);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Plan-selection MLP (no counterpart in the paper, which leaves access-path */
/* selection to "an optimizer (or a user)", Sec. 5.2 / 5.3 takeaways).       */
/* Network 6 -> 64 -> 64 -> 3, ReLU, linear output; loss = masked mean       */
/* squared error.  float64 throughout.                                       */
/* ------------------------------------------------------------------------ */

/* Parameter block layout (all row-major, float64):
 *   W1[h1 x in] b1[h1] W2[h2 x h1] b2[h2] W3[out x h2] b3[out] */
static int64_t mlp_nparams(int in, int h1, int h2, int out) {
    return (int64_t)h1 * in + h1 + (int64_t)h2 * h1 + h2 + (int64_t)out * h2 + out;
}

ORACLE_API int64_t vrs_oracle_mlp_nparams(int32_t in, int32_t h1, int32_t h2, int32_t out) {
    return mlp_nparams(in, h1, h2, out);
}

/* Forward for m samples: y[m x out].  Loss = sum_{j,o} mask*(y-t)^2 / sum mask
 * (0 if mask sums to 0).  If grad != NULL, also d loss / d params. */
ORACLE_API double vrs_oracle_mlp(const double *P, int32_t in, int32_t h1, int32_t h2,
                                 int32_t out, const double *X, int64_t m, const double *T,
                                 const double *mask, double *Y, double *grad) {
    const double *W1 = P, *b1 = W1 + (int64_t)h1 * in, *W2 = b1 + h1, *b2 = W2 + (int64_t)h2 * h1,
                 *W3 = b2 + h2, *b3 = W3 + (int64_t)out * h2;
    double *gW1 = NULL, *gb1 = NULL, *gW2 = NULL, *gb2 = NULL, *gW3 = NULL, *gb3 = NULL;
    if (grad) {
        memset(grad, 0, sizeof(double) * (size_t)mlp_nparams(in, h1, h2, out));
        gW1 = grad; gb1 = gW1 + (int64_t)h1 * in; gW2 = gb1 + h1; gb2 = gW2 + (int64_t)h2 * h1;
        gW3 = gb2 + h2; gb3 = gW3 + (int64_t)out * h2;
    }
    double msum = 0.0;
    if (T && mask)
        for (int64_t j = 0; j < m * out; ++j) msum += mask[j];
    double *a1 = (double *)malloc(sizeof(double) * (size_t)(h1 + h2 + out + h1 + h2 + out));
    double *a2 = a1 + h1, *y = a2 + h2, *d1 = y + out, *d2 = d1 + h1, *d3 = d2 + h2;
    double loss = 0.0;
    for (int64_t j = 0; j < m; ++j) {
        const double *xj = X + j * in;
        for (int r = 0; r < h1; ++r) {
            double s = b1[r];
            for (int c = 0; c < in; ++c) s += W1[(int64_t)r * in + c] * xj[c];
            a1[r] = s > 0.0 ? s : 0.0;
        }
        for (int r = 0; r < h2; ++r) {
            double s = b2[r];
            for (int c = 0; c < h1; ++c) s += W2[(int64_t)r * h1 + c] * a1[c];
            a2[r] = s > 0.0 ? s : 0.0;
        }
        for (int r = 0; r < out; ++r) {
            double s = b3[r];
            for (int c = 0; c < h2; ++c) s += W3[(int64_t)r * h2 + c] * a2[c];
            y[r] = s;
            if (Y) Y[j * out + r] = s;
        }
        if (!(T && mask) || msum == 0.0) continue;
        for (int r = 0; r < out; ++r) {
            double e = y[r] - T[j * out + r], w = mask[j * out + r];
            loss += w * e * e / msum;
            d3[r] = 2.0 * w * e / msum;
        }
        if (!grad) continue;
        for (int r = 0; r < out; ++r) {
            gb3[r] += d3[r];
            for (int c = 0; c < h2; ++c) gW3[(int64_t)r * h2 + c] += d3[r] * a2[c];
        }
        for (int c = 0; c < h2; ++c) {
            double s = 0.0;
            for (int r = 0; r < out; ++r) s += W3[(int64_t)r * h2 + c] * d3[r];
            d2[c] = a2[c] > 0.0 ? s : 0.0;
        }
        for (int r = 0; r < h2; ++r) {
            gb2[r] += d2[r];
            for (int c = 0; c < h1; ++c) gW2[(int64_t)r * h1 + c] += d2[r] * a1[c];
        }
        for (int c = 0; c < h1; ++c) {
            double s = 0.0;
            for (int r = 0; r < h2; ++r) s += W2[(int64_t)r * h1 + c] * d2[r];
            d1[c] = a1[c] > 0.0 ? s : 0.0;
        }
        for (int r = 0; r < h1; ++r) {
            gb1[r] += d1[r];
            for (int c = 0; c < in; ++c) gW1[(int64_t)r * in + c] += d1[r] * xj[c];
        }
    }
    free(a1);
    return loss;
}

/* One Adam step (Kingma & Ba, 2015, Algorithm 1) on np parameters, in place.
 * t is the 1-based step number. */
ORACLE_API void vrs_oracle_adam(double *P, const double *g, double *m1, double *m2, int64_t np,
                                int32_t t, double lr, double beta1, double beta2, double eps) {
    double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
    for (int64_t i = 0; i < np; ++i) {
        m1[i] = beta1 * m1[i] + (1.0 - beta1) * g[i];
        m2[i] = beta2 * m2[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = m1[i] / c1, vh = m2[i] / c2;
        P[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
