/*
 * oracle.c -- plain, slow, single-threaded CPU statement of NN-sort
 * (Zhu, Zhang, Zhou, Liu: "Deep Learning Service for Efficient Data Distribution Aware Sorting",
 *  arXiv 1907.08817).
 *
 * TEST INFRASTRUCTURE ONLY. The product library never links, loads or calls this file. Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark use it, as the reference the
 * CUDA path is compared against. It shares no code, header, table or constant generator with the
 * CUDA path.
 *
 * What each part follows:
 *   - translate(A): Sec. "Input Phase" (the translate step of Fig. "Algorithm NN-sort"): keys are encoded as
 *     model inputs; numeric keys are min-max normalised with the training sample's range.
 *   - the model f and its training: Sec. "Training" and Sec. "Experimental Study / Training details"
 *     (regression MLP, rounding to a position, Adam; Huber loss of Eq. (loss)).
 *   - slots: pos = round(w_pos * m) of Fig. "Algorithm NN-sort", with w_pos = F(x) * n the
 *     expected position and m the relaxation factor.
 *   - rounds, conflict arrays, threshold tau and limit eps: Fig. "Algorithm NN-sort" and
 *     Sec. "Sorting Phase".
 *   - leftover sort and polish: Fig. "Algorithm polish", Sec. "Polish Phase" and its Remark.
 *   - stats: conflict rate sigma_i and out-of-order rate e_i of Sec. "Model Analysis";
 *     traditional sorting rate of Eq. (ratio).
 *
 * Parity-relevant floating point is written with explicit fmaf / ordinary IEEE binary32
 * operations in a fixed order; this file must be compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_ROUNDS 8
#define ORC_EMPTY 0xFFFFFFFFu

enum { ORC_F32 = 0, ORC_F64 = 1, ORC_U32 = 2, ORC_U64 = 3 };
enum { ORC_ORDBITS = 0, ORC_VALUE = 1 };
enum { ORC_MSE = 0, ORC_HUBER = 1 };

/* ------------------------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used counter-style: draw i of stream `seed` is  */
/* the output function applied to seed + (i+1)*gamma.                                         */
/* ------------------------------------------------------------------------------------------ */
uint64_t orc_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t orc_rng(uint64_t seed, uint64_t i) { return orc_mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ull); }

uint64_t orc_stream_seed(uint64_t seed, uint64_t tag) { return orc_rng(seed, tag); }

/* uniform index in [0, n): floor(u * n / 2^64) */
static uint64_t uidx(uint64_t u, uint64_t n) { return (uint64_t)(((__uint128_t)u * n) >> 64); }

static double unit53(uint64_t u) { return (double)(u >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------------------------------------ */
/* Key order. Keys are compared by their order-preserving unsigned image: IEEE floats map to    */
/* integers whose unsigned order is the numeric order, with -0.0 ordered before +0.0; unsigned  */
/* keys are their own image. Ties between equal keys are broken by original row.               */
/* ------------------------------------------------------------------------------------------ */
uint64_t orc_ordbits(const void *keys, int dtype, uint64_t i) {
    switch (dtype) {
    case ORC_F32: {
        uint32_t b;
        memcpy(&b, (const char *)keys + 4 * i, 4);
        return (b & 0x80000000u) ? (uint64_t)(uint32_t)~b : (uint64_t)(b | 0x80000000u);
    }
    case ORC_F64: {
        uint64_t b;
        memcpy(&b, (const char *)keys + 8 * i, 8);
        return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
    }
    case ORC_U32: return ((const uint32_t *)keys)[i];
    default: return ((const uint64_t *)keys)[i];
    }
}

static int key_size(int dtype) { return (dtype == ORC_F32 || dtype == ORC_U32) ? 4 : 8; }

static int is_nan_key(const void *keys, int dtype, uint64_t i) {
    if (dtype == ORC_F32) { float v; memcpy(&v, (const char *)keys + 4 * i, 4); return v != v; }
    if (dtype == ORC_F64) { double v; memcpy(&v, (const char *)keys + 8 * i, 8); return v != v; }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* translate(A): normalisation of a key into the model's input range.                          */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t dtype;      /* key type */
    int32_t translate;  /* ORC_ORDBITS or ORC_VALUE */
    uint64_t lo_bits;   /* order image of the smallest training key */
    double lo_val;      /* value of the smallest training key (VALUE mode) */
    double scale;       /* 1 / (hi - lo) in the translate's own units, 1 if hi == lo */
    float lo_f;         /* (float)lo_val */
    float scale_f;      /* (float)scale */
} orc_norm;

static double key_value(const void *keys, int dtype, uint64_t i) {
    switch (dtype) {
    case ORC_F32: return (double)((const float *)keys)[i];
    case ORC_F64: return ((const double *)keys)[i];
    case ORC_U32: return (double)((const uint32_t *)keys)[i];
    default: return (double)((const uint64_t *)keys)[i];
    }
}

/* VALUE mode on integer keys is the same map as ORDBITS (their image is the value). */
static int uses_ordbits(const orc_norm *nm) {
    return nm->translate == ORC_ORDBITS || nm->dtype == ORC_U32 || nm->dtype == ORC_U64;
}

/* The model input in binary32, bit-defined:
 *   ORDBITS: d = image - lo_bits as an exact signed integer; x = float(d) * scale_f
 *            (int -> float conversion rounds to nearest).
 *   VALUE, f32 keys: x = (key - lo_f) * scale_f in binary32.
 *   VALUE, f64 keys: x = float((key - lo_val) * scale) in binary64, rounded once to binary32. */
float orc_translate1_f32(const void *keys, int dtype, uint64_t i, const orc_norm *nm) {
    if (uses_ordbits(nm)) {
        uint64_t u = orc_ordbits(keys, dtype, i);
        float d = (u >= nm->lo_bits) ? (float)(u - nm->lo_bits) : -(float)(nm->lo_bits - u);
        return d * nm->scale_f;
    }
    if (dtype == ORC_F32) {
        float k = ((const float *)keys)[i];
        float d = k - nm->lo_f;
        return d * nm->scale_f;
    }
    double k = ((const double *)keys)[i];
    return (float)((k - nm->lo_val) * nm->scale);
}

/* The same normalisation in binary64 (reference input for displacement reports). */
double orc_translate1_f64(const void *keys, int dtype, uint64_t i, const orc_norm *nm) {
    if (uses_ordbits(nm)) {
        uint64_t u = orc_ordbits(keys, dtype, i);
        double d = (u >= nm->lo_bits) ? (double)(u - nm->lo_bits) : -(double)(nm->lo_bits - u);
        return d * nm->scale;
    }
    return (key_value(keys, dtype, i) - nm->lo_val) * nm->scale;
}

void orc_translate_f32(const void *keys, int dtype, uint64_t n, const orc_norm *nm, float *x) {
    for (uint64_t i = 0; i < n; ++i) x[i] = orc_translate1_f32(keys, dtype, i, nm);
}

void orc_translate_f64(const void *keys, int dtype, uint64_t n, const orc_norm *nm, double *x) {
    for (uint64_t i = 0; i < n; ++i) x[i] = orc_translate1_f64(keys, dtype, i, nm);
}

/* Normaliser from a sample: lo/hi are the sample's smallest and largest keys. */
void orc_make_norm(const void *keys, int dtype, const uint64_t *idx, uint64_t S, int translate,
                   orc_norm *out) {
    memset(out, 0, sizeof(*out));
    out->dtype = dtype;
    out->translate = translate;
    uint64_t lo = ~0ull, hi = 0, ilo = 0;
    for (uint64_t j = 0; j < S; ++j) {
        uint64_t u = orc_ordbits(keys, dtype, idx[j]);
        if (u < lo) { lo = u; ilo = idx[j]; }
        if (u > hi) hi = u;
    }
    if (S == 0) { lo = hi = 0; }
    out->lo_bits = lo;
    out->lo_val = S ? key_value(keys, dtype, ilo) : 0.0;
    if (uses_ordbits(out)) {
        out->scale = (hi > lo) ? 1.0 / (double)(hi - lo) : 1.0;
    } else {
        /* hi value is the key with the largest image */
        double hv = out->lo_val;
        for (uint64_t j = 0; j < S; ++j)
            if (orc_ordbits(keys, dtype, idx[j]) == hi) { hv = key_value(keys, dtype, idx[j]); break; }
        out->scale = (hv > out->lo_val) ? 1.0 / (hv - out->lo_val) : 1.0;
    }
    out->lo_f = (float)out->lo_val;
    out->scale_f = (float)out->scale;
}

/* ------------------------------------------------------------------------------------------ */
/* The model f: a ReLU MLP 1 -> H1 [-> H2] -> 1.                                                 */
/* Flat parameter layout, one hidden layer:  W1[H1] b1[H1] W3[H1] b3                            */
/*                        two hidden layers: W1[H1] b1[H1] W2[H2*H1] (row k = unit k) b2[H2]    */
/*                                           W3[H2] b3                                          */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int32_t layers; /* hidden layers: 1 or 2 */
    int32_t h1, h2;
} orc_arch;

uint64_t orc_num_params(const orc_arch *a) {
    if (a->layers == 1) return 3ull * a->h1 + 1;
    return 2ull * a->h1 + (uint64_t)a->h2 * a->h1 + 2ull * a->h2 + 1;
}

static float relu_f(float v) { return (v > 0.0f) ? v : 0.0f; }
static double relu_d(double v) { return (v > 0.0) ? v : 0.0; }

/* binary32 forward; every dot product accumulates left to right with one fmaf per term,
 * starting from the bias. */
float orc_mlp1_f32(const orc_arch *a, const float *p, float x) {
    float h1[256], h2[256];
    const int H1 = a->h1, H2 = a->h2;
    const float *W1 = p, *b1 = p + H1;
    for (int j = 0; j < H1; ++j) h1[j] = relu_f(fmaf(W1[j], x, b1[j]));
    const float *hl = h1;
    int HL = H1;
    const float *W3;
    float b3;
    if (a->layers == 2) {
        const float *W2 = p + 2 * H1, *b2 = W2 + (size_t)H2 * H1;
        for (int k = 0; k < H2; ++k) {
            float z = b2[k];
            for (int j = 0; j < H1; ++j) z = fmaf(W2[(size_t)k * H1 + j], h1[j], z);
            h2[k] = relu_f(z);
        }
        hl = h2;
        HL = H2;
        W3 = b2 + H2;
    } else {
        W3 = p + 2 * H1;
    }
    b3 = W3[HL];
    float y = b3;
    for (int k = 0; k < HL; ++k) y = fmaf(W3[k], hl[k], y);
    return y;
}

double orc_mlp1_f64(const orc_arch *a, const double *p, double x) {
    double h1[256], h2[256];
    const int H1 = a->h1, H2 = a->h2;
    const double *W1 = p, *b1 = p + H1;
    for (int j = 0; j < H1; ++j) h1[j] = relu_d(fma(W1[j], x, b1[j]));
    const double *hl = h1;
    int HL = H1;
    const double *W3;
    if (a->layers == 2) {
        const double *W2 = p + 2 * H1, *b2 = W2 + (size_t)H2 * H1;
        for (int k = 0; k < H2; ++k) {
            double z = b2[k];
            for (int j = 0; j < H1; ++j) z = fma(W2[(size_t)k * H1 + j], h1[j], z);
            h2[k] = relu_d(z);
        }
        hl = h2;
        HL = H2;
        W3 = b2 + H2;
    } else {
        W3 = p + 2 * H1;
    }
    double y = W3[HL];
    for (int k = 0; k < HL; ++k) y = fma(W3[k], hl[k], y);
    return y;
}

/* Hidden layer 1 activations relu(fmaf(W1_j, x, b1_j)) in binary32, row-major [n][h1]. */
void orc_mlp_layer1_f32(const orc_arch *a, const float *p, const float *x, uint64_t n, float *h) {
    for (uint64_t i = 0; i < n; ++i)
        for (int j = 0; j < a->h1; ++j) h[i * a->h1 + j] = relu_f(fmaf(p[j], x[i], p[a->h1 + j]));
}

void orc_mlp_forward_f32(const orc_arch *a, const float *p, const float *x, uint64_t n, float *y) {
    for (uint64_t i = 0; i < n; ++i) y[i] = orc_mlp1_f32(a, p, x[i]);
}

void orc_mlp_forward_f64(const orc_arch *a, const double *p, const double *x, uint64_t n, double *y) {
    for (uint64_t i = 0; i < n; ++i) y[i] = orc_mlp1_f64(a, p, x[i]);
}

/* Per-sample loss and its derivative with respect to the model output r = y - label.
 * MSE: r^2. Huber (Eq. (loss)): r^2/2 if |r| <= delta, else delta*|r| - delta^2/2. */
static double loss_val(int loss, double r, double delta) {
    if (loss == ORC_HUBER) {
        double ar = fabs(r);
        return (ar <= delta) ? 0.5 * r * r : delta * ar - 0.5 * delta * delta;
    }
    return r * r;
}

static double loss_der(int loss, double r, double delta) {
    if (loss == ORC_HUBER) {
        if (r > delta) return delta;
        if (r < -delta) return -delta;
        return r;
    }
    return 2.0 * r;
}

/* Mean loss over the n samples and its exact gradient (binary64 backpropagation).
 * grad has orc_num_params entries; gx (nullable) receives d(mean loss)/dx per sample. */
double orc_mlp_loss_grad_f64(const orc_arch *a, const double *p, const double *x,
                             const double *label, uint64_t n, int loss, double delta,
                             double *grad, double *gx) {
    const int H1 = a->h1, H2 = a->h2;
    const uint64_t P = orc_num_params(a);
    memset(grad, 0, P * sizeof(double));
    if (n == 0) return 0.0;
    const double *W1 = p, *b1 = p + H1;
    const double *W2 = p + 2 * H1, *b2 = W2 + (size_t)H2 * H1;
    const double *W3 = (a->layers == 2) ? b2 + H2 : p + 2 * H1;
    const int HL = (a->layers == 2) ? H2 : H1;
    double *gW1 = grad, *gb1 = grad + H1;
    double *gW2 = grad + 2 * H1, *gb2 = gW2 + (size_t)H2 * H1;
    double *gW3 = (a->layers == 2) ? gb2 + H2 : grad + 2 * H1;
    double a1[256], h1[256], a2[256], h2[256], d1[256], d2[256];
    double total = 0.0;
    const double inv_n = 1.0 / (double)n;
    for (uint64_t i = 0; i < n; ++i) {
        const double xi = x[i];
        for (int j = 0; j < H1; ++j) { a1[j] = fma(W1[j], xi, b1[j]); h1[j] = relu_d(a1[j]); }
        const double *hl = h1;
        if (a->layers == 2) {
            for (int k = 0; k < H2; ++k) {
                double z = b2[k];
                for (int j = 0; j < H1; ++j) z = fma(W2[(size_t)k * H1 + j], h1[j], z);
                a2[k] = z;
                h2[k] = relu_d(z);
            }
            hl = h2;
        }
        double y = W3[HL];
        for (int k = 0; k < HL; ++k) y = fma(W3[k], hl[k], y);
        const double r = y - label[i];
        total += loss_val(loss, r, delta);
        const double gy = loss_der(loss, r, delta) * inv_n;
        /* output layer */
        for (int k = 0; k < HL; ++k) gW3[k] += gy * hl[k];
        gW3[HL] += gy;
        if (a->layers == 2) {
            for (int k = 0; k < H2; ++k) d2[k] = (a2[k] > 0.0) ? gy * W3[k] : 0.0;
            for (int j = 0; j < H1; ++j) d1[j] = 0.0;
            for (int k = 0; k < H2; ++k) {
                if (d2[k] == 0.0) continue;
                gb2[k] += d2[k];
                for (int j = 0; j < H1; ++j) {
                    gW2[(size_t)k * H1 + j] += d2[k] * h1[j];
                    d1[j] += d2[k] * W2[(size_t)k * H1 + j];
                }
            }
            for (int j = 0; j < H1; ++j) d1[j] = (a1[j] > 0.0) ? d1[j] : 0.0;
        } else {
            for (int j = 0; j < H1; ++j) d1[j] = (a1[j] > 0.0) ? gy * W3[j] : 0.0;
        }
        double gxi = 0.0;
        for (int j = 0; j < H1; ++j) {
            gW1[j] += d1[j] * xi;
            gb1[j] += d1[j];
            gxi += d1[j] * W1[j];
        }
        if (gx) gx[i] = gxi;
    }
    return total * inv_n;
}

/* Adam (Kingma & Ba), bias-corrected, one step; `step` counts from 1. */
void orc_adam_f64(double *p, const double *g, double *m, double *v, uint64_t P, uint64_t step,
                  double lr, double b1, double b2, double eps) {
    const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
    for (uint64_t i = 0; i < P; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        const double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}

/* Initial parameters from stream TAG_INIT of `seed`, rounded to binary32.
 * Hidden layer 1 has fan-in 1: W1_j ~ U(-sqrt6, sqrt6) and its kink is placed at c_j ~ U(0,1)
 * inside the normalised input range (b1_j = -W1_j c_j). Deeper weights are He-uniform,
 * U(-sqrt(6/fan_in), sqrt(6/fan_in)); their biases start at 0. */
#define TAG_SAMPLE 1
#define TAG_INIT 2
#define TAG_BATCH 3
void orc_init_params(const orc_arch *a, uint64_t seed, float *p) {
    const uint64_t s = orc_stream_seed(seed, TAG_INIT);
    const int H1 = a->h1, H2 = a->h2;
    uint64_t c = 0;
    const double r1 = sqrt(6.0);
    for (int j = 0; j < H1; ++j) p[j] = (float)((2.0 * unit53(orc_rng(s, c++)) - 1.0) * r1);
    for (int j = 0; j < H1; ++j) {
        const double cj = unit53(orc_rng(s, c++));
        p[H1 + j] = (float)(-(double)p[j] * cj);
    }
    float *q = p + 2 * H1;
    int HL = H1;
    if (a->layers == 2) {
        const double r2 = sqrt(6.0 / H1);
        for (int k = 0; k < H2 * H1; ++k) q[k] = (float)((2.0 * unit53(orc_rng(s, c++)) - 1.0) * r2);
        q += (size_t)H2 * H1;
        for (int k = 0; k < H2; ++k) q[k] = 0.0f;
        q += H2;
        HL = H2;
    }
    const double r3 = sqrt(6.0 / HL);
    for (int k = 0; k < HL; ++k) q[k] = (float)((2.0 * unit53(orc_rng(s, c++)) - 1.0) * r3);
    q[HL] = 0.0f;
}

/* ------------------------------------------------------------------------------------------ */
/* Training data (Sec. "Training"): a seeded sample of S keys drawn with replacement, sorted by */
/* (key, draw index); label_j = j / S is the empirical CDF at the j-th smallest sample key.      */
/* ------------------------------------------------------------------------------------------ */
static const void *g_cmp_keys;
static int g_cmp_dtype;
static const uint64_t *g_cmp_idx;

static int cmp_sample(const void *pa, const void *pb) {
    const uint64_t ja = *(const uint64_t *)pa, jb = *(const uint64_t *)pb;
    const uint64_t ua = orc_ordbits(g_cmp_keys, g_cmp_dtype, g_cmp_idx[ja]);
    const uint64_t ub = orc_ordbits(g_cmp_keys, g_cmp_dtype, g_cmp_idx[jb]);
    if (ua != ub) return ua < ub ? -1 : 1;
    return ja < jb ? -1 : (ja > jb ? 1 : 0);
}

/* Outputs (each nullable): sorted sample keys' order images, normaliser, binary32 model inputs,
 * binary32 labels. Returns 0, or -1 on a NaN key in the sample / bad arguments. */
int orc_sample_labels(const void *keys, int dtype, uint64_t n, uint64_t S, uint64_t seed, int translate,
                      uint64_t *sorted_rows, orc_norm *norm, float *x, float *label) {
    if (n == 0 || S == 0) return -1;
    uint64_t *idx = (uint64_t *)malloc(S * sizeof(uint64_t));
    uint64_t *ord = (uint64_t *)malloc(S * sizeof(uint64_t));
    const uint64_t s = orc_stream_seed(seed, TAG_SAMPLE);
    int rc = 0;
    for (uint64_t j = 0; j < S; ++j) {
        idx[j] = uidx(orc_rng(s, j), n);
        if (is_nan_key(keys, dtype, idx[j])) rc = -1;
        ord[j] = j;
    }
    if (rc == 0) {
        g_cmp_keys = keys; g_cmp_dtype = dtype; g_cmp_idx = idx;
        qsort(ord, S, sizeof(uint64_t), cmp_sample);
        uint64_t *rows = (uint64_t *)malloc(S * sizeof(uint64_t));
        for (uint64_t j = 0; j < S; ++j) rows[j] = idx[ord[j]];
        orc_norm nm;
        orc_make_norm(keys, dtype, rows, S, translate, &nm);
        if (norm) *norm = nm;
        for (uint64_t j = 0; j < S; ++j) {
            if (sorted_rows) sorted_rows[j] = rows[j];
            if (x) x[j] = orc_translate1_f32(keys, dtype, rows[j], &nm);
            if (label) label[j] = (float)((double)j / (double)S);
        }
        free(rows);
    }
    free(idx);
    free(ord);
    return rc;
}

/* Training in binary64 from the binary32 inputs and labels. batch == 0 is full-batch; otherwise
 * step t (0-based) uses samples uidx(rng(TAG_BATCH stream, t*batch + k), S), k < batch. */
typedef struct {
    orc_arch arch;
    int32_t translate;
    int32_t loss;
    double huber_delta;
    uint64_t sample_n;
    uint64_t steps;
    uint64_t batch;
    double lr, beta1, beta2, adam_eps;
    uint64_t seed;
    int32_t monotone;
} orc_train_opts;

/* Monotone option: every path from the input to the output gets a non-negative weight product,
 * so F is non-decreasing in x. Hidden unit j of layer 1 keeps the sign s_j of its initial input
 * weight; with one hidden layer W3_j must carry s_j; with two, output unit k keeps the sign q_k of
 * its initial W3_k and W2_kj must carry s_j q_k. sgn[i] is +1/-1 for constrained parameters and 0
 * for free ones (biases). */
void orc_monotone_signs(const orc_arch *a, const float *p0, double *sgn) {
    const int H1 = a->h1, H2 = a->h2;
    const uint64_t P = orc_num_params(a);
    for (uint64_t i = 0; i < P; ++i) sgn[i] = 0.0;
    for (int j = 0; j < H1; ++j) sgn[j] = (p0[j] >= 0.0f) ? 1.0 : -1.0;
    if (a->layers == 1) {
        for (int j = 0; j < H1; ++j) sgn[2 * H1 + j] = sgn[j];
    } else {
        const uint64_t w2 = 2 * (uint64_t)H1, w3 = w2 + (uint64_t)H2 * H1 + H2;
        for (int k = 0; k < H2; ++k) {
            const double q = (p0[w3 + k] >= 0.0f) ? 1.0 : -1.0;
            sgn[w3 + k] = q;
            for (int j = 0; j < H1; ++j) sgn[w2 + (uint64_t)k * H1 + j] = sgn[j] * q;
        }
    }
}

int orc_train(const void *keys, int dtype, uint64_t n, const orc_train_opts *o, orc_norm *norm_out,
              double *params_out, double *loss_hist) {
    const uint64_t S = o->sample_n < 1 ? 1 : o->sample_n;
    float *xf = (float *)malloc(S * sizeof(float));
    float *lf = (float *)malloc(S * sizeof(float));
    if (orc_sample_labels(keys, dtype, n, S, o->seed, o->translate, NULL, norm_out, xf, lf) != 0) {
        free(xf); free(lf);
        return -1;
    }
    const uint64_t P = orc_num_params(&o->arch);
    float *pf = (float *)malloc(P * sizeof(float));
    orc_init_params(&o->arch, o->seed, pf);
    double *m = (double *)calloc(P, sizeof(double)), *v = (double *)calloc(P, sizeof(double));
    double *g = (double *)malloc(P * sizeof(double));
    double *sgn = (double *)calloc(P, sizeof(double));
    if (o->monotone) {
        /* initial weights take the required signs (magnitudes kept) */
        orc_monotone_signs(&o->arch, pf, sgn);
        for (uint64_t i = 0; i < P; ++i)
            if (sgn[i] != 0.0) pf[i] = (float)(sgn[i] * fabs((double)pf[i]));
    }
    for (uint64_t i = 0; i < P; ++i) params_out[i] = (double)pf[i];
    const uint64_t B = o->batch ? o->batch : S;
    double *xb = (double *)malloc(B * sizeof(double)), *lb = (double *)malloc(B * sizeof(double));
    const uint64_t sb = orc_stream_seed(o->seed, TAG_BATCH);
    for (uint64_t t = 0; t < o->steps; ++t) {
        for (uint64_t k = 0; k < B; ++k) {
            const uint64_t j = o->batch ? uidx(orc_rng(sb, t * B + k), S) : k;
            xb[k] = (double)xf[j];
            lb[k] = (double)lf[j];
        }
        const double L = orc_mlp_loss_grad_f64(&o->arch, params_out, xb, lb, B, o->loss, o->huber_delta,
                                               g, NULL);
        if (loss_hist) loss_hist[t] = L;
        orc_adam_f64(params_out, g, m, v, P, t + 1, o->lr, o->beta1, o->beta2, o->adam_eps);
        if (o->monotone)  /* projection: a weight that crossed zero stops at zero */
            for (uint64_t i = 0; i < P; ++i)
                if (sgn[i] * params_out[i] < 0.0) params_out[i] = 0.0;
    }
    free(xf); free(lf); free(pf); free(m); free(v); free(g); free(xb); free(lb); free(sgn);
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Slots: pos = round(F * n * m) with round-half-up, clamped to [0, L-1], L = floor(n m) + 1.    */
/* Evaluated in binary32 with the product n*m carried as an unevaluated sum nm_hi + nm_lo, so    */
/* that y*nm is resolved below one slot even when n*m exceeds 2^24:                             */
/*   p = y*nm_hi; e = fma(y,nm_hi,-p) (exact); e = fma(y,nm_lo,e); f = floor(p);                */
/*   r = (p - f) + e; slot = f + floor(r + 0.5)                                                  */
/* y <= 0 (or NaN) maps to slot 0 and y is capped at 1 before the product.                     */
/* ------------------------------------------------------------------------------------------ */
void orc_nm_split(uint64_t n, float m, uint64_t *L, float *nm_hi, float *nm_lo) {
    const double nm = (double)n * (double)m;
    *L = (uint64_t)floor(nm) + 1;
    *nm_hi = (float)nm;
    *nm_lo = (float)(nm - (double)*nm_hi);
}

uint32_t orc_slot1(float y, float nm_hi, float nm_lo, uint64_t L) {
    if (!(y > 0.0f)) return 0;
    if (y > 1.0f) y = 1.0f;
    const float p = y * nm_hi;
    float e = fmaf(y, nm_hi, -p);
    e = fmaf(y, nm_lo, e);
    const float f = floorf(p);
    const float r = (p - f) + e;
    const float g = floorf(r + 0.5f);
    int64_t s = (int64_t)f + (int64_t)g;
    if (s < 0) s = 0;
    if ((uint64_t)s > L - 1) s = (int64_t)(L - 1);
    return (uint32_t)s;
}

/* translate -> binary32 MLP -> slot for every key; y_out (nullable) receives F(x). Returns -1 on
 * a NaN key. */
int orc_predict_slots(const void *keys, int dtype, uint64_t n, const orc_norm *nm, const orc_arch *a,
                      const float *params, float m, uint32_t *slots, float *y_out) {
    uint64_t L;
    float hi, lo;
    orc_nm_split(n, m, &L, &hi, &lo);
    for (uint64_t i = 0; i < n; ++i) {
        if (is_nan_key(keys, dtype, i)) return -1;
        const float y = orc_mlp1_f32(a, params, orc_translate1_f32(keys, dtype, i, nm));
        if (y_out) y_out[i] = y;
        slots[i] = orc_slot1(y, hi, lo, L);
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* NN-sort proper: Fig. "Algorithm NN-sort" + Fig. "Algorithm polish".                          */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    uint32_t t;   /* rounds completed */
    uint32_t eps; /* round limit */
    uint64_t n, L, tau;
    uint64_t w_size[ORC_MAX_ROUNDS + 1];    /* |w| entering round i+1 (w_size[0] = n); w_size[i] = |c_i| */
    uint64_t placed[ORC_MAX_ROUNDS];        /* elements stored in o_i */
    uint64_t out_of_order[ORC_MAX_ROUNDS];  /* elements of o_i inserted (not appended) by polish */
} orc_stats;

typedef struct {
    const void *keys;
    int dtype;
} elem_ctx;

/* (key, row) order */
static int elem_less(const elem_ctx *c, uint32_t a, uint32_t b) {
    const uint64_t ua = orc_ordbits(c->keys, c->dtype, a), ub = orc_ordbits(c->keys, c->dtype, b);
    if (ua != ub) return ua < ub;
    return a < b;
}

static elem_ctx g_sort_ctx;
static int cmp_rows(const void *pa, const void *pb) {
    const uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    if (elem_less(&g_sort_ctx, a, b)) return -1;
    if (elem_less(&g_sort_ctx, b, a)) return 1;
    return 0;
}

/* The leftover sort ("QuickSort(w)") and the reference sort: rows by (key, row). */
void orc_sort_rows(const void *keys, int dtype, uint32_t *rows, uint64_t cnt) {
    g_sort_ctx.keys = keys;
    g_sort_ctx.dtype = dtype;
    qsort(rows, cnt, sizeof(uint32_t), cmp_rows);
}

/* InsertSort(A', o_i) of Fig. "Algorithm polish": walk o_i's stored elements in position order;
 * an element no smaller than the last element appended from o_i is appended after every
 * remaining element of A' that precedes it; a smaller one is out of order and is inserted into
 * the result at its sorted place. Returns the number of inserted (out-of-order) elements. */
static uint64_t insert_sort_merge(const elem_ctx *c, const uint32_t *A, uint64_t na, const uint32_t *seq,
                                  uint64_t ns, uint32_t *out, int8_t *fate, int round) {
    uint64_t j = 0, len = 0, ooo = 0;
    int have_last = 0;
    uint32_t last = 0;
    for (uint64_t q = 0; q < ns; ++q) {
        const uint32_t x = seq[q];
        if (!have_last || !elem_less(c, x, last)) {
            while (j < na && elem_less(c, A[j], x)) out[len++] = A[j++];
            out[len++] = x;
            last = x;
            have_last = 1;
            if (fate) fate[x] = (int8_t)round;
        } else {
            /* binary search for the first result element greater than x */
            uint64_t lo = 0, hi = len;
            while (lo < hi) {
                const uint64_t mid = (lo + hi) / 2;
                if (elem_less(c, x, out[mid])) hi = mid; else lo = mid + 1;
            }
            memmove(out + lo + 1, out + lo, (len - lo) * sizeof(uint32_t));
            out[lo] = x;
            ++len;
            ++ooo;
            if (fate) fate[x] = (int8_t)(-round);
        }
    }
    while (j < na) out[len++] = A[j++];
    return ooo;
}

/* keys[n] (dtype), payload[n] nullable, slots[n] in [0, L): the model's positions (or injected).
 * Writes the sorted keys/payload to out_keys/out_payload (nullable), stats (nullable) and
 * fate[n] (nullable): +i placed in o_i and appended, -i placed in o_i and inserted, 0 sorted as
 * leftover. Returns 0, -1 on bad arguments, -2 on a slot outside [0, L). */
int orc_nnsort(const void *keys, int dtype, const int32_t *payload, uint64_t n, const uint32_t *slots,
               uint64_t L, int eps, uint64_t tau, void *out_keys, int32_t *out_payload, orc_stats *st,
               int8_t *fate) {
    if (eps < 0 || eps > ORC_MAX_ROUNDS || n >= 0xFFFFFFFFull) return -1;
    for (uint64_t i = 0; i < n; ++i)
        if (slots[i] >= L) return -2;
    orc_stats s;
    memset(&s, 0, sizeof(s));
    s.eps = (uint32_t)eps;
    s.n = n;
    s.L = L;
    s.tau = tau;
    s.w_size[0] = n;
    const elem_ctx c = {keys, dtype};
    if (fate) memset(fate, 0, n);

    uint32_t *w = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
    uint32_t *cbuf = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
    uint32_t *table = (uint32_t *)malloc((L + 1) * sizeof(uint32_t));
    uint32_t *seqs[ORC_MAX_ROUNDS];
    uint64_t seqn[ORC_MAX_ROUNDS];
    uint64_t wn = n;
    for (uint64_t i = 0; i < n; ++i) w[i] = (uint32_t)i; /* w <- translate(A), in input order */

    uint32_t i = 0;
    while (i < (uint32_t)eps && wn > tau) {              /* loop condition, read as i < eps */
        for (uint64_t q = 0; q < L; ++q) table[q] = ORC_EMPTY;
        uint64_t cn = 0;
        for (uint64_t q = 0; q < wn; ++q) {                 /* first element to reach a slot wins */
            const uint32_t r = w[q];
            const uint32_t pos = slots[r];
            if (table[pos] == ORC_EMPTY) table[pos] = r;
            else cbuf[cn++] = r;                            /* conflict array keeps arrival order */
        }
        uint64_t pn = 0;
        for (uint64_t q = 0; q < L; ++q) if (table[q] != ORC_EMPTY) ++pn;
        seqs[i] = (uint32_t *)malloc((pn + 1) * sizeof(uint32_t));
        seqn[i] = pn;
        pn = 0;
        for (uint64_t q = 0; q < L; ++q) if (table[q] != ORC_EMPTY) seqs[i][pn++] = table[q];
        s.placed[i] = pn;
        memcpy(w, cbuf, cn * sizeof(uint32_t));
        wn = cn;
        ++i;
        s.w_size[i] = wn;
    }
    s.t = i;

    /* QuickSort(w): the final conflict array, sorted by (key, row) */
    orc_sort_rows(keys, dtype, w, wn);

    /* polish(O, w): A' <- w; A' <- InsertSort(A', o_i) for o_1 .. o_t */
    uint32_t *A = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
    uint32_t *B = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
    memcpy(A, w, wn * sizeof(uint32_t));
    uint64_t an = wn;
    for (uint32_t r = 0; r < s.t; ++r) {
        s.out_of_order[r] = insert_sort_merge(&c, A, an, seqs[r], seqn[r], B, fate, (int)r + 1);
        an += seqn[r];
        uint32_t *tmp = A; A = B; B = tmp;
        free(seqs[r]);
    }
    const int ks = key_size(dtype);
    for (uint64_t q = 0; q < an; ++q) {
        if (out_keys) memcpy((char *)out_keys + q * ks, (const char *)keys + (uint64_t)A[q] * ks, ks);
        if (out_payload && payload) out_payload[q] = payload[A[q]];
    }
    if (st) *st = s;
    free(w); free(cbuf); free(table); free(A); free(B);
    return 0;
}

/* Whole method from keys: slots from the model, then orc_nnsort. Returns -1 on NaN keys. */
int orc_nnsort_model(const void *keys, int dtype, const int32_t *payload, uint64_t n, const orc_norm *nm,
                     const orc_arch *a, const float *params, float m, int eps, uint64_t tau,
                     void *out_keys, int32_t *out_payload, orc_stats *st, int8_t *fate) {
    uint32_t *slots = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
    int rc = orc_predict_slots(keys, dtype, n, nm, a, params, m, slots, NULL);
    if (rc == 0) {
        uint64_t L;
        float hi, lo;
        orc_nm_split(n, m, &L, &hi, &lo);
        rc = orc_nnsort(keys, dtype, payload, n, slots, L, eps, tau, out_keys, out_payload, st, fate);
    }
    free(slots);
    return rc;
}

/* Reference: the stable sort of the input by (key, row). */
void orc_stable_sort(const void *keys, int dtype, const int32_t *payload, uint64_t n, void *out_keys,
                     int32_t *out_payload) {
    uint32_t *rows = (uint32_t *)malloc((n + 1) * sizeof(uint32_t));
    for (uint64_t i = 0; i < n; ++i) rows[i] = (uint32_t)i;
    orc_sort_rows(keys, dtype, rows, n);
    const int ks = key_size(dtype);
    for (uint64_t q = 0; q < n; ++q) {
        memcpy((char *)out_keys + q * ks, (const char *)keys + (uint64_t)rows[q] * ks, ks);
        if (out_payload && payload) out_payload[q] = payload[rows[q]];
    }
    free(rows);
}
