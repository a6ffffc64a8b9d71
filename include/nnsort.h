/*
 * nnsort.h -- C ABI of the GB300 (sm_103a) NN-sort library (libnnsort.so).
 *
 * NN-sort (Zhu, Zhang, Zhou, Liu, "Deep Learning Service for Efficient Data Distribution Aware
 * Sorting", arXiv 1907.08817) sorts an array A by mapping every element through a learned model f
 * to an expected position, storing it at round(f(x) * m) of a roughly ordered array o_i if that
 * position is free, sending it to a conflict array otherwise, repeating on the conflict array while
 * fewer than eps iterations ran and it holds more than tau elements, sorting what is left
 * conventionally and merging everything in a polish phase that inserts out-of-order elements
 * (Sec. "Neural Network Based Sort", Fig. "Algorithm NN-sort", Fig. "Algorithm polish").
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are device pointers, h_* host pointers; sizes are element counts.
 *   - The caller owns every buffer it passes. The library owns models (until nnsort_model_free)
 *     and its internal workspace (until nnsort_release).
 *   - Work is enqueued on `stream`. Unless stated otherwise a call returns after enqueueing, and
 *     device outputs are valid once the stream has been synchronised.
 *   - Return value: NNSORT_OK (0) or a negative nnsort_status. No C++ exception crosses the ABI.
 *     When an error is detected before the first write to a caller buffer, the buffer is left
 *     unmodified.
 *   - Keys are ordered by value with a total order: IEEE floats by their sign-adjusted bit
 *     pattern (so -0.0 sorts before +0.0); NaN keys are rejected with NNSORT_E_NAN_KEY.
 *     Equal keys keep their input order (the sort is stable), which fixes the payload order.
 *   - Limits: n * m < 2^32 - 1 and n < 2^32 - 1.
 */
#ifndef NNSORT_H
#define NNSORT_H

#include <stddef.h>
#include <stdint.h>

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NNSORT_VERSION 10000
#define NNSORT_MAX_ROUNDS 8
#define NNSORT_MAX_HIDDEN 64

typedef enum {
    NNSORT_OK = 0,
    NNSORT_E_INVALID_ARG = -1, /* null pointer, size out of range, dtype/model mismatch */
    NNSORT_E_NAN_KEY = -2,     /* a floating-point key is NaN */
    NNSORT_E_OOM = -3,         /* device or pinned host allocation failed */
    NNSORT_E_BUDGET = -4,      /* request does not fit the server's HBM budget */
    NNSORT_E_CUDA = -5,        /* a CUDA runtime call failed; see nnsort_last_cuda_error() */
    NNSORT_E_TIMEOUT = -6,     /* a bounded device-side wait expired */
    NNSORT_E_UNSUPPORTED = -7, /* combination of options not built (e.g. BF16 on this arch) */
    NNSORT_E_STATE = -8        /* object used in the wrong state (e.g. unknown ticket) */
} nnsort_status;

typedef enum { NNSORT_F32 = 0, NNSORT_F64 = 1, NNSORT_U32 = 2, NNSORT_U64 = 3 } nnsort_dtype;

/* translate(A), Sec. "Input Phase": how a key becomes the model input x in [0, 1] over the
 * training sample's range. ORDBITS: min-max normalisation of the key's order-preserving integer
 * image (an exact integer difference, then one rounding to binary32). VALUE: min-max
 * normalisation of the key's value (binary32 arithmetic for f32 keys, binary64 for f64 keys).
 * For integer keys both are the same map. */
typedef enum { NNSORT_TRANSLATE_ORDBITS = 0, NNSORT_TRANSLATE_VALUE = 1 } nnsort_translate;

/* Arithmetic of the model's forward pass inside a sort. FP32: binary32 FMA chains, bit-identical
 * to the CPU reference. BF16: the hidden-to-hidden layer runs on the tensor cores (tcgen05, BF16
 * operands, FP32 accumulation); first and output layers stay binary32. BF16X2: as BF16, but each
 * first-layer activation a is passed as the pair hi = a truncated to BF16, lo = (a - hi) rounded to
 * FP16; hi multiplies the BF16 weights and lo an FP16 copy of them, into the same FP32 accumulator
 * (two MMA chains): the activations keep ~19 significant bits, so F stays about as finely resolved
 * in x as the binary32 model (the weights' rounding only changes f smoothly). Two-hidden-layer
 * models only; others use binary32. */
typedef enum {
    NNSORT_PREC_FP32 = 0,
    NNSORT_PREC_BF16 = 1,
    NNSORT_PREC_BF16X2 = 2,
    /* PWL: f compiled into its piecewise-linear form (a 1-D ReLU MLP is piecewise linear in x) in
     * binary64 on the host, then per key one binary search over the segments' order-image
     * thresholds and one multiply-add in pairs of binary32 (~48 significant bits; binary64 only to
     * normalise f64 keys): the positions of the binary64 model up to rounding, and no binary32
     * resolution limit in translate or the forward pass. Single-array sorts and nnsort_predict only (a batch
     * returns NNSORT_E_UNSUPPORTED). */
    NNSORT_PREC_PWL = 3
} nnsort_precision;

/* Training loss: mean squared error, or the Huber loss of Eq. (loss). */
typedef enum { NNSORT_LOSS_MSE = 0, NNSORT_LOSS_HUBER = 1 } nnsort_loss;

/* Model f (Sec. "Training details"): a ReLU MLP 1 -> h1 [-> h2] -> 1 plus the normaliser of
 * translate(A). Parameter layout, one hidden layer (layers = 1, h2 = 0):
 *     W1[h1] b1[h1] W3[h1] b3
 * two hidden layers (layers = 2):
 *     W1[h1] b1[h1] W2[h2*h1] (row k holds unit k's h1 input weights) b2[h2] W3[h2] b3
 * The forward pass is h1_j = relu(fma(W1_j, x, b1_j)); z_k = b2_k + sum_j W2_kj h1_j accumulated
 * in j order with one FMA per term; y = b3 + sum_k W3_k h_k accumulated in k order. */
typedef struct {
    int32_t dtype;     /* nnsort_dtype of the keys this model sorts */
    int32_t translate; /* nnsort_translate */
    int32_t layers;    /* hidden layers: 1 or 2 */
    int32_t h1, h2;    /* hidden widths, 1 .. NNSORT_MAX_HIDDEN; h2 = 0 when layers = 1 */
    uint64_t lo_bits;  /* order image of the smallest training key (ORDBITS) */
    double lo_val;     /* value of the smallest training key (VALUE) */
    double scale;      /* 1 / (hi - lo) in the translate's units; 1 when hi == lo */
} nnsort_model_desc;

typedef struct nnsort_model nnsort_model;

/* Training options (Sec. "Training"; Adam per Kingma & Ba). Defaults: 1 -> 32 -> 1, ORDBITS,
 * MSE, 10000 samples, 100 full-batch steps, lr 1e-2, betas (0.9, 0.999), eps 1e-8, seed 0. */
typedef struct {
    int32_t layers, h1, h2;
    int32_t translate;
    int32_t loss;
    float huber_delta;
    uint64_t sample_n; /* S: keys drawn with replacement to form the labelled training set */
    uint32_t steps;    /* Adam steps */
    uint32_t batch;    /* 0: full batch; otherwise samples per step drawn from the labelled set */
    float lr, beta1, beta2, adam_eps;
    uint64_t seed;     /* SplitMix64 stream for sampling, initialisation and mini-batches */
    int32_t monotone;  /* 1: sign-structured weights (layer-1 unit j keeps the sign s_j of its
                          initial input weight, output unit k the sign q_k of its initial output
                          weight; W2_kj carries s_j q_k, or W3_j carries s_j with one hidden
                          layer), projected after every Adam step, so f never decreases */
} nnsort_train_opts;

/* Sort options (Fig. "Algorithm NN-sort" inputs m, eps, tau). Defaults: m 1.25 (the paper's
 * setting), eps 3, tau 1024, FP32, automatic bucket width, no injected slots, no trace. */
typedef struct {
    float m;                  /* relaxation factor */
    int32_t eps;              /* iteration limit, 0 .. NNSORT_MAX_ROUNDS */
    uint64_t tau;             /* conflict-array threshold */
    int32_t precision;        /* nnsort_precision */
    int32_t bucket_log2;      /* 0: automatic; else log2 of the slots per on-chip bucket (9 .. 14) */
    const uint32_t *d_slots;  /* nullable: injected positions in [0, floor(n m)] replace the model */
    int8_t *d_fate;           /* nullable: per input row, +i stored in o_i and appended, -i stored
                                 in o_i and inserted out of order, 0 sorted as leftover */
    int32_t no_sync;          /* 1: skip the statistics read-back; errors raised on the device are
                                 then reported by nnsort_stream_status(). The call still waits once
                                 for the device after the polish, to send a large seam repair to
                                 the multi-block sort. */
    int32_t timing;           /* 1: record per-stage CUDA events into nnsort_stats.ms_stage */
    int32_t polish_blocks;    /* 0: automatic (3); 1, 2 or 3 polish blocks per SM: fewer blocks
                                 let a bucket hold more keys on chip, more blocks leave more L1
                                 and overlap more buckets */
} nnsort_sort_opts;

/* Per-array statistics (Sec. "Model Analysis", Eq. (sorting rate), Eq. (ratio)). */
typedef struct {
    uint32_t rounds;                           /* t: completed iterations */
    uint32_t eps;
    uint64_t n, L, tau;                        /* L = floor(n m) + 1 positions */
    uint64_t w_size[NNSORT_MAX_ROUNDS + 1];    /* count(w) entering iteration i+1; w_size[i] = |c_i| */
    uint64_t placed[NNSORT_MAX_ROUNDS];        /* elements stored in o_i */
    uint64_t out_of_order[NNSORT_MAX_ROUNDS];  /* elements of o_i the polish inserts */
    double sigma[NNSORT_MAX_ROUNDS];           /* conflict rate |c_i| / count(w) of iteration i */
    double e[NNSORT_MAX_ROUNDS];               /* out-of-order rate of o_i */
    double trad_rate;                          /* traditional sorting rate: |w_t| / n */
    uint64_t buckets;                          /* on-chip buckets the positions were cut into */
    uint64_t oversized_buckets;                /* buckets processed from global memory */
    uint64_t repaired;                         /* elements re-sorted across bucket seams */
    /* stage durations (CUDA events on the call's stream), filled when nnsort_sort_opts.timing = 1:
     * [0] predict, [1] partition (all passes), [2] bucket bounds, [3] rounds, [4] finalize,
     * [5] polish, [6] seam/repair, [7] whole call. Batched sorts report them in entry 0. */
    float ms_stage[8];
    uint32_t partition_passes;                 /* stable partition passes run */
    uint32_t bucket_log2;                      /* log2 of the positions per bucket */
    uint64_t repair_ranges;                    /* disjoint output ranges re-sorted across seams */
} nnsort_stats;

/* ---- library ---------------------------------------------------------------------------- */
int nnsort_version(void);
/* Static description of a status code. */
const char *nnsort_strerror(int status);
/* The cudaError_t of the last failing CUDA call (0 if none). */
int nnsort_last_cuda_error(void);
void nnsort_default_train_opts(nnsort_train_opts *o);
void nnsort_default_sort_opts(nnsort_sort_opts *o);
/* Frees the library's cached device workspace and pinned staging buffers. */
int nnsort_release(void);
/* Device-side error word raised by kernels on `stream` since the last call that read it
 * (NNSORT_OK, NNSORT_E_NAN_KEY, NNSORT_E_TIMEOUT or NNSORT_E_INVALID_ARG); synchronises. */
int nnsort_stream_status(cudaStream_t stream);
/* Self-test of the timeout path shared by every device-side wait in the library: one thread waits
 * on a device flag that nothing sets, polling %globaltimer with the library's wait loop, for
 * limit_us microseconds (clamped to [1, 1,000,000]) or a fixed number of polls, then raises the
 * timeout bit of a device error word and returns. Returns NNSORT_E_TIMEOUT when the wait expired
 * as it must (NNSORT_OK would mean the flag was seen set). Nothing faults, traps or hangs; the
 * context stays usable. Synchronous; uses two words of static device memory, so concurrent calls
 * must not overlap. */
int nnsort_selftest_wait(uint32_t limit_us, cudaStream_t stream);
/* Number of kernels the library has launched in this process (all devices and streams). */
uint64_t nnsort_launch_count(void);
/* Bytes of device workspace a sort of n keys of `dtype` (payload or not) uses. */
size_t nnsort_workspace_bytes(uint64_t n, int32_t dtype, int32_t with_payload,
                              const nnsort_sort_opts *o);

/* ---- model f ---------------------------------------------------------------------------- */
/* Creates a model from a description and h_params (binary32, layout above, host memory).
 * Synchronous. */
int nnsort_model_create(const nnsort_model_desc *desc, const float *h_params, nnsort_model **out);
int nnsort_model_free(nnsort_model *f);
/* Copies the description and (h_params nullable) the binary32 parameters to the host. */
int nnsort_model_describe(const nnsort_model *f, nnsort_model_desc *desc, float *h_params);
/* Serialised model: versioned blob of description + parameters. */
size_t nnsort_model_blob_size(const nnsort_model *f);
int nnsort_model_save(const nnsort_model *f, void *h_blob, size_t cap);
int nnsort_model_load(const void *h_blob, size_t size, nnsort_model **out);

/* The piecewise-linear form of the model f with parameters h_params (binary32, the layout of
 * nnsort_model_create, host memory): a ReLU MLP of one input is piecewise linear (the map line of
 * Fig. "Algorithm NN-sort"). Computed on the host in binary64: segment i covers translated inputs
 * x in [h_breaks[i], h_breaks[i+1]) (h_breaks[0] = -infinity, the last segment is unbounded) and
 * there F(x) = h_slope[i] * x + h_icept[i]. Host arrays of `cap` entries, written in increasing x;
 * *count receives the number of segments (at most h1 + 1 for one hidden layer, 1 + h1 + (h1 + 1) h2
 * for two). Returns NNSORT_E_INVALID_ARG, with *count set, when cap is too small. No device work;
 * usable without a GPU. NNSORT_PREC_PWL sorts use this form. */
int nnsort_mlp_pwl(int32_t layers, int32_t h1, int32_t h2, const float *h_params, double *h_breaks,
                   double *h_slope, double *h_icept, uint32_t cap, uint32_t *count);

/* ---- training (Sec. "Training", Eq. (loss)) ------------------------------------------- */
/* Training data: S keys drawn with replacement (draw j picks row floor(u_j n / 2^64) with u_j
 * the j-th output of the SplitMix64 stream of `seed`), sorted by (key, draw); the normaliser
 * is the sample's [min, max]; d_x[j] is translate(key_j) in binary32 and d_label[j] = j / S
 * (the empirical CDF). d_rows (nullable) receives the sorted draws' rows. desc_out receives the
 * normaliser (dtype, translate, lo_bits, lo_val, scale; layer fields zero). Synchronous. */
int nnsort_sample_labels(const void *d_keys, uint64_t n, int32_t dtype, uint64_t S, uint64_t seed,
                         int32_t translate, nnsort_model_desc *desc_out, float *d_x, float *d_label,
                         uint32_t *d_rows, cudaStream_t stream);
/* Trains f on the device: sample + labels as above, parameters initialised from the seed, then
 * `steps` Adam steps on the mean loss, with the gradient from the library's backward kernels.
 * h_loss (nullable, `steps` floats) receives the loss before each step. Synchronous. */
int nnsort_train(const void *d_keys, uint64_t n, int32_t dtype, const nnsort_train_opts *o,
                 nnsort_model **out, float *h_loss, cudaStream_t stream);
/* Trains `count` models at once, model j on the device array d_keys[j] (host array of device
 * pointers) of ns[j] keys, with the recipe of nnsort_train and seed o->seed + j; model j's sample
 * size is sample_ns[j] (nullable: o->sample_n for every model). One thread block per model draws
 * the sample, sorts it, labels it and runs all `steps` Adam steps on chip, so the whole batch is
 * one launch per sample-size class. Needs one hidden layer of at most 32 units (o->layers == 1,
 * o->h1 <= 32), no monotone constraint, and 1 <= sample size <= NNSORT_TRAIN_BLOCK_MAX_S; else
 * NNSORT_E_UNSUPPORTED. out[j] receives model j (free each with nnsort_model_free); h_loss
 * (nullable, count x steps floats, model-major) the losses. Errors as nnsort_train (NaN in a
 * sample: NNSORT_E_NAN_KEY, no model is returned). Synchronous. The paper trains one model; this
 * is the batched form the per-array models of a batch of sorts need. */
#define NNSORT_TRAIN_BLOCK_MAX_S 16384
int nnsort_train_batch(void *const *d_keys, const uint64_t *ns, int32_t count, int32_t dtype,
                       const nnsort_train_opts *o, const uint64_t *sample_ns, nnsort_model **out,
                       float *h_loss, cudaStream_t stream);
/* Forward pass of a ReLU MLP with parameters d_params (layout above) on d_x[n] -> d_y[n]. */
int nnsort_mlp_forward(const float *d_params, int32_t layers, int32_t h1, int32_t h2,
                       const float *d_x, uint64_t n, float *d_y, cudaStream_t stream);
/* Backward pass: given upstream gradients d_gy[n] of a scalar s with respect to y, writes
 * d_gparams (ds/dparams, same layout, overwritten) and d_gx (nullable, ds/dx). The reduction over
 * samples is a fixed-order tree, so results are reproducible run to run. */
int nnsort_mlp_backward(const float *d_params, int32_t layers, int32_t h1, int32_t h2,
                        const float *d_x, const float *d_gy, uint64_t n, float *d_gparams,
                        float *d_gx, cudaStream_t stream);
/* Mean loss over (d_x, d_label)[n] and its parameter gradient (overwritten); d_loss: one float. */
int nnsort_mlp_loss_grad(const float *d_params, int32_t layers, int32_t h1, int32_t h2,
                         const float *d_x, const float *d_label, uint64_t n, int32_t loss,
                         float huber_delta, float *d_loss, float *d_gparams, cudaStream_t stream);

/* ---- the sort ----------------------------------------------------------------------------- */
/* Lines 1 and 5-7 of Fig. "Algorithm NN-sort" alone: translate, model forward and the position
 * round(f(x) * n * m) clamped to [0, floor(n m)], for each of d_keys[n]. d_slots and d_y
 * (F(x) before rounding) are nullable outputs. `precision` selects the nnsort_precision arithmetic. */
int nnsort_predict(const void *d_keys, uint64_t n, int32_t dtype, const nnsort_model *f, float m,
                   int32_t precision, uint32_t *d_slots, float *d_y, cudaStream_t stream);
/* The whole method on device arrays, in place: d_keys[n] (and d_payload[n] when not null) are
 * replaced by the stably sorted sequence. f may be NULL only when o->d_slots injects positions.
 * st (nullable) receives statistics; unless o->no_sync, the call synchronises `stream` before
 * returning. */
int nnsort_sort(void *d_keys, int32_t *d_payload, uint64_t n, int32_t dtype, const nnsort_model *f,
                const nnsort_sort_opts *o, nnsort_stats *st, cudaStream_t stream);
/* End-to-end variant on host arrays: copies h_keys (and h_payload) to the device, sorts, copies
 * the result back. Synchronous. */
int nnsort_sort_host(void *h_keys, int32_t *h_payload, uint64_t n, int32_t dtype,
                     const nnsort_model *f, const nnsort_sort_opts *o, nnsort_stats *st,
                     cudaStream_t stream);
/* The whole job from host arrays: copies h_keys (and h_payload) to the device, trains a model on
 * the device with `to` (nnsort_train), sorts with it using `so`, copies the sorted arrays back.
 * h_loss (nullable) as in nnsort_train. Synchronous; the model is freed before returning. */
int nnsort_train_sort_host(void *h_keys, int32_t *h_payload, uint64_t n, int32_t dtype,
                           const nnsort_train_opts *to, const nnsort_sort_opts *so,
                           nnsort_stats *st, float *h_loss, cudaStream_t stream);
/* `count` independent arrays (host arrays of device pointers, sizes and models; all models of
 * one architecture and dtype) sorted in one pass of the pipeline: every kernel of the method
 * runs once over all arrays' buckets. st (nullable) receives `count` entries. */
int nnsort_sort_batch(void *const *d_keys, int32_t *const *d_payloads, const uint64_t *ns,
                      int32_t count, int32_t dtype, const nnsort_model *const *fs,
                      const nnsort_sort_opts *o, nnsort_stats *st, cudaStream_t stream);
/* The "no model" reference of the ablation in Sec. "Experimental Study" (what the learned part
 * gains is measured against sorting without it): a stable LSD radix sort of d_keys[n] (and
 * d_payload[n], nullable) by the keys' order images (8-bit digits; -0.0 before +0.0), every pass
 * the same partition kernel the NN-sort pipeline uses for its buckets. In place, caller-owned
 * device arrays; scratch from the stream's workspace. Synchronous. Errors: NNSORT_E_INVALID_ARG
 * (bad dtype, null keys with n > 0, n >= 2^32 - 1), NNSORT_E_OOM, NNSORT_E_CUDA,
 * NNSORT_E_TIMEOUT (reserved: the partition passes hold no device-side waits). */
int nnsort_radix_sort(void *d_keys, int32_t *d_payload, uint64_t n, int32_t dtype,
                      cudaStream_t stream);

/* ---- serving: continuous batching of sort requests ------------------------------------ */
/* A server owns `workers` CUDA streams on the current device and a host scheduler thread.
 * Requests (host arrays) are admitted in arrival order while the device memory they need fits
 * the HBM budget; admitted requests wait in a queue that every idle worker drains into its next
 * batch (up to max_batch requests or max_batch_keys keys), so requests that arrive while other
 * batches run join the following batch and work on different streams overlaps on the device.
 * Per batch a worker copies the requests in, trains each request's model on the device
 * (nnsort_train with `train` options and a per-request seed), sorts all of them with one
 * nnsort_sort_batch call (`sort` options), and copies the results back into the caller's host
 * arrays. Latency is measured from submit to the result being in host memory. The paper has no
 * serving layer; this is the batched, served form of its method. */
typedef struct {
    size_t hbm_budget;          /* bytes of device memory admitted requests may hold */
    int32_t workers;            /* streams / batches in flight (1 .. 8) */
    int32_t max_batch;          /* requests per batch (>= 1); 1 makes the server FIFO */
    uint64_t max_batch_keys;    /* keys per batch (0: unlimited) */
    nnsort_train_opts train;    /* per-request training (seed is replaced by request seed) */
    nnsort_sort_opts sort;      /* sort options (no injected positions, no trace) */
} nnsort_server_opts;

typedef struct nnsort_server nnsort_server;

#define NNSORT_PENDING 1  /* status of nnsort_server_poll for a request not finished yet */

/* Defaults: 120 GiB budget, 2 workers, max_batch 32, no key limit, default train/sort options. */
void nnsort_default_server_opts(nnsort_server_opts *o);
int nnsort_server_create(const nnsort_server_opts *o, nnsort_server **out);
/* Queues one request. h_keys[n] (and h_payload[n], nullable) are host arrays the caller keeps
 * alive and untouched until the request completes; they receive the sorted result in place.
 * `seed` seeds the request's training. Returns NNSORT_E_BUDGET if the request alone exceeds the
 * budget. *ticket identifies the request. Thread-safe. */
int nnsort_server_submit(nnsort_server *srv, void *h_keys, int32_t *h_payload, uint64_t n,
                         int32_t dtype, uint64_t seed, uint64_t *ticket);
/* NNSORT_OK once the request finished (st, latency_s filled when not null; the ticket is then
 * retired), NNSORT_PENDING before, NNSORT_E_STATE for an unknown ticket, or the request's error. */
int nnsort_server_poll(nnsort_server *srv, uint64_t ticket, nnsort_stats *st, double *latency_s);
/* As poll, but waits until the request finished. */
int nnsort_server_wait(nnsort_server *srv, uint64_t ticket, nnsort_stats *st, double *latency_s);
/* Finishes queued work, stops the workers and frees everything. */
int nnsort_server_destroy(nnsort_server *srv);

/* ---- sorting without device allocation ------------------------------------------------- */
/* The paper has no counterpart to this entry point; it serves callers that cannot allocate
 * device memory when they sort: code whose memory budget was fixed up front, code that must not
 * pay for (or synchronise on) cudaMalloc/cudaFree, and hosts whose allocator belongs to another
 * framework. It runs the same method and kernels as nnsort_sort on one device array, but takes all
 * of its scratch from one fixed device array that is part of the library image (about 13 MiB,
 * held on every GPU that loads the library until the process exits). It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   - n may be at most NNSORT_NOALLOC_MAX_N, and floor(n m) + 1 at most 1024 buckets of
 *     2^bucket_log2 positions; larger requests return NNSORT_E_INVALID_ARG and touch nothing.
 *   - f is required (o->d_slots and o->d_fate must be NULL).
 *   - The first call on a device looks up the scratch's device address (cudaGetSymbolAddress);
 *     make that first call before any stream capture.
 *   - Every call shares the one scratch array and finds the previous call's contents there; each
 *     call clears what must start at zero. Calls whose work overlaps on the GPU (for example on
 *     two streams at once) race on the scratch and must be serialised by the caller.
 *   - The call synchronises `stream` before returning and fills st (nullable) like nnsort_sort. */
#define NNSORT_NOALLOC_MAX_N 262144
int nnsort_sort_noalloc(void *d_keys, int32_t *d_payload, uint64_t n, int32_t dtype,
                        const nnsort_model *f, const nnsort_sort_opts *o, nnsort_stats *st,
                        cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* NNSORT_H */
