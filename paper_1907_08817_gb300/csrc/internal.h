// internal.h -- host-side declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <memory>
#include <vector>
#include <cuda_runtime.h>

#include "nnsort.h"

namespace nns {

// counts kernels launched by the library (nnsort_launch_count)
void note_launch(int kernels);

struct Seg;
struct SegStats;
struct OKey;

constexpr int RADIX_MAX_BITS = 9;
constexpr int RADIX_BINS = 1 << RADIX_MAX_BITS;  // 512
constexpr int PRED_THREADS = 256;
constexpr int PRED_ITEMS = 8;
constexpr int PRED_TILE = PRED_THREADS * PRED_ITEMS;  // 2048
constexpr int MAX_PASSES = 4;

struct PassPlan {
    int npass;
    int wlog;                 // log2 of the bucket width in positions
    int shift[MAX_PASSES];    // digit shift applied to the global position
    int bits[MAX_PASSES];
};

// padded architecture actually instantiated on the device
struct PadArch {
    int layers, h1, h2;  // padded widths (8, 16, 32 or 64; h2 = 0 for one hidden layer)
};
PadArch pad_arch(int layers, int h1, int h2);
size_t padded_param_count(const PadArch &a);

// ---- predict (k_predict.cu)
// Fills gs (global position per element) and optional key / payload / row copies into the element
// space. Also serves nnsort_predict through slots_out / y_out (element space of a single array).
// one segment of the compiled piecewise-linear model in the keys' order-image domain (pwl.cu)
struct PwlEntry {
    unsigned long long thr;  // smallest order image in the segment (0 for the first)
    float Ah, Al, Ch, Cl;    // position = floor(A d + C), d = translate offset of the key, with
                             // A = Ah + Al and C = Ch + Cl (pairs of binary32: ~48 significant bits)
};
struct PwlDev {
    const PwlEntry *tab;     // device table, null when the compiled form is not used
    uint32_t S;              // segments
};

struct PredictArgs {
    const Seg *segs;
    int nseg;
    uint32_t total_tiles;
    uint32_t *gs;            // nullable
    void *key_copy;          // nullable
    uint32_t *pay_copy;      // nullable
    uint32_t *row_init;      // nullable
    uint32_t *slots_out;     // nullable
    float *y_out;            // nullable
    uint32_t *err;
    int key_bytes;
    int dtype;
    PwlDev pwl;              // NNSORT_PREC_PWL (single array)
    int single_model;        // 1: one array whose positions come from its model (no injected slots)
    const float *host_pad;   // single_model: that model's padded parameters in host memory
};
cudaError_t launch_predict(const PadArch &a, int precision, const PredictArgs &p, int sms,
                           cudaStream_t s);
cudaError_t launch_predict_pwl(const PredictArgs &p, int sms, cudaStream_t s);
// host side of the compiled form (pwl.cu)
void pwl_segments(int layers, int h1, int h2, const float *params, std::vector<double> &brk,
                  std::vector<double> &slope, std::vector<double> &icept);
uint32_t pwl_max_segments(int layers, int h1, int h2);
void pwl_key_table(const nnsort_model_desc &d, const std::vector<double> &brk, const std::vector<double> &slope,
                   const std::vector<double> &icept, double nm, PwlEntry *out);

// ---- partition (k_partition.cu)
// One pass of the stable digit partition without inter-block waits (reduce, then scan, then
// scatter): per tile of SC_TILE elements a digit histogram, per chunk of SC_CHUNK tiles the
// in-chunk exclusive prefixes and chunk totals (and the digit totals), the chunk bases over all
// chunks and digits, then the scatter of every tile to its chunk's base + its in-chunk prefix.
// The pass finds its own digit offsets, so no histogram is needed beforehand; tile_hist, chunk and
// bin_total are scratch.
constexpr int SC_THREADS = 512;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;  // 4096
constexpr int SC_CHUNK = 16;                    // tiles per chunk (in-chunk prefix < 2^16)
struct PartitionArgs {
    uint64_t N;
    const uint32_t *gs_in;  uint32_t *gs_out;   // null when sorting by key bits
    const void *key_in;     void *key_out;
    const uint32_t *pay_in; uint32_t *pay_out;  // nullable
    const uint32_t *row_in; uint32_t *row_out;  // nullable
    int key_digits;         // 1: digit from the key's order image, 0: from gs
    int shift, bits;
    uint16_t *tile_hist;    // [tiles * RADIX_BINS] scratch
    uint32_t *chunk;        // [chunks * RADIX_BINS] scratch
    uint32_t *bin_total;    // [RADIX_BINS] scratch: elements per digit
    int key_bytes, dtype;
};
inline uint64_t partition_tiles(uint64_t N) { return (N + SC_TILE - 1) / SC_TILE; }
inline uint64_t partition_chunks(uint64_t N) { return (partition_tiles(N) + SC_CHUNK - 1) / SC_CHUNK; }
cudaError_t launch_partition(const PartitionArgs &a, cudaStream_t s);
// bucket starts by binary search over the partitioned global positions
cudaError_t launch_bucket_bounds(const uint32_t *gs, uint64_t N, uint32_t nb, int wlog,
                                 uint32_t *bstart, cudaStream_t s);

// ---- rounds / finalize / polish / seam / repair (k_solve.cu)
// an output range [lo, hi) of array `seg` (positions relative to the array) to be re-sorted
struct SeamRange {
    unsigned long long lo, hi;
    uint32_t seg, pad;
};

// a bucket too large for one block's polish: partitioned elements [lo, hi) of array `seg`, bucket b,
// offset `off` in the packed buffer
struct BigRange {
    unsigned long long lo, hi;
    uint32_t seg, off, b, pad;
};
constexpr uint32_t POLISH_BIG = 1u << 16;  // buckets above this many elements sort multi-block

struct SolveArgs {
    const Seg *segs;
    int nseg;
    uint32_t NB;
    int wlog;
    const uint32_t *bstart;   // [NB + 1]
    const uint32_t *gs;       // partitioned
    const void *keys;         // partitioned
    const uint32_t *pay;      // partitioned, nullable
    const uint32_t *rows;     // partitioned, nullable
    uint8_t *rank;            // [N]
    SegStats *stats;          // [nseg]
    OKey *bmax;               // [NB * MAXR]
    OKey *carry;              // [NB * MAXR]
    OKey *blo, *bhi;          // [NB]
    // global scratch for buckets beyond on-chip capacity
    uint8_t *g_flag;          // [N]
    uint32_t *g_x, *g_y;  // [N] each
    uint64_t N;               // elements (the sizes of the [N] scratch arrays)
    int8_t *fate;             // nullable, per row (single array only)
    uint32_t *out_rows;       // [N] rows of the output order (when rows are carried)
    void *key_scratch;        // [N] free partition buffer reused by the seam repair
    uint32_t *pay_scratch, *row_scratch;
    uint32_t *err;
    int key_bytes, dtype;
    int polish_cap;           // elements a bucket may hold on chip
    size_t polish_smem;
    int allow_defer;          // 1: seam repairs above SEAM_CTA_MAX are left to the host's
                              //    multi-block sort (never when rows are carried)
    SeamRange *ranges;        // [max_ranges]: block-sized repairs from the front, large from the back
    uint32_t max_ranges;      // >= NB + nseg
    uint32_t *seam_cnt;       // [4]: block-sized ranges, large ranges, next range to repair
    OKey *seam_suf;           // [NB] scratch: smallest element of the later buckets
    OKey *seam_pre;           // [NB] scratch: largest element of the earlier buckets
    unsigned long long *seam_cut;  // [2 NB] scratch: first and last sorted-boundary cut per bucket
    const uint32_t *order;    // [NB] nullable: block i of k_rounds / k_polish takes bucket order[i]
    BigRange *giant;          // nullable: k_bucket_order lists buckets above POLISH_BIG here and
    uint32_t *giant_cnt;      //   k_rounds leaves them to launch_giant_rounds
    BigRange *big;            // nullable: k_polish lists buckets above POLISH_BIG here (and only
    uint32_t *big_cnt;        //   splits their runs); their sort is left to the host's multi-block sort
};
constexpr uint64_t SEAM_CTA_MAX = 1u << 16;  // largest seam repair one block performs
// order[]: buckets holding more than `heavy` elements first (they run longest), the rest after
cudaError_t launch_bucket_order(const SolveArgs &a, uint32_t heavy, uint32_t *order,
                                uint32_t *cnt /*[2], zeroed here*/, cudaStream_t s);
// buckets above POLISH_BIG elements run their rounds on the whole GPU (global claim tables); the
// list, its count and the per-(bucket, round) statistics live in GiantRounds
struct GiantRounds {
    BigRange *list;               // [N / POLISH_BIG + 1]
    uint32_t *count;              // [1]
    unsigned long long *table;    // [list entries x W] round-tagged claims
    unsigned int *cnt;            // [entries x MAXR] elements stored per round
    unsigned long long *kmax;     // [entries x MAXR] largest order image stored per round
    unsigned int *tbmax;          // [entries x MAXR] its largest tie-break
    uint32_t cap;                 // list entries
};
cudaError_t launch_giant_rounds(const SolveArgs &a, const GiantRounds &g, int eps, int sms, cudaStream_t s);
cudaError_t launch_rounds(const SolveArgs &a, cudaStream_t s);
cudaError_t launch_finalize(const SolveArgs &a, cudaStream_t s);
cudaError_t launch_polish(const SolveArgs &a, cudaStream_t s);
cudaError_t launch_seam_repair(const SolveArgs &a, int sms, cudaStream_t s);
cudaError_t launch_big_pack(const BigRange *br, uint32_t nr, const Seg *segs, uint64_t total, int key_bytes,
                            const void *src_k, const uint32_t *src_p, void *pk, uint32_t *pp, uint32_t *pj,
                            int unpack, int sms, cudaStream_t s);
cudaError_t launch_big_bounds(const BigRange *br, uint32_t nr, const Seg *segs, int key_bytes, int dtype,
                              OKey *blo, OKey *bhi, cudaStream_t s);
cudaError_t launch_seam_pack(const SeamRange *rg, uint32_t nr, const Seg *segs, uint64_t total,
                             int key_bytes, void *pk, uint32_t *pp, uint32_t *ps, int unpack, int sms,
                             cudaStream_t s);
int polish_capacity(int key_bytes, bool payload, bool rows, int wlog, int blocks_per_sm,
                    size_t *smem_bytes);

// ---- training (k_train.cu)
cudaError_t launch_sample(const void *keys, uint64_t n, int key_bytes, int dtype, uint64_t S,
                          uint64_t stream_seed, void *sample_keys, uint32_t *sample_rows,
                          uint32_t *err, cudaStream_t s);
cudaError_t launch_minmax_norm(const void *sorted_keys, uint64_t S, int key_bytes, int dtype,
                               int translate, double *norm_out /*lo_val, scale*/,
                               unsigned long long *lobits_out, cudaStream_t s);
cudaError_t launch_make_xy(const void *sorted_keys, uint64_t S, int key_bytes, const Norm *nm_dev,
                           float *x, float *label, cudaStream_t s);
struct TrainStepArgs {
    float *params;        // padded layout, updated in place
    float *m, *v;         // Adam moments (padded layout)
    float *grad;          // padded layout
    float *partials;      // [blocks * P]
    float *loss_partials; // [blocks]
    float *loss_out;      // [steps]
    const float *x, *label;
    uint64_t S;
    uint32_t batch;       // 0 = full
    uint64_t batch_seed;
    int step;             // 0-based
    int loss; float delta;
    float lr, b1, b2, eps;
    size_t P;
    const float *mask;    // 1 for real parameters, 0 for padding
};
cudaError_t launch_train_step(const PadArch &a, const TrainStepArgs &t, cudaStream_t s);
// many small models at once, one block per model (k_train_block.cu): one hidden layer of padded
// width 8, 16 or 32, samples of at most TB_MAX_S keys; the sort buffer holds `cap` keys (a power of
// two >= every S of the launch)
constexpr uint32_t TB_MAX_S = 16384;
struct TrainBlockArgs {
    const void *const *keys;   // [models] device key arrays
    const uint64_t *n, *S;     // [models] keys, sample size
    const uint32_t *ids;       // [blocks] model index of each block
    uint32_t cap;
    int dtype, translate, h1;  // h1: real hidden width (<= padded width)
    uint64_t seed0;            // model m uses seed seed0 + m
    int steps;
    uint64_t batch;            // 0: full batch
    int loss;
    float delta, lr, b1, b2, eps;
    const float *c1, *c2;      // [steps] Adam bias corrections 1 - beta^(t+1)
    float *params_out;         // [models][3 H + 1] padded layout
    Norm *norm_out;            // [models]
    float *loss_out;           // nullable [models][steps]
    uint32_t *err;
};
cudaError_t launch_train_block(const TrainBlockArgs &a, int key_bytes, int padded_h, uint32_t blocks,
                               cudaStream_t s);
// gradient of a sum over samples (k_train.cu, k_train_tc.cu). mode 0: s = sum_i gy_i * y_i (explicit
// upstream gradient); mode 1: mean loss over the batch with labels; mode 2: as mode 1 with batch
// indices drawn from the batch stream. Each block (or block group) writes one partial gradient row.
struct GradArgs {
    const float *params;
    const float *x, *gy, *label;
    uint64_t n;          // samples in the batch
    uint64_t S;          // labelled set size (mode 2)
    uint64_t bseed;      // batch stream (mode 2)
    uint64_t bofs;       // first draw of this step (mode 2)
    int mode, loss;
    float delta;
    float inv_n;
    float *partials;     // [rows * P]
    float *loss_partials;  // [rows], nullable
    float *gx;           // nullable (mode 0)
};
int train_grad_blocks(const PadArch &a, uint64_t nsamples);
// two hidden layers of width 64 on the tensor cores (k_train_tc.cu): blocks of the launch (each
// writes one partial row), and the launch; a bounded wait that expired sets ERR_TIMEOUT in the
// library's training error word (train_err_word)
int grad_tc64_blocks(uint64_t nsamples);
cudaError_t launch_grad_tc64(const GradArgs &g, cudaStream_t s);
// every Adam step of a training run of that model in one cooperative launch: c12 = device
// [2 * steps] bias corrections (1 - beta1^(t+1), then 1 - beta2^(t+1)), count = a device word zeroed
// before the launch
cudaError_t launch_train_tc64(const TrainStepArgs &t, uint32_t steps, const float *c12, unsigned int *count,
                              cudaStream_t s);
uint32_t *train_err_word();
// forward / backward / loss-grad for explicit arrays (nnsort_mlp_* entry points)
cudaError_t launch_mlp_forward(const PadArch &a, const float *params, const float *x, uint64_t n,
                               float *y, cudaStream_t s);
cudaError_t launch_mlp_backward(const PadArch &a, const float *params, const float *x,
                                const float *gy, const float *label, uint64_t n, int mode,
                                int loss, float delta, float *partials, float *loss_partials,
                                float *gx, cudaStream_t s, int *blocks_out);
cudaError_t launch_reduce_partials(const float *partials, int blocks, size_t P, float *out,
                                   const float *loss_partials, float *loss_out, float scale,
                                   cudaStream_t s);

}  // namespace nns

// The model handle behind the opaque nnsort_model of the C ABI: one definition for every
// translation unit that reads it.
struct nnsort_model {
    nnsort_model_desc desc;
    std::vector<float> params;  // caller layout
    std::vector<float> hpad;    // padded layout in host memory (the tensor-core predict passes its
                                // vectors as launch constants)
    nns::PadArch pad;
    size_t P = 0, Ppad = 0;
    float *d_params = nullptr;  // padded layout
    int device = 0;
    std::shared_ptr<void> owner;  // set when d_params lies in a device block shared by several
                                  // models (freed with the last of them), else d_params is its own
};
