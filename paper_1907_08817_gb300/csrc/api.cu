// api.cu -- the C ABI of libnnsort.so: argument checking, models, per-stream device workspaces,
// and the launch sequence of the method's kernels. No arithmetic of the method runs on the host
// except the scalar set-up the paper's definitions need (n*m, L, normaliser, initial weights).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace nns;

namespace nns {
void note_launch(int kernels);
}

namespace {

thread_local int g_last_cuda = 0;
std::mutex g_mu;
std::atomic<unsigned long long> g_launches{0};

#define CK(x)                                                                    \
    do {                                                                         \
        cudaError_t e_ = (x);                                                    \
        if (e_ != cudaSuccess) {                                                 \
            g_last_cuda = (int)e_;                                               \
            return NNSORT_E_CUDA;                                                \
        }                                                                        \
    } while (0)

int key_bytes_of(int dt) { return (dt == NNSORT_F32 || dt == NNSORT_U32) ? 4 : 8; }
bool dtype_ok(int dt) { return dt >= NNSORT_F32 && dt <= NNSORT_U64; }
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

uint64_t mix64h(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
uint64_t rng_h(uint64_t seed, uint64_t i) { return mix64h(seed + (i + 1) * 0x9E3779B97F4A7C15ull); }
double unit53h(uint64_t u) { return (double)(u >> 11) * (1.0 / 9007199254740992.0); }
constexpr uint64_t TAG_SAMPLE = 1, TAG_INIT = 2, TAG_BATCH = 3;

// ---- per-(device, stream) workspace
struct Workspace {
    int device = -1;
    unsigned char *arena = nullptr;
    size_t cap = 0;
    unsigned char *part = nullptr;  // partition scratch: tile histograms, then chunk bases
    size_t part_cap = 0;
    unsigned char *pinned = nullptr;
    size_t pcap = 0;
    uint32_t *last_err = nullptr;  // device error word of the last sort on this stream
    void *host_dev = nullptr;      // device staging for the host-array entry point
    size_t host_cap = 0;
    cudaEvent_t ev[8] = {};        // stage timing
};
std::map<std::pair<int, cudaStream_t>, Workspace *> g_ws;

int get_ws(cudaStream_t s, Workspace **out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    auto key = std::make_pair(dev, s);
    auto it = g_ws.find(key);
    if (it == g_ws.end()) {
        Workspace *w = new (std::nothrow) Workspace();
        if (!w) return NNSORT_E_OOM;
        w->device = dev;
        it = g_ws.emplace(key, w).first;
    }
    *out = it->second;
    return NNSORT_OK;
}

int ensure_arena(Workspace *w, size_t bytes, cudaStream_t s) {
    if (bytes <= w->cap) return NNSORT_OK;
    CK(cudaStreamSynchronize(s));
    if (w->arena) CK(cudaFree(w->arena));
    w->arena = nullptr;
    w->cap = 0;
    const size_t want = align_up(bytes + bytes / 8, 1 << 20);
    cudaError_t e = cudaMalloc(&w->arena, want);
    if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        cudaGetLastError();
        return NNSORT_E_OOM;
    }
    w->cap = want;
    return NNSORT_OK;
}

int ensure_pinned(Workspace *w, size_t bytes, cudaStream_t s) {
    if (bytes <= w->pcap) return NNSORT_OK;
    CK(cudaStreamSynchronize(s));
    if (w->pinned) CK(cudaFreeHost(w->pinned));
    w->pinned = nullptr;
    w->pcap = 0;
    const size_t want = align_up(bytes, 1 << 16);
    cudaError_t e = cudaMallocHost((void **)&w->pinned, want);
    if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        cudaGetLastError();
        return NNSORT_E_OOM;
    }
    w->pcap = want;
    return NNSORT_OK;
}

size_t part_hist_bytes(uint64_t N) { return align_up(partition_tiles(N) * RADIX_BINS * sizeof(uint16_t), 256); }
size_t part_chunk_bytes(uint64_t N) { return align_up(partition_chunks(N) * RADIX_BINS * sizeof(uint32_t), 256); }
size_t part_bytes(uint64_t N) { return part_hist_bytes(N) + part_chunk_bytes(N) + RADIX_BINS * sizeof(uint32_t); }

// scratch of the partition passes over up to N elements
int ensure_part(Workspace *w, uint64_t N, cudaStream_t s) {
    const size_t bytes = part_bytes(N);
    if (bytes <= w->part_cap) return NNSORT_OK;
    CK(cudaStreamSynchronize(s));
    if (w->part) CK(cudaFree(w->part));
    w->part = nullptr;
    w->part_cap = 0;
    const size_t want = align_up(bytes + bytes / 4, 1 << 16);
    cudaError_t e = cudaMalloc(&w->part, want);
    if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        cudaGetLastError();
        return NNSORT_E_OOM;
    }
    w->part_cap = want;
    return NNSORT_OK;
}

// one partition pass over N elements with the workspace's scratch
cudaError_t part_pass(Workspace *w, PartitionArgs a, cudaStream_t s) {
    a.tile_hist = reinterpret_cast<uint16_t *>(w->part);
    a.chunk = reinterpret_cast<uint32_t *>(w->part + part_hist_bytes(a.N));
    a.bin_total = reinterpret_cast<uint32_t *>(w->part + part_hist_bytes(a.N) + part_chunk_bytes(a.N));
    return launch_partition(a, s);
}

// bump allocator over the arena
struct Carve {
    size_t off = 0;
    unsigned char *base = nullptr;
    template <typename T> T *take(size_t count) {
        off = align_up(off, 256);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

}  // namespace

void nns::note_launch(int kernels) { g_launches.fetch_add((unsigned long long)kernels); }

// ---------------------------------------------------------------------------------------------
// models
namespace nns {
PadArch pad_arch(int layers, int h1, int h2) {
    auto up = [](int h) { return h <= 8 ? 8 : h <= 16 ? 16 : h <= 32 ? 32 : 64; };
    PadArch a;
    a.layers = layers;
    if (layers == 1) { a.h1 = up(h1); a.h2 = 0; }
    else { const int m = std::max(up(h1), up(h2)); a.h1 = m; a.h2 = m; }
    return a;
}
size_t padded_param_count(const PadArch &a) {
    return a.layers == 1 ? (size_t)3 * a.h1 + 1 : (size_t)2 * a.h1 + (size_t)a.h2 * a.h1 + 2 * a.h2 + 1;
}
}  // namespace nns

namespace {
size_t param_count(int layers, int h1, int h2) {
    return layers == 1 ? (size_t)3 * h1 + 1 : (size_t)2 * h1 + (size_t)h2 * h1 + 2 * (size_t)h2 + 1;
}
// padded position of caller-layout parameter u
size_t pad_index(int layers, int h1, int h2, const PadArch &p, size_t u) {
    const size_t H1 = p.h1, H2 = p.h2;
    if (layers == 1) {
        if (u < (size_t)h1) return u;
        if (u < 2 * (size_t)h1) return H1 + (u - h1);
        if (u < 3 * (size_t)h1) return 2 * H1 + (u - 2 * h1);
        return 3 * H1;
    }
    const size_t a = h1, b = 2 * (size_t)h1, c = b + (size_t)h2 * h1, d = c + h2, e = d + h2;
    if (u < a) return u;
    if (u < b) return H1 + (u - a);
    if (u < c) { const size_t v = u - b, k = v / h1, j = v % h1; return 2 * H1 + k * H1 + j; }
    if (u < d) return 2 * H1 + H2 * H1 + (u - c);
    if (u < e) return 2 * H1 + H2 * H1 + H2 + (u - d);
    return 2 * H1 + H2 * H1 + 2 * H2;
}
bool arch_ok(int layers, int h1, int h2) {
    if (layers == 1) return h1 >= 1 && h1 <= NNSORT_MAX_HIDDEN && h2 == 0;
    if (layers == 2) return h1 >= 1 && h1 <= NNSORT_MAX_HIDDEN && h2 >= 1 && h2 <= NNSORT_MAX_HIDDEN;
    return false;
}
std::vector<float> to_padded(const nnsort_model_desc &d, const PadArch &p, const float *src) {
    std::vector<float> out(padded_param_count(p), 0.0f);
    const size_t P = param_count(d.layers, d.h1, d.h2);
    for (size_t u = 0; u < P; ++u) out[pad_index(d.layers, d.h1, d.h2, p, u)] = src[u];
    return out;
}
Norm norm_of(const nnsort_model_desc &d) {
    Norm n;
    n.dtype = d.dtype;
    n.translate = d.translate;
    n.lo_bits = d.lo_bits;
    n.lo_val = d.lo_val;
    n.scale = d.scale;
    n.lo_f = (float)d.lo_val;
    n.scale_f = (float)d.scale;
    return n;
}
}  // namespace

__global__ void k_unpad(const float *src, float *dst, int layers, int h1, int h2, int H1, int H2, size_t P) {
    const size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= P) return;
    size_t q;
    if (layers == 1) {
        if (u < (size_t)h1) q = u;
        else if (u < 2 * (size_t)h1) q = H1 + (u - h1);
        else if (u < 3 * (size_t)h1) q = 2 * (size_t)H1 + (u - 2 * h1);
        else q = 3 * (size_t)H1;
    } else {
        const size_t a = h1, b = 2 * (size_t)h1, c = b + (size_t)h2 * h1, d = c + h2, e = d + h2;
        if (u < a) q = u;
        else if (u < b) q = H1 + (u - a);
        else if (u < c) { const size_t v = u - b, k = v / h1, j = v % h1; q = 2 * (size_t)H1 + k * H1 + j; }
        else if (u < d) q = 2 * (size_t)H1 + (size_t)H2 * H1 + (u - c);
        else if (u < e) q = 2 * (size_t)H1 + (size_t)H2 * H1 + H2 + (u - d);
        else q = 2 * (size_t)H1 + (size_t)H2 * H1 + 2 * (size_t)H2;
    }
    dst[u] = src[q];
}

__global__ void k_pad(const float *src, float *dst, int layers, int h1, int h2, int H1, int H2, size_t P) {
    const size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= P) return;
    size_t q;
    if (layers == 1) {
        if (u < (size_t)h1) q = u;
        else if (u < 2 * (size_t)h1) q = H1 + (u - h1);
        else if (u < 3 * (size_t)h1) q = 2 * (size_t)H1 + (u - 2 * h1);
        else q = 3 * (size_t)H1;
    } else {
        const size_t a = h1, b = 2 * (size_t)h1, c = b + (size_t)h2 * h1, d = c + h2, e = d + h2;
        if (u < a) q = u;
        else if (u < b) q = H1 + (u - a);
        else if (u < c) { const size_t v = u - b, k = v / h1, j = v % h1; q = 2 * (size_t)H1 + k * H1 + j; }
        else if (u < d) q = 2 * (size_t)H1 + (size_t)H2 * H1 + (u - c);
        else if (u < e) q = 2 * (size_t)H1 + (size_t)H2 * H1 + H2 + (u - d);
        else q = 2 * (size_t)H1 + (size_t)H2 * H1 + 2 * (size_t)H2;
    }
    dst[q] = src[u];
}

extern "C" {

int nnsort_version(void) { return NNSORT_VERSION; }

const char *nnsort_strerror(int st) {
    switch (st) {
    case NNSORT_OK: return "ok";
    case NNSORT_E_INVALID_ARG: return "invalid argument";
    case NNSORT_E_NAN_KEY: return "NaN key";
    case NNSORT_E_OOM: return "out of memory";
    case NNSORT_E_BUDGET: return "over the HBM budget";
    case NNSORT_E_CUDA: return "CUDA error";
    case NNSORT_E_TIMEOUT: return "device wait timed out";
    case NNSORT_E_UNSUPPORTED: return "unsupported option";
    case NNSORT_E_STATE: return "invalid state";
    }
    return "unknown status";
}

int nnsort_last_cuda_error(void) { return g_last_cuda; }

uint64_t nnsort_launch_count(void) { return g_launches.load(); }

void nnsort_default_train_opts(nnsort_train_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->layers = 1; o->h1 = 32; o->h2 = 0;
    o->translate = NNSORT_TRANSLATE_ORDBITS;
    o->loss = NNSORT_LOSS_MSE;
    o->huber_delta = 0.01f;
    o->sample_n = 10000;
    o->steps = 100;
    o->batch = 0;
    o->lr = 1e-2f; o->beta1 = 0.9f; o->beta2 = 0.999f; o->adam_eps = 1e-8f;
    o->seed = 0;
}

void nnsort_default_sort_opts(nnsort_sort_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->m = 1.25f;
    o->eps = 3;
    o->tau = 1024;
    o->precision = NNSORT_PREC_FP32;
}

int nnsort_release(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto &kv : g_ws) {
        Workspace *w = kv.second;
        cudaSetDevice(w->device);
        cudaDeviceSynchronize();
        if (w->arena) cudaFree(w->arena);
        if (w->part) cudaFree(w->part);
        if (w->pinned) cudaFreeHost(w->pinned);
        if (w->host_dev) cudaFree(w->host_dev);
        delete w;
    }
    g_ws.clear();
    cudaSetDevice(cur);
    return NNSORT_OK;
}

int nnsort_model_create(const nnsort_model_desc *desc, const float *h_params, nnsort_model **out) {
    if (!desc || !h_params || !out) return NNSORT_E_INVALID_ARG;
    if (!dtype_ok(desc->dtype) || !arch_ok(desc->layers, desc->h1, desc->h2)) return NNSORT_E_INVALID_ARG;
    if (desc->translate != NNSORT_TRANSLATE_ORDBITS && desc->translate != NNSORT_TRANSLATE_VALUE)
        return NNSORT_E_INVALID_ARG;
    nnsort_model *f = new (std::nothrow) nnsort_model();
    if (!f) return NNSORT_E_OOM;
    f->desc = *desc;
    f->P = param_count(desc->layers, desc->h1, desc->h2);
    f->params.assign(h_params, h_params + f->P);
    f->pad = pad_arch(desc->layers, desc->h1, desc->h2);
    f->Ppad = padded_param_count(f->pad);
    f->hpad = to_padded(*desc, f->pad, h_params);
    const std::vector<float> &pp = f->hpad;
    cudaGetDevice(&f->device);
    cudaError_t e = cudaMalloc(&f->d_params, f->Ppad * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(f->d_params, pp.data(), f->Ppad * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        if (f->d_params) cudaFree(f->d_params);
        delete f;
        return NNSORT_E_CUDA;
    }
    *out = f;
    return NNSORT_OK;
}

int nnsort_model_free(nnsort_model *f) {
    if (!f) return NNSORT_E_INVALID_ARG;
    if (f->d_params && !f->owner) cudaFree(f->d_params);
    delete f;  // a shared parameter block is freed with its last model
    return NNSORT_OK;
}

int nnsort_model_describe(const nnsort_model *f, nnsort_model_desc *desc, float *h_params) {
    if (!f) return NNSORT_E_INVALID_ARG;
    if (desc) *desc = f->desc;
    if (h_params) std::memcpy(h_params, f->params.data(), f->P * sizeof(float));
    return NNSORT_OK;
}

int nnsort_mlp_pwl(int32_t layers, int32_t h1, int32_t h2, const float *h_params, double *h_breaks,
                   double *h_slope, double *h_icept, uint32_t cap, uint32_t *count) {
    if (!count || !h_params || !arch_ok(layers, h1, h2)) return NNSORT_E_INVALID_ARG;
    std::vector<double> brk, slope, icept;
    pwl_segments(layers, h1, layers == 1 ? 0 : h2, h_params, brk, slope, icept);
    *count = (uint32_t)brk.size();
    if (cap < brk.size() || !h_breaks || !h_slope || !h_icept) return NNSORT_E_INVALID_ARG;
    std::memcpy(h_breaks, brk.data(), brk.size() * sizeof(double));
    std::memcpy(h_slope, slope.data(), slope.size() * sizeof(double));
    std::memcpy(h_icept, icept.data(), icept.size() * sizeof(double));
    return NNSORT_OK;
}

static const uint32_t BLOB_MAGIC = 0x4E4E5331u;  // "NNS1"
size_t nnsort_model_blob_size(const nnsort_model *f) {
    return f ? 8 + sizeof(nnsort_model_desc) + f->P * sizeof(float) : 0;
}
int nnsort_model_save(const nnsort_model *f, void *h_blob, size_t cap) {
    if (!f || !h_blob || cap < nnsort_model_blob_size(f)) return NNSORT_E_INVALID_ARG;
    unsigned char *p = (unsigned char *)h_blob;
    const uint32_t ver = NNSORT_VERSION;
    std::memcpy(p, &BLOB_MAGIC, 4);
    std::memcpy(p + 4, &ver, 4);
    std::memcpy(p + 8, &f->desc, sizeof(nnsort_model_desc));
    std::memcpy(p + 8 + sizeof(nnsort_model_desc), f->params.data(), f->P * sizeof(float));
    return NNSORT_OK;
}
int nnsort_model_load(const void *h_blob, size_t size, nnsort_model **out) {
    if (!h_blob || !out || size < 8 + sizeof(nnsort_model_desc)) return NNSORT_E_INVALID_ARG;
    const unsigned char *p = (const unsigned char *)h_blob;
    uint32_t magic;
    std::memcpy(&magic, p, 4);
    if (magic != BLOB_MAGIC) return NNSORT_E_INVALID_ARG;
    nnsort_model_desc d;
    std::memcpy(&d, p + 8, sizeof(d));
    if (!arch_ok(d.layers, d.h1, d.h2)) return NNSORT_E_INVALID_ARG;
    const size_t P = param_count(d.layers, d.h1, d.h2);
    if (size < 8 + sizeof(d) + P * sizeof(float)) return NNSORT_E_INVALID_ARG;
    std::vector<float> params(P);
    std::memcpy(params.data(), p + 8 + sizeof(d), P * sizeof(float));
    return nnsort_model_create(&d, params.data(), out);
}

}  // extern "C"

namespace {
__device__ uint32_t g_selftest_flag;  // never set
__device__ uint32_t g_selftest_err;

__global__ void k_selftest_wait(unsigned long long limit_ns) {
    const volatile uint32_t *flag = &g_selftest_flag;
    const unsigned long long t0 = nns::globaltimer_ns();
    uint32_t polls = 0;
    while (*flag == 0u) {
        if (nns::globaltimer_ns() - t0 > limit_ns || ++polls > nns::SPIN_LIMIT_POLLS) {
            atomicOr(&g_selftest_err, nns::ERR_TIMEOUT);
            return;
        }
        __nanosleep(256);
    }
}
}  // namespace

extern "C" {

int nnsort_selftest_wait(uint32_t limit_us, cudaStream_t stream) {
    const uint32_t us = limit_us < 1u ? 1u : (limit_us > 1000000u ? 1000000u : limit_us);
    void *pf = nullptr, *pe = nullptr;
    CK(cudaGetSymbolAddress(&pf, g_selftest_flag));
    CK(cudaGetSymbolAddress(&pe, g_selftest_err));
    CK(cudaMemsetAsync(pf, 0, sizeof(uint32_t), stream));
    CK(cudaMemsetAsync(pe, 0, sizeof(uint32_t), stream));
    k_selftest_wait<<<1, 1, 0, stream>>>((unsigned long long)us * 1000ull);
    CK(cudaGetLastError());
    nns::note_launch(1);
    uint32_t e = 0;
    CK(cudaMemcpyAsync(&e, pe, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    return (e & nns::ERR_TIMEOUT) ? NNSORT_E_TIMEOUT : NNSORT_OK;
}

int nnsort_stream_status(cudaStream_t s) {
    Workspace *w = nullptr;
    int rc = get_ws(s, &w);
    if (rc) return rc;
    CK(cudaStreamSynchronize(s));
    // the training kernels' word (process-wide) holds only the timeout bit
    uint32_t te = 0;
    if (uint32_t *tw = train_err_word()) CK(cudaMemcpy(&te, tw, 4, cudaMemcpyDeviceToHost));
    if (te & ERR_TIMEOUT) return NNSORT_E_TIMEOUT;
    if (!w->last_err) return NNSORT_OK;
    uint32_t e = 0;
    CK(cudaMemcpy(&e, w->last_err, 4, cudaMemcpyDeviceToHost));
    if (e & ERR_NAN) return NNSORT_E_NAN_KEY;
    if (e & ERR_SLOT) return NNSORT_E_INVALID_ARG;
    if (e & ERR_TIMEOUT) return NNSORT_E_TIMEOUT;
    return NNSORT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// the sort pipeline over one or more arrays
namespace {

struct SegIn {
    void *keys;
    int32_t *payload;
    uint64_t n;
    const nnsort_model *f;
};

struct Layout {
    Seg *segs; SegStats *stats; uint32_t *err;
    uint32_t *gs[2]; void *key[2]; uint32_t *pay[2]; uint32_t *row[2]; uint32_t *out_rows;
    uint8_t *rank; uint8_t *g_flag; uint32_t *g_x, *g_y; uint32_t *bstart;
    OKey *bmax, *carry, *blo, *bhi;
    SeamRange *ranges; uint32_t *seam_cnt;
    uint32_t *order, *order_cnt;
    BigRange *big; uint32_t *big_cnt;
    BigRange *giant; uint32_t *giant_cnt; unsigned int *g_cnt, *g_tbmax; unsigned long long *g_kmax;
};

Layout carve(unsigned char *base, int nseg, uint64_t N, uint32_t NB, int kb, bool pay, bool rows,
             size_t *total) {
    Carve c;
    c.base = base;
    Layout L{};
    L.segs = c.take<Seg>(nseg);
    L.stats = c.take<SegStats>(nseg);
    L.err = c.take<uint32_t>(4);
    for (int i = 0; i < 2; ++i) {
        L.gs[i] = c.take<uint32_t>(N);
        L.key[i] = c.take<unsigned char>(N * kb);
        L.pay[i] = pay ? c.take<uint32_t>(N) : nullptr;
        L.row[i] = rows ? c.take<uint32_t>(N) : nullptr;
    }
    L.out_rows = rows ? c.take<uint32_t>(N) : nullptr;
    L.rank = c.take<uint8_t>(N);
    L.g_flag = c.take<uint8_t>(N);
    L.g_x = c.take<uint32_t>(N);
    L.g_y = c.take<uint32_t>(N);
    L.bstart = c.take<uint32_t>((size_t)NB + 1);
    L.bmax = c.take<OKey>((size_t)NB * MAXR);
    L.carry = c.take<OKey>((size_t)NB * MAXR);
    L.blo = c.take<OKey>(NB);
    L.bhi = c.take<OKey>(NB);
    L.ranges = c.take<SeamRange>((size_t)NB + nseg);
    L.seam_cnt = c.take<uint32_t>(4);
    L.order = c.take<uint32_t>(NB);
    L.order_cnt = c.take<uint32_t>(4);
    L.big = c.take<BigRange>(N / POLISH_BIG + 1);
    L.big_cnt = c.take<uint32_t>(4);
    L.giant = c.take<BigRange>(N / POLISH_BIG + 1);
    L.giant_cnt = c.take<uint32_t>(4);
    L.g_cnt = c.take<unsigned int>((N / POLISH_BIG + 1) * MAXR);
    L.g_tbmax = c.take<unsigned int>((N / POLISH_BIG + 1) * MAXR);
    L.g_kmax = c.take<unsigned long long>((N / POLISH_BIG + 1) * MAXR);
    *total = align_up(c.off, 256);
    return L;
}

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

struct Plan {
    int wlog;
    uint32_t NB;
    PassPlan pp;
    std::vector<Seg> segs;
    uint64_t N;
    uint32_t tiles;
};

int make_plan(const std::vector<SegIn> &in, const nnsort_sort_opts &o, int dtype, Plan &P) {
    int wlog = o.bucket_log2 ? o.bucket_log2 : 12;
    if (wlog < 9 || wlog > 14) return NNSORT_E_INVALID_ARG;
    const uint64_t W = 1ull << wlog;
    P.wlog = wlog;
    P.segs.resize(in.size());
    uint64_t e = 0, gsb = 0, tb = 0;
    uint32_t bb = 0;
    for (size_t i = 0; i < in.size(); ++i) {
        Seg &s = P.segs[i];
        std::memset(&s, 0, sizeof(s));
        const uint64_t n = in[i].n;
        const double nm = (double)n * (double)o.m;
        s.keys = in[i].keys;
        s.payload = in[i].payload;
        s.n = n;
        s.ebase = e;
        s.L = (uint64_t)std::floor(nm) + 1;
        s.nm_hi = (float)nm;
        s.nm_lo = (float)(nm - (double)s.nm_hi);
        s.gs_base = gsb;
        s.nb = (uint32_t)((s.L + W - 1) / W);
        s.bbase = bb;
        s.tbase = (uint32_t)tb;
        s.ntiles = (uint32_t)((n + PRED_TILE - 1) / PRED_TILE);
        s.eps = (uint32_t)o.eps;
        s.tau = o.tau;
        s.slots = (i == 0) ? o.d_slots : nullptr;
        if (in[i].f) {
            s.params = in[i].f->d_params;
            s.norm = norm_of(in[i].f->desc);
        } else {
            s.norm.dtype = dtype;
        }
        e += n;
        gsb += (uint64_t)s.nb * W;
        bb += s.nb;
        tb += s.ntiles;
        if (gsb >= 0xFFFFFFFFull || e >= 0xFFFFFFFFull || tb >= 0xFFFFFFFFull) return NNSORT_E_INVALID_ARG;
    }
    P.N = e;
    P.NB = bb;
    P.tiles = (uint32_t)tb;
    int bits = 1;
    while ((1ull << bits) < (uint64_t)bb) ++bits;
    const int npass = (bits + RADIX_MAX_BITS - 1) / RADIX_MAX_BITS;
    if (npass > MAX_PASSES) return NNSORT_E_INVALID_ARG;
    P.pp.npass = npass;
    P.pp.wlog = wlog;
    int sh = wlog;
    for (int p = 0; p < npass; ++p) {
        const int b = (bits - (sh - wlog) + (npass - p) - 1) / (npass - p);
        P.pp.shift[p] = sh;
        P.pp.bits[p] = b;
        sh += b;
    }
    return NNSORT_OK;
}

void fill_stats(const Seg &s, const SegStats &d, nnsort_stats *st) {
    std::memset(st, 0, sizeof(*st));
    st->rounds = d.t;
    st->eps = s.eps;
    st->n = s.n;
    st->L = s.L;
    st->tau = s.tau;
    st->w_size[0] = s.n;
    for (uint32_t r = 1; r <= d.t; ++r) st->w_size[r] = d.count_ge[r];
    for (uint32_t r = 0; r < d.t; ++r) {
        st->placed[r] = st->w_size[r] - st->w_size[r + 1];
        st->out_of_order[r] = d.ooo[r];
        st->sigma[r] = st->w_size[r] ? (double)st->w_size[r + 1] / (double)st->w_size[r] : 0.0;
        st->e[r] = st->placed[r] ? (double)st->out_of_order[r] / (double)st->placed[r] : 0.0;
    }
    st->trad_rate = s.n ? (double)st->w_size[d.t] / (double)s.n : 0.0;
    st->buckets = s.nb;
    st->oversized_buckets = d.oversized;
    st->repaired = d.repaired;
    st->repair_ranges = d.ranges;
}

// Stable multi-block radix sort of `total` packed elements: by key (every 8-bit digit of the order
// image), then, when `gmax` > 0, stably by a group index in [0, gmax] carried alongside (J). K, P, J
// are ping-pong pairs with the data in index 0 (P nullable, J null when gmax == 0). *fin receives
// the index of the pair holding the result.
int sort_packed(Workspace *w, uint64_t total, int kb, int dtype, void *const K[2], uint32_t *const P[2],
                uint32_t *const J[2], uint32_t gmax, int *fin, cudaStream_t s) {
    auto pass = [&](int si, bool keydig, int shift, int bits) -> int {
        const int di = si ^ 1;
        PartitionArgs a{};
        a.N = total;
        a.key_in = K[si];
        a.key_out = K[di];
        if (P[0]) {
            a.pay_in = P[si];
            a.pay_out = P[di];
        }
        if (keydig) {
            if (gmax) { a.row_in = J[si]; a.row_out = J[di]; }
        } else {
            a.gs_in = J[si];
            a.gs_out = J[di];
        }
        a.key_digits = keydig ? 1 : 0;
        a.shift = shift;
        a.bits = bits;
        a.key_bytes = kb;
        a.dtype = dtype;
        CK(part_pass(w, a, s));
        return NNSORT_OK;
    };
    int rc;
    const int npass = kb;  // even, so the key passes end in pair 0
    for (int p = 0; p < npass; ++p)
        if ((rc = pass(p & 1, true, 8 * p, 8))) return rc;
    *fin = 0;
    if (gmax) {
        // group-index passes of at most 9 bits
        int gbits = 1;
        while ((1ull << gbits) <= (unsigned long long)gmax) ++gbits;
        const int nsp = (gbits + RADIX_MAX_BITS - 1) / RADIX_MAX_BITS;
        if (nsp > 4) return NNSORT_E_INVALID_ARG;
        for (int q = 0, at = 0; q < nsp; ++q) {
            const int bt = (gbits - at + (nsp - q) - 1) / (nsp - q);
            if ((rc = pass(q & 1, false, at, bt))) return rc;
            at += bt;
        }
        *fin = nsp & 1;
    }
    return NNSORT_OK;
}

// the long seam ranges hr[0..nr) (host copy), sorted together: packed in output order into the
// (now free) partition buffers key[0] / pay[0], stable multi-block radix sort by key, then (when
// the ranges belong to more than one array) by array index, unpacked
int repair_long_ranges(Workspace *w, Layout &L, SeamRange *hr, uint32_t nr, int kb, int dtype,
                       bool anypay, cudaStream_t s) {
    std::sort(hr, hr + nr, [](const SeamRange &x, const SeamRange &y) {
        return x.seg != y.seg ? x.seg < y.seg : x.lo < y.lo;
    });
    uint64_t total = 0;
    for (uint32_t j = 0; j < nr; ++j) {
        hr[j].pad = (uint32_t)total;
        total += hr[j].hi - hr[j].lo;
    }
    if (total < 2) return NNSORT_OK;
    const bool multi = hr[0].seg != hr[nr - 1].seg;
    CK(cudaMemcpyAsync(L.ranges, hr, sizeof(SeamRange) * nr, cudaMemcpyHostToDevice, s));
    const int sms = sm_count();
    void *const K[2] = {L.key[0], L.key[1]};
    uint32_t *const P[2] = {anypay ? L.pay[0] : nullptr, anypay ? L.pay[1] : nullptr};
    uint32_t *const J[2] = {L.gs[0], L.gs[1]};
    CK(launch_seam_pack(L.ranges, nr, L.segs, total, kb, K[0], P[0], multi ? J[0] : nullptr, 0, sms, s));
    int fin = 0, rc;
    if ((rc = sort_packed(w, total, kb, dtype, K, P, J, multi ? hr[nr - 1].seg : 0u, &fin, s)))
        return rc;
    CK(launch_seam_pack(L.ranges, nr, L.segs, total, kb, K[fin], P[fin], nullptr, 1, sms, s));
    return NNSORT_OK;  // the next call on this stream waits before it rewrites the staging area
}

// buckets too large for one block's polish (listed by k_polish, host copy hb[0..nb)): their
// elements, packed from the partition buffers (pair `src`), sorted by key and then by bucket, and
// written to their output positions; then their first/last elements for the seam
int sort_big_buckets(Workspace *w, Layout &L, BigRange *hb, uint32_t nb, int src, int kb, int dtype,
                     bool anypay, cudaStream_t s) {
    std::sort(hb, hb + nb, [](const BigRange &x, const BigRange &y) { return x.lo < y.lo; });
    uint64_t total = 0;
    for (uint32_t j = 0; j < nb; ++j) {
        hb[j].off = (uint32_t)total;
        total += hb[j].hi - hb[j].lo;
    }
    CK(cudaMemcpyAsync(L.big, hb, sizeof(BigRange) * nb, cudaMemcpyHostToDevice, s));
    const int sms = sm_count(), o = src ^ 1;
    // pack into the free pair, then ping-pong between it and the (now dead) source pair
    void *const K[2] = {L.key[o], L.key[src]};
    uint32_t *const P[2] = {anypay ? L.pay[o] : nullptr, anypay ? L.pay[src] : nullptr};
    uint32_t *const J[2] = {L.gs[o], L.gs[src]};
    CK(launch_big_pack(L.big, nb, L.segs, total, kb, L.key[src], anypay ? L.pay[src] : nullptr, K[0], P[0],
                       nb > 1 ? J[0] : nullptr, 0, sms, s));
    int fin = 0, rc;
    if ((rc = sort_packed(w, total, kb, dtype, K, P, J, nb > 1 ? nb - 1 : 0u, &fin, s)))
        return rc;
    CK(launch_big_pack(L.big, nb, L.segs, total, kb, nullptr, nullptr, K[fin], P[fin], nullptr, 1, sms, s));
    CK(launch_big_bounds(L.big, nb, L.segs, kb, dtype, L.blo, L.bhi, s));
    return NNSORT_OK;
}

int run_sort(const std::vector<SegIn> &in, const nnsort_sort_opts *op, int dtype, nnsort_stats *st,
             cudaStream_t s) {
    nnsort_sort_opts o;
    if (op) o = *op; else nnsort_default_sort_opts(&o);
    if (!dtype_ok(dtype)) return NNSORT_E_INVALID_ARG;
    if (!(o.m > 0.0f) || o.eps < 0 || o.eps > NNSORT_MAX_ROUNDS) return NNSORT_E_INVALID_ARG;
    if (o.precision < NNSORT_PREC_FP32 || o.precision > NNSORT_PREC_PWL) return NNSORT_E_INVALID_ARG;
    if (in.size() > 1 && (o.d_slots || o.d_fate)) return NNSORT_E_INVALID_ARG;
    const nnsort_model *f0 = nullptr;
    bool anypay = false;
    for (const SegIn &x : in) {
        if (x.n && !x.keys) return NNSORT_E_INVALID_ARG;
        if (x.n >= 0xFFFFFFFFull) return NNSORT_E_INVALID_ARG;
        if (!x.f && !o.d_slots) return NNSORT_E_INVALID_ARG;
        if (x.f) {
            if (x.f->desc.dtype != dtype) return NNSORT_E_INVALID_ARG;
            if (f0 && (f0->pad.layers != x.f->pad.layers || f0->pad.h1 != x.f->pad.h1)) return NNSORT_E_INVALID_ARG;
            if (!f0) f0 = x.f;
        }
        if (x.payload) anypay = true;
    }
    Plan P;
    int rc = make_plan(in, o, dtype, P);
    if (rc) return rc;
    const int nseg = (int)in.size();
    if (st) for (int i = 0; i < nseg; ++i) fill_stats(P.segs[i], SegStats{}, &st[i]);
    if (P.N == 0) return NNSORT_OK;
    const int kb = key_bytes_of(dtype);
    const bool rows = o.d_fate != nullptr || (o.d_slots != nullptr && anypay);
    // the compiled piecewise-linear form of f: computed here on the host, staged after the layout
    const bool pwl = f0 && !o.d_slots && o.precision == NNSORT_PREC_PWL;
    std::vector<double> pbrk, pslope, picept;
    if (pwl) {
        if (nseg != 1) return NNSORT_E_UNSUPPORTED;
        pwl_segments(f0->desc.layers, f0->desc.h1, f0->desc.h2, f0->params.data(), pbrk, pslope, picept);
    }
    const size_t pwl_bytes = pbrk.size() * sizeof(PwlEntry);
    size_t need = 0;
    carve(nullptr, nseg, P.N, P.NB, kb, anypay, rows, &need);
    const size_t pwl_off = align_up(need, 256);
    Workspace *w = nullptr;
    if ((rc = get_ws(s, &w))) return rc;
    if ((rc = ensure_arena(w, pwl_off + pwl_bytes, s))) return rc;
    if ((rc = ensure_part(w, P.N, s))) return rc;
    // staging: the segment table, then the statistics, the seam counters and the long seam ranges
    // (disjoint and longer than SEAM_CTA_MAX each, so at most N / SEAM_CTA_MAX of them)
    const size_t pin_stats = align_up(sizeof(Seg) * nseg, 64);
    const size_t pin_cnt = pin_stats + align_up(sizeof(SegStats) * nseg + 16, 64);
    const size_t pin_rng = pin_cnt + 64;
    const size_t pin_big = align_up(pin_rng + sizeof(SeamRange) * (P.N / SEAM_CTA_MAX + 1), 64);
    const size_t pin_pwl = align_up(pin_big + sizeof(BigRange) * (P.N / POLISH_BIG + 1), 64);
    const size_t pin_need = pin_pwl + pwl_bytes + 256;
    if ((rc = ensure_pinned(w, pin_need, s))) return rc;
    size_t total = 0;
    Layout L = carve(w->arena, nseg, P.N, P.NB, kb, anypay, rows, &total);
    w->last_err = L.err;

    // stage the segment table through pinned memory (the previous call on this stream may still
    // read the staging area, so wait for it first)
    CK(cudaStreamSynchronize(s));
    std::memcpy(w->pinned, P.segs.data(), sizeof(Seg) * nseg);
    CK(cudaMemcpyAsync(L.segs, w->pinned, sizeof(Seg) * nseg, cudaMemcpyHostToDevice, s));
    PwlDev pwl_dev{};
    if (pwl) {
        PwlEntry *hp = reinterpret_cast<PwlEntry *>(w->pinned + pin_pwl);
        pwl_key_table(f0->desc, pbrk, pslope, picept, (double)P.segs[0].nm_hi + (double)P.segs[0].nm_lo, hp);
        PwlEntry *dp = reinterpret_cast<PwlEntry *>(w->arena + pwl_off);
        CK(cudaMemcpyAsync(dp, hp, pwl_bytes, cudaMemcpyHostToDevice, s));
        pwl_dev.tab = dp;
        pwl_dev.S = (uint32_t)pbrk.size();
    }
    CK(cudaMemsetAsync(L.stats, 0, sizeof(SegStats) * nseg, s));
    CK(cudaMemsetAsync(L.err, 0, 16, s));

    const bool timing = o.timing && st;
    if (timing && !w->ev[0])
        for (int i = 0; i < 8; ++i) CK(cudaEventCreate(&w->ev[i]));
    auto mark = [&](int i) -> cudaError_t { return timing ? cudaEventRecord(w->ev[i], s) : cudaSuccess; };
    CK(mark(0));
    const bool single = nseg == 1;
    PredictArgs pa{};
    pa.segs = L.segs;
    pa.nseg = nseg;
    pa.total_tiles = P.tiles;
    pa.gs = L.gs[0];
    pa.key_copy = single ? nullptr : L.key[0];
    pa.pay_copy = (single || !anypay) ? nullptr : L.pay[0];
    pa.row_init = rows ? L.row[0] : nullptr;
    pa.err = L.err;
    pa.key_bytes = kb;
    pa.dtype = dtype;
    pa.pwl = pwl_dev;
    pa.single_model = (single && f0 && !o.d_slots) ? 1 : 0;
    pa.host_pad = f0 ? f0->hpad.data() : nullptr;
    const PadArch arch = f0 ? f0->pad : pad_arch(1, 8, 0);
    const int prec = f0 ? o.precision : NNSORT_PREC_FP32;
    {
        cudaError_t e = launch_predict(arch, prec, pa, sm_count(), s);
        if (e == cudaErrorNotSupported) return NNSORT_E_UNSUPPORTED;
        CK(e);
    }
    CK(mark(1));
    for (int p = 0; p < P.pp.npass; ++p) {
        const int si = p & 1, di = si ^ 1;
        PartitionArgs a{};
        a.N = P.N;
        a.gs_in = L.gs[si];
        a.gs_out = L.gs[di];
        a.key_in = (p == 0 && single) ? in[0].keys : L.key[si];
        a.key_out = L.key[di];
        if (anypay) {
            a.pay_in = (p == 0 && single) ? reinterpret_cast<const uint32_t *>(in[0].payload) : L.pay[si];
            a.pay_out = L.pay[di];
        }
        if (rows) { a.row_in = L.row[si]; a.row_out = L.row[di]; }
        a.key_digits = 0;
        a.shift = P.pp.shift[p];
        a.bits = P.pp.bits[p];
        a.key_bytes = kb;
        a.dtype = dtype;
        CK(part_pass(w, a, s));
    }
    const int fi = P.pp.npass & 1, oi = fi ^ 1;
    CK(mark(2));
    CK(launch_bucket_bounds(L.gs[fi], P.N, P.NB, P.wlog, L.bstart, s));
    CK(mark(3));

    SolveArgs sa{};
    sa.segs = L.segs;
    sa.nseg = nseg;
    sa.NB = P.NB;
    sa.wlog = P.wlog;
    sa.bstart = L.bstart;
    sa.gs = L.gs[fi];
    sa.keys = L.key[fi];
    sa.pay = anypay ? L.pay[fi] : nullptr;
    sa.rows = rows ? L.row[fi] : nullptr;
    sa.rank = L.rank;
    sa.stats = L.stats;
    sa.bmax = L.bmax;
    sa.carry = L.carry;
    sa.blo = L.blo;
    sa.bhi = L.bhi;
    sa.g_flag = L.g_flag;
    sa.g_x = L.g_x;
    sa.g_y = L.g_y;
    sa.N = P.N;
    sa.fate = o.d_fate;
    sa.out_rows = L.out_rows;
    sa.key_scratch = L.key[oi];
    sa.pay_scratch = anypay ? L.pay[oi] : nullptr;
    sa.row_scratch = rows ? L.row[oi] : nullptr;
    sa.err = L.err;
    sa.key_bytes = kb;
    sa.dtype = dtype;
    const int pblocks = (o.polish_blocks >= 1 && o.polish_blocks <= 3) ? o.polish_blocks : 3;
    sa.polish_cap = polish_capacity(kb, anypay, rows, P.wlog, pblocks, &sa.polish_smem);
    sa.allow_defer = 1;
    sa.ranges = L.ranges;
    sa.max_ranges = P.NB + (uint32_t)nseg;
    sa.seam_cnt = L.seam_cnt;
    sa.seam_suf = L.bmax;  // free once the polish has run
    sa.seam_pre = L.bmax + P.NB;
    sa.seam_cut = reinterpret_cast<unsigned long long *>(L.carry);
    // buckets above POLISH_BIG elements (possible only when N exceeds it) run their rounds on the
    // whole GPU; their claim tables reuse the g_x scratch ((N / POLISH_BIG + 1) W entries of 8 bytes
    // fit in 4 N bytes for N > POLISH_BIG, W <= 2^14), which the polish needs only later
    GiantRounds gr{};
    if (P.N > POLISH_BIG) {
        sa.giant = L.giant;
        sa.giant_cnt = L.giant_cnt;
        gr.list = L.giant;
        gr.count = L.giant_cnt;
        gr.table = reinterpret_cast<unsigned long long *>(L.g_x);
        gr.cnt = L.g_cnt;
        gr.kmax = L.g_kmax;
        gr.tbmax = L.g_tbmax;
        gr.cap = (uint32_t)(P.N / POLISH_BIG + 1);
    }
    CK(launch_bucket_order(sa, (uint32_t)sa.polish_cap, L.order, L.order_cnt, s));
    sa.order = L.order;
    if (!rows) {
        sa.big = L.big;
        sa.big_cnt = L.big_cnt;
        CK(cudaMemsetAsync(L.big_cnt, 0, sizeof(uint32_t), s));
    }
    CK(launch_rounds(sa, s));
    if (sa.giant) CK(launch_giant_rounds(sa, gr, o.eps, sm_count(), s));
    CK(mark(4));
    CK(launch_finalize(sa, s));
    CK(mark(5));
    CK(launch_polish(sa, s));
    if (sa.big) {
        // buckets too large for one block: one wait, then one multi-block sort of all of them
        uint32_t *hc = reinterpret_cast<uint32_t *>(w->pinned + pin_cnt);
        CK(cudaMemcpyAsync(hc, L.big_cnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const uint32_t nbig = hc[0];
        if (nbig) {
            if (nbig > P.N / POLISH_BIG + 1) return NNSORT_E_STATE;
            BigRange *hb = reinterpret_cast<BigRange *>(w->pinned + pin_big);
            CK(cudaMemcpyAsync(hb, L.big, sizeof(BigRange) * nbig, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (uint32_t j = 0; j < nbig; ++j)
                if (hb[j].seg >= (uint32_t)nseg || hb[j].lo >= hb[j].hi || hb[j].hi > P.N) return NNSORT_E_STATE;
            if ((rc = sort_big_buckets(w, L, hb, nbig, fi, kb, dtype, anypay, s))) return rc;
        }
    }
    CK(mark(6));
    CK(launch_seam_repair(sa, sm_count(), s));
    if (sa.allow_defer) {
        // one wait at the end of the pipeline: long seam ranges run as one multi-block sort
        uint32_t *hc = reinterpret_cast<uint32_t *>(w->pinned + pin_cnt);
        CK(cudaMemcpyAsync(hc, L.seam_cnt, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        const uint32_t nlong = hc[1];
        if (nlong) {
            if (nlong > P.N / SEAM_CTA_MAX + 1) return NNSORT_E_STATE;
            SeamRange *hr = reinterpret_cast<SeamRange *>(w->pinned + pin_rng);
            CK(cudaMemcpyAsync(hr, L.ranges + (sa.max_ranges - nlong), sizeof(SeamRange) * nlong,
                               cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (uint32_t i = 0; i < nlong; ++i) {
                const SeamRange r = hr[i];
                if (r.seg >= (uint32_t)nseg || r.hi > P.segs[r.seg].n || r.lo >= r.hi) return NNSORT_E_STATE;
            }
            if ((rc = repair_long_ranges(w, L, hr, nlong, kb, dtype, anypay, s))) return rc;
        }
    }
    CK(mark(7));

    if (o.no_sync && !st) return NNSORT_OK;
    unsigned char *hp = w->pinned + pin_stats;
    CK(cudaMemcpyAsync(hp, L.stats, sizeof(SegStats) * nseg, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp + sizeof(SegStats) * nseg, L.err, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    uint32_t err = 0;
    std::memcpy(&err, hp + sizeof(SegStats) * nseg, 4);
    if (st) {
        for (int i = 0; i < nseg; ++i) {
            SegStats d;
            std::memcpy(&d, hp + sizeof(SegStats) * i, sizeof(SegStats));
            fill_stats(P.segs[i], d, &st[i]);
            st[i].partition_passes = (uint32_t)P.pp.npass;
            st[i].bucket_log2 = (uint32_t)P.wlog;
        }
        if (timing) {
            for (int i = 0; i < 7; ++i) CK(cudaEventElapsedTime(&st[0].ms_stage[i], w->ev[i], w->ev[i + 1]));
            CK(cudaEventElapsedTime(&st[0].ms_stage[7], w->ev[0], w->ev[7]));
        }
    }
    if (err & ERR_NAN) return NNSORT_E_NAN_KEY;
    if (err & ERR_SLOT) return NNSORT_E_INVALID_ARG;
    if (err & ERR_TIMEOUT) return NNSORT_E_TIMEOUT;
    return NNSORT_OK;
}

}  // namespace

extern "C" {

size_t nnsort_workspace_bytes(uint64_t n, int32_t dtype, int32_t with_payload, const nnsort_sort_opts *op) {
    nnsort_sort_opts o;
    if (op) o = *op; else nnsort_default_sort_opts(&o);
    if (!dtype_ok(dtype)) return 0;
    std::vector<SegIn> in(1);
    in[0].n = n;
    in[0].keys = (void *)1;
    Plan P;
    if (make_plan(in, o, dtype, P)) return 0;
    size_t need = 0;
    const bool rows = o.d_fate != nullptr || (o.d_slots != nullptr && with_payload);
    carve(nullptr, 1, n, P.NB, key_bytes_of(dtype), with_payload != 0, rows, &need);
    return need + part_bytes(n);
}

int nnsort_sort(void *d_keys, int32_t *d_payload, uint64_t n, int32_t dtype, const nnsort_model *f,
                const nnsort_sort_opts *o, nnsort_stats *st, cudaStream_t stream) {
    std::vector<SegIn> in(1);
    in[0] = SegIn{d_keys, d_payload, n, f};
    return run_sort(in, o, dtype, st, stream);
}

int nnsort_train_sort_host(void *h_keys, int32_t *h_payload, uint64_t n, int32_t dtype,
                           const nnsort_train_opts *to, const nnsort_sort_opts *so, nnsort_stats *st,
                           float *h_loss, cudaStream_t stream) {
    if (!dtype_ok(dtype) || !h_keys || n == 0) return NNSORT_E_INVALID_ARG;
    Workspace *w = nullptr;
    int rc = get_ws(stream, &w);
    if (rc) return rc;
    const size_t kbytes = (size_t)n * key_bytes_of(dtype), pbytes = h_payload ? (size_t)n * 4 : 0;
    const size_t need = align_up(kbytes, 256) + pbytes;
    if (need > w->host_cap) {
        CK(cudaStreamSynchronize(stream));
        if (w->host_dev) CK(cudaFree(w->host_dev));
        w->host_dev = nullptr;
        w->host_cap = 0;
        cudaError_t e = cudaMalloc(&w->host_dev, need);
        if (e != cudaSuccess) { g_last_cuda = (int)e; cudaGetLastError(); return NNSORT_E_OOM; }
        w->host_cap = need;
    }
    unsigned char *dk = (unsigned char *)w->host_dev;
    int32_t *dp = h_payload ? reinterpret_cast<int32_t *>(dk + align_up(kbytes, 256)) : nullptr;
    CK(cudaMemcpyAsync(dk, h_keys, kbytes, cudaMemcpyHostToDevice, stream));
    if (dp) CK(cudaMemcpyAsync(dp, h_payload, pbytes, cudaMemcpyHostToDevice, stream));
    nnsort_model *f = nullptr;
    rc = nnsort_train(dk, n, dtype, to, &f, h_loss, stream);
    if (rc) return rc;
    nnsort_sort_opts oo;
    if (so) oo = *so; else nnsort_default_sort_opts(&oo);
    oo.no_sync = 1;
    oo.d_slots = nullptr;
    oo.d_fate = nullptr;
    rc = nnsort_sort(dk, dp, n, dtype, f, &oo, st, stream);
    if (rc == NNSORT_OK) {
        CK(cudaMemcpyAsync(h_keys, dk, kbytes, cudaMemcpyDeviceToHost, stream));
        if (dp) CK(cudaMemcpyAsync(h_payload, dp, pbytes, cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        rc = nnsort_stream_status(stream);
    }
    nnsort_model_free(f);
    return rc;
}

int nnsort_sort_batch(void *const *d_keys, int32_t *const *d_payloads, const uint64_t *ns, int32_t count,
                      int32_t dtype, const nnsort_model *const *fs, const nnsort_sort_opts *o,
                      nnsort_stats *st, cudaStream_t stream) {
    if (count <= 0 || !d_keys || !ns || !fs) return NNSORT_E_INVALID_ARG;
    std::vector<SegIn> in(count);
    for (int i = 0; i < count; ++i)
        in[i] = SegIn{d_keys[i], d_payloads ? d_payloads[i] : nullptr, ns[i], fs[i]};
    return run_sort(in, o, dtype, st, stream);
}

int nnsort_radix_sort(void *d_keys, int32_t *d_payload, uint64_t n, int32_t dtype, cudaStream_t s) {
    if (!dtype_ok(dtype) || n >= 0xFFFFFFFFull) return NNSORT_E_INVALID_ARG;
    if (n == 0) return NNSORT_OK;
    if (!d_keys) return NNSORT_E_INVALID_ARG;
    Workspace *w = nullptr;
    int rc = get_ws(s, &w);
    if (rc) return rc;
    const int kb = key_bytes_of(dtype);
    const bool pay = d_payload != nullptr;
    Carve c;
    auto layout = [&](unsigned char *base) {
        c = Carve();
        c.base = base;
        struct { uint32_t *err; void *k1; uint32_t *p1; } r;
        r.err = c.take<uint32_t>(4);
        r.k1 = c.take<unsigned char>(n * kb);
        r.p1 = pay ? c.take<uint32_t>(n) : nullptr;
        return r;
    };
    layout(nullptr);
    if ((rc = ensure_arena(w, c.off, s))) return rc;
    if ((rc = ensure_part(w, n, s))) return rc;
    auto L = layout(w->arena);
    w->last_err = L.err;
    CK(cudaMemsetAsync(L.err, 0, 16, s));
    const int npass = kb;  // 8-bit digits; an even count, so the result ends in the caller's arrays
    void *K[2] = {d_keys, L.k1};
    uint32_t *P[2] = {reinterpret_cast<uint32_t *>(d_payload), L.p1};
    for (int p = 0; p < npass; ++p) {
        const int si = p & 1, di = si ^ 1;
        PartitionArgs a{};
        a.N = n;
        a.key_in = K[si];
        a.key_out = K[di];
        if (pay) { a.pay_in = P[si]; a.pay_out = P[di]; }
        a.key_digits = 1;
        a.shift = 8 * p;
        a.bits = 8;
        a.key_bytes = kb;
        a.dtype = dtype;
        CK(part_pass(w, a, s));
    }
    uint32_t err = 0;
    CK(cudaMemcpyAsync(&err, L.err, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return (err & ERR_TIMEOUT) ? NNSORT_E_TIMEOUT : NNSORT_OK;
}

int nnsort_sort_host(void *h_keys, int32_t *h_payload, uint64_t n, int32_t dtype, const nnsort_model *f,
                     const nnsort_sort_opts *o, nnsort_stats *st, cudaStream_t stream) {
    if (!dtype_ok(dtype) || (n && !h_keys)) return NNSORT_E_INVALID_ARG;
    if (n == 0) return nnsort_sort(nullptr, nullptr, 0, dtype, f, o, st, stream);
    Workspace *w = nullptr;
    int rc = get_ws(stream, &w);
    if (rc) return rc;
    const size_t kbytes = (size_t)n * key_bytes_of(dtype), pbytes = h_payload ? (size_t)n * 4 : 0;
    const size_t need = align_up(kbytes, 256) + pbytes;
    if (need > w->host_cap) {
        CK(cudaStreamSynchronize(stream));
        if (w->host_dev) CK(cudaFree(w->host_dev));
        w->host_dev = nullptr;
        w->host_cap = 0;
        cudaError_t e = cudaMalloc(&w->host_dev, need);
        if (e != cudaSuccess) { g_last_cuda = (int)e; cudaGetLastError(); return NNSORT_E_OOM; }
        w->host_cap = need;
    }
    unsigned char *dk = (unsigned char *)w->host_dev;
    int32_t *dp = h_payload ? reinterpret_cast<int32_t *>(dk + align_up(kbytes, 256)) : nullptr;
    CK(cudaMemcpyAsync(dk, h_keys, kbytes, cudaMemcpyHostToDevice, stream));
    if (dp) CK(cudaMemcpyAsync(dp, h_payload, pbytes, cudaMemcpyHostToDevice, stream));
    nnsort_sort_opts oo;
    if (o) oo = *o; else nnsort_default_sort_opts(&oo);
    const int32_t keep_sync = oo.no_sync;
    oo.no_sync = 1;
    rc = nnsort_sort(dk, dp, n, dtype, f, &oo, st, stream);
    if (rc) return rc;
    CK(cudaMemcpyAsync(h_keys, dk, kbytes, cudaMemcpyDeviceToHost, stream));
    if (dp) CK(cudaMemcpyAsync(h_payload, dp, pbytes, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    (void)keep_sync;
    return nnsort_stream_status(stream);
}

int nnsort_predict(const void *d_keys, uint64_t n, int32_t dtype, const nnsort_model *f, float m,
                   int32_t precision, uint32_t *d_slots, float *d_y, cudaStream_t stream) {
    if (!f || !dtype_ok(dtype) || f->desc.dtype != dtype || !(m > 0.0f)) return NNSORT_E_INVALID_ARG;
    if (precision < NNSORT_PREC_FP32 || precision > NNSORT_PREC_PWL) return NNSORT_E_INVALID_ARG;
    if (n && !d_keys) return NNSORT_E_INVALID_ARG;
    if (n >= 0xFFFFFFFFull || (double)n * m >= 4294967295.0) return NNSORT_E_INVALID_ARG;
    if (n == 0) return NNSORT_OK;
    nnsort_sort_opts o;
    nnsort_default_sort_opts(&o);
    o.m = m;
    std::vector<SegIn> in(1);
    in[0] = SegIn{const_cast<void *>(d_keys), nullptr, n, f};
    Plan P;
    int rc = make_plan(in, o, dtype, P);
    if (rc) return rc;
    std::vector<double> pbrk, pslope, picept;
    if (precision == NNSORT_PREC_PWL)
        pwl_segments(f->desc.layers, f->desc.h1, f->desc.h2, f->params.data(), pbrk, pslope, picept);
    const size_t pwl_bytes = pbrk.size() * sizeof(PwlEntry);
    Workspace *w = nullptr;
    if ((rc = get_ws(stream, &w))) return rc;
    if ((rc = ensure_arena(w, 4096 + pwl_bytes, stream))) return rc;
    if ((rc = ensure_pinned(w, 256 + pwl_bytes, stream))) return rc;
    static_assert(sizeof(Seg) <= 256, "the staged segment fits before the compiled table");
    Seg *dseg = reinterpret_cast<Seg *>(w->arena);
    uint32_t *err = reinterpret_cast<uint32_t *>(w->arena + 2048);
    CK(cudaStreamSynchronize(stream));
    std::memcpy(w->pinned, &P.segs[0], sizeof(Seg));
    CK(cudaMemcpyAsync(dseg, w->pinned, sizeof(Seg), cudaMemcpyHostToDevice, stream));
    CK(cudaMemsetAsync(err, 0, 4, stream));
    PwlDev pwl_dev{};
    if (!pbrk.empty()) {
        PwlEntry *hp = reinterpret_cast<PwlEntry *>(w->pinned + 256);
        pwl_key_table(f->desc, pbrk, pslope, picept, (double)P.segs[0].nm_hi + (double)P.segs[0].nm_lo, hp);
        PwlEntry *dp = reinterpret_cast<PwlEntry *>(w->arena + 4096);
        CK(cudaMemcpyAsync(dp, hp, pwl_bytes, cudaMemcpyHostToDevice, stream));
        pwl_dev.tab = dp;
        pwl_dev.S = (uint32_t)pbrk.size();
    }
    PredictArgs pa{};
    pa.segs = dseg;
    pa.nseg = 1;
    pa.total_tiles = P.tiles;
    pa.slots_out = d_slots;
    pa.y_out = d_y;
    pa.err = err;
    pa.key_bytes = key_bytes_of(dtype);
    pa.dtype = dtype;
    pa.pwl = pwl_dev;
    pa.single_model = 1;
    pa.host_pad = f->hpad.data();
    w->last_err = err;
    cudaError_t e = launch_predict(f->pad, precision, pa, sm_count(), stream);
    if (e == cudaErrorNotSupported) return NNSORT_E_UNSUPPORTED;
    CK(e);
    return NNSORT_OK;
}

// ---- training
int nnsort_sample_labels(const void *d_keys, uint64_t n, int32_t dtype, uint64_t S, uint64_t seed,
                         int32_t translate, nnsort_model_desc *desc_out, float *d_x, float *d_label,
                         uint32_t *d_rows, cudaStream_t s) {
    if (!d_keys || n == 0 || S == 0 || !dtype_ok(dtype) || S >= 0xFFFFFFFFull) return NNSORT_E_INVALID_ARG;
    if (translate != NNSORT_TRANSLATE_ORDBITS && translate != NNSORT_TRANSLATE_VALUE) return NNSORT_E_INVALID_ARG;
    const int kb = key_bytes_of(dtype);
    const int npass = kb;  // 8-bit digits
    Workspace *w = nullptr;
    int rc = get_ws(s, &w);
    if (rc) return rc;
    Carve c;
    auto lay = [&](unsigned char *base) {
        c = Carve();
        c.base = base;
        struct { void *k[2]; uint32_t *r[2]; uint32_t *err; Norm *norm; } L;
        L.k[0] = c.take<unsigned char>(S * kb);
        L.k[1] = c.take<unsigned char>(S * kb);
        L.r[0] = c.take<uint32_t>(S);
        L.r[1] = c.take<uint32_t>(S);
        L.err = c.take<uint32_t>(4);
        L.norm = c.take<Norm>(1);
        return L;
    };
    lay(nullptr);
    if ((rc = ensure_arena(w, c.off + 1024, s))) return rc;
    auto L = lay(w->arena);
    if ((rc = ensure_part(w, S, s))) return rc;
    if ((rc = ensure_pinned(w, 256, s))) return rc;
    CK(cudaMemsetAsync(L.err, 0, 16, s));
    CK(launch_sample(d_keys, n, kb, dtype, S, rng_h(seed, TAG_SAMPLE), L.k[0], L.r[0], L.err, s));
    for (int p = 0; p < npass; ++p) {
        const int si = p & 1, di = si ^ 1;
        PartitionArgs a{};
        a.N = S;
        a.key_in = L.k[si];
        a.key_out = L.k[di];
        a.row_in = L.r[si];
        a.row_out = L.r[di];
        a.key_digits = 1;
        a.shift = 8 * p;
        a.bits = 8;
        a.key_bytes = kb;
        a.dtype = dtype;
        CK(part_pass(w, a, s));
    }
    const int fi = npass & 1;  // even pass count -> result back in buffer 0
    // extremes of the sorted sample -> normaliser (host scalar set-up)
    unsigned char *hp = w->pinned;
    CK(cudaMemcpyAsync(hp, L.k[fi], kb, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp + 8, (unsigned char *)L.k[fi] + (S - 1) * kb, kb, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(hp + 16, L.err, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    uint32_t err;
    std::memcpy(&err, hp + 16, 4);
    if (err & ERR_NAN) return NNSORT_E_NAN_KEY;
    if (err & ERR_TIMEOUT) return NNSORT_E_TIMEOUT;
    uint64_t wlo = 0, whi = 0;
    std::memcpy(&wlo, hp, kb);
    std::memcpy(&whi, hp + 8, kb);
    auto ordh = [&](uint64_t wv) -> uint64_t {
        if (dtype == NNSORT_F32) { const uint32_t b = (uint32_t)wv; return (b & 0x80000000u) ? (uint64_t)(uint32_t)~b : (uint64_t)(b | 0x80000000u); }
        if (dtype == NNSORT_F64) return (wv >> 63) ? ~wv : (wv | 0x8000000000000000ull);
        return wv;
    };
    auto valh = [&](uint64_t wv) -> double {
        if (dtype == NNSORT_F32) { float f; uint32_t b = (uint32_t)wv; std::memcpy(&f, &b, 4); return (double)f; }
        if (dtype == NNSORT_F64) { double d; std::memcpy(&d, &wv, 8); return d; }
        if (dtype == NNSORT_U32) return (double)(uint32_t)wv;
        return (double)wv;
    };
    nnsort_model_desc d;
    std::memset(&d, 0, sizeof(d));
    d.dtype = dtype;
    d.translate = translate;
    const uint64_t lo = ordh(wlo), hi = ordh(whi);
    d.lo_bits = lo;
    d.lo_val = valh(wlo);
    const bool ob = translate == NNSORT_TRANSLATE_ORDBITS || dtype == NNSORT_U32 || dtype == NNSORT_U64;
    if (ob) d.scale = (hi > lo) ? 1.0 / (double)(hi - lo) : 1.0;
    else { const double hv = valh(whi); d.scale = (hv > d.lo_val) ? 1.0 / (hv - d.lo_val) : 1.0; }
    if (desc_out) *desc_out = d;
    const Norm nm = norm_of(d);
    std::memcpy(hp + 64, &nm, sizeof(Norm));
    CK(cudaMemcpyAsync(L.norm, hp + 64, sizeof(Norm), cudaMemcpyHostToDevice, s));
    if (d_x || d_label) {
        float *x = d_x, *lab = d_label;
        if (!x || !lab) return NNSORT_E_INVALID_ARG;
        CK(launch_make_xy(L.k[fi], S, kb, L.norm, x, lab, s));
    }
    if (d_rows) CK(cudaMemcpyAsync(d_rows, L.r[fi], S * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    return NNSORT_OK;
}

static void init_params_host(int layers, int h1, int h2, uint64_t seed, float *p) {
    const uint64_t s = rng_h(seed, TAG_INIT);
    uint64_t c = 0;
    const double r1 = std::sqrt(6.0);
    for (int j = 0; j < h1; ++j) p[j] = (float)((2.0 * unit53h(rng_h(s, c++)) - 1.0) * r1);
    for (int j = 0; j < h1; ++j) {
        const double cj = unit53h(rng_h(s, c++));
        p[h1 + j] = (float)(-(double)p[j] * cj);
    }
    float *q = p + 2 * h1;
    int HL = h1;
    if (layers == 2) {
        const double r2 = std::sqrt(6.0 / h1);
        for (int k = 0; k < h2 * h1; ++k) q[k] = (float)((2.0 * unit53h(rng_h(s, c++)) - 1.0) * r2);
        q += (size_t)h2 * h1;
        for (int k = 0; k < h2; ++k) q[k] = 0.0f;
        q += h2;
        HL = h2;
    }
    const double r3 = std::sqrt(6.0 / HL);
    for (int k = 0; k < HL; ++k) q[k] = (float)((2.0 * unit53h(rng_h(s, c++)) - 1.0) * r3);
    q[HL] = 0.0f;
}

static_assert(NNSORT_TRAIN_BLOCK_MAX_S == TB_MAX_S, "header and kernel agree on the sample limit");

static bool block_trainable(const nnsort_train_opts &o, uint64_t S) {
    return o.layers == 1 && o.h1 >= 1 && o.h1 <= 32 && !o.monotone && S >= 1 && S <= TB_MAX_S;
}

int nnsort_train_batch(void *const *d_keys, const uint64_t *ns, int32_t count, int32_t dtype,
                       const nnsort_train_opts *op, const uint64_t *sample_ns, nnsort_model **out,
                       float *h_loss, cudaStream_t s) {
    nnsort_train_opts o;
    if (op) o = *op; else nnsort_default_train_opts(&o);
    if (count < 0 || (count > 0 && (!d_keys || !ns || !out)) || !dtype_ok(dtype)) return NNSORT_E_INVALID_ARG;
    if (!arch_ok(o.layers, o.h1, o.h2) || o.loss < 0 || o.loss > 1) return NNSORT_E_INVALID_ARG;
    if (count == 0) return NNSORT_OK;
    std::vector<uint64_t> S(count), N(count), K(count);
    for (int j = 0; j < count; ++j) {
        S[j] = sample_ns ? sample_ns[j] : o.sample_n;
        N[j] = ns[j];
        K[j] = reinterpret_cast<uint64_t>(d_keys[j]);
        if (!d_keys[j] || ns[j] == 0) return NNSORT_E_INVALID_ARG;
        if (!block_trainable(o, S[j])) return NNSORT_E_UNSUPPORTED;
        out[j] = nullptr;
    }
    const PadArch pa = pad_arch(1, o.h1, 0);
    const size_t Pp = padded_param_count(pa), P = param_count(1, o.h1, 0);
    const int steps = (int)o.steps;
    // models by sample-size class, so each launch's shared sort buffer fits its largest sample
    const uint32_t caps[3] = {1024, 4096, TB_MAX_S};
    std::vector<uint32_t> ids;
    uint32_t first[4] = {0, 0, 0, 0};
    for (int c = 0; c < 3; ++c) {
        first[c] = (uint32_t)ids.size();
        for (int j = 0; j < count; ++j)
            if (S[j] <= caps[c] && (c == 0 || S[j] > caps[c - 1])) ids.push_back((uint32_t)j);
    }
    first[3] = (uint32_t)ids.size();
    // one device block: tables, outputs, bias corrections, error word
    const size_t off_n = (size_t)count * 8, off_s = off_n + (size_t)count * 8, off_ids = off_s + (size_t)count * 8;
    const size_t off_c = align_up(off_ids + (size_t)count * 4, 16);
    const size_t off_par = align_up(off_c + (size_t)std::max(steps, 1) * 8, 16);
    const size_t off_norm = align_up(off_par + (size_t)count * Pp * 4, 16);
    const size_t off_loss = align_up(off_norm + (size_t)count * sizeof(Norm), 16);
    const size_t off_err = align_up(off_loss + (h_loss ? (size_t)count * steps * 4 : 0), 16);
    const size_t total = off_err + 16;
    std::vector<unsigned char> host(total, 0);
    std::memcpy(host.data(), K.data(), (size_t)count * 8);
    std::memcpy(host.data() + off_n, N.data(), (size_t)count * 8);
    std::memcpy(host.data() + off_s, S.data(), (size_t)count * 8);
    std::memcpy(host.data() + off_ids, ids.data(), (size_t)count * 4);
    for (int t = 0; t < steps; ++t) {
        const float c1 = (float)(1.0 - std::pow((double)o.beta1, (double)(t + 1)));
        const float c2 = (float)(1.0 - std::pow((double)o.beta2, (double)(t + 1)));
        std::memcpy(host.data() + off_c + (size_t)t * 4, &c1, 4);
        std::memcpy(host.data() + off_c + (size_t)(steps + t) * 4, &c2, 4);
    }
    unsigned char *dev = nullptr;
    CK(cudaMallocAsync((void **)&dev, total, s));
    // the trained parameters stay where the kernel writes them: one device block that the models
    // share (each model's padded parameters are a slice; the block is freed with the last model)
    float *dpar = nullptr;
    cudaError_t e = cudaMalloc((void **)&dpar, (size_t)count * Pp * sizeof(float));
    if (e != cudaSuccess) {
        cudaFreeAsync(dev, s);
        g_last_cuda = (int)e;
        return NNSORT_E_OOM;
    }
    std::shared_ptr<void> block(dpar, [](void *p) { cudaFree(p); });
    e = cudaMemcpyAsync(dev, host.data(), off_par, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev + off_err, 0, 16, s);
    TrainBlockArgs a{};
    a.keys = reinterpret_cast<const void *const *>(dev);
    a.n = reinterpret_cast<const uint64_t *>(dev + off_n);
    a.S = reinterpret_cast<const uint64_t *>(dev + off_s);
    a.dtype = dtype;
    a.translate = o.translate;
    a.h1 = o.h1;
    a.seed0 = o.seed;
    a.steps = steps;
    a.batch = o.batch;
    a.loss = o.loss;
    a.delta = o.huber_delta;
    a.lr = o.lr; a.b1 = o.beta1; a.b2 = o.beta2; a.eps = o.adam_eps;
    a.c1 = reinterpret_cast<const float *>(dev + off_c);
    a.c2 = a.c1 + steps;
    a.params_out = dpar;
    a.norm_out = reinterpret_cast<Norm *>(dev + off_norm);
    a.loss_out = h_loss ? reinterpret_cast<float *>(dev + off_loss) : nullptr;
    a.err = reinterpret_cast<uint32_t *>(dev + off_err);
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
        uint32_t cap = 2;
        for (uint32_t i = first[c]; i < first[c + 1]; ++i)
            while (cap < S[ids[i]]) cap <<= 1;
        a.ids = reinterpret_cast<const uint32_t *>(dev + off_ids) + first[c];
        a.cap = cap;
        e = launch_train_block(a, key_bytes_of(dtype), pa.h1, first[c + 1] - first[c], s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host.data() + off_par, dpar, (size_t)count * Pp * sizeof(float),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host.data() + off_norm, dev + off_norm, total - off_norm,
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(dev, s);
    if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        return NNSORT_E_CUDA;
    }
    uint32_t err = 0;
    std::memcpy(&err, host.data() + off_err, 4);
    if (err & ERR_NAN) return NNSORT_E_NAN_KEY;
    if (h_loss) std::memcpy(h_loss, host.data() + off_loss, (size_t)count * steps * 4);
    std::vector<float> up(P);
    for (int j = 0; j < count; ++j) {
        Norm q;
        std::memcpy(&q, host.data() + off_norm + (size_t)j * sizeof(Norm), sizeof(Norm));
        nnsort_model_desc d;
        std::memset(&d, 0, sizeof(d));
        d.dtype = dtype;
        d.translate = o.translate;
        d.layers = 1;
        d.h1 = o.h1;
        d.lo_bits = q.lo_bits;
        d.lo_val = q.lo_val;
        d.scale = q.scale;
        const float *pp = reinterpret_cast<const float *>(host.data() + off_par) + (size_t)j * Pp;
        for (size_t u = 0; u < P; ++u) up[u] = pp[pad_index(1, o.h1, 0, pa, u)];
        nnsort_model *f = new (std::nothrow) nnsort_model();
        if (!f) {
            for (int q2 = 0; q2 < j; ++q2) { nnsort_model_free(out[q2]); out[q2] = nullptr; }
            return NNSORT_E_OOM;
        }
        f->desc = d;
        f->P = P;
        f->params = up;
        f->pad = pa;
        f->Ppad = Pp;
        f->hpad.assign(pp, pp + Pp);
        f->d_params = dpar + (size_t)j * Pp;
        f->owner = block;
        cudaGetDevice(&f->device);
        out[j] = f;
    }
    return NNSORT_OK;
}

int nnsort_train(const void *d_keys, uint64_t n, int32_t dtype, const nnsort_train_opts *op,
                 nnsort_model **out, float *h_loss, cudaStream_t s) {
    nnsort_train_opts o;
    if (op) o = *op; else nnsort_default_train_opts(&o);
    if (!out || !d_keys || n == 0 || !dtype_ok(dtype) || !arch_ok(o.layers, o.h1, o.h2)) return NNSORT_E_INVALID_ARG;
    if (o.sample_n == 0 || o.loss < 0 || o.loss > 1) return NNSORT_E_INVALID_ARG;
    const uint64_t S = o.sample_n;
    const uint64_t B = o.batch ? o.batch : S;
    const PadArch pa = pad_arch(o.layers, o.h1, o.h2);
    const size_t Pp = padded_param_count(pa), P = param_count(o.layers, o.h1, o.h2);
    const int blocks = train_grad_blocks(pa, B);
    uint32_t *terr = train_err_word();
    if (!terr) return NNSORT_E_CUDA;
    // device buffers for this call (separate from the per-stream arena used by sampling)
    float *dx = nullptr;
    const uint32_t nst = std::max<uint32_t>(o.steps, 1);
    const size_t fl = S * 2 + Pp * 5 + (size_t)blocks * Pp + blocks + nst + 2 * (size_t)nst + 64;
    CK(cudaMallocAsync((void **)&dx, fl * sizeof(float), s));
    float *dlab = dx + S, *dp = dlab + S, *dm = dp + Pp, *dv = dm + Pp, *dg = dv + Pp;
    float *dmask = dg + Pp;
    float *dpart = dmask + Pp, *dlp = dpart + (size_t)blocks * Pp, *dloss = dlp + blocks;
    float *dc12 = dloss + nst;                                           // [2 * steps]
    unsigned int *dcount = reinterpret_cast<unsigned int *>(dc12 + 2 * (size_t)nst);  // [1]
    nnsort_model_desc d;
    int rc = nnsort_sample_labels(d_keys, n, dtype, S, o.seed, o.translate, &d, dx, dlab, nullptr, s);
    if (rc) { cudaFreeAsync(dx, s); return rc; }
    d.layers = o.layers; d.h1 = o.h1; d.h2 = o.h2;
    std::vector<float> p0(P);
    init_params_host(o.layers, o.h1, o.h2, o.seed, p0.data());
    std::vector<float> mask;
    if (o.monotone) {
        // sign structure: layer-1 unit j keeps sign s_j of W1_j; with two hidden layers output
        // unit k keeps sign q_k of W3_k and W2_kj carries s_j q_k; with one, W3_j carries s_j
        std::vector<float> sg(P, 0.0f);
        for (int j = 0; j < o.h1; ++j) sg[j] = p0[j] >= 0.0f ? 1.0f : -1.0f;
        if (o.layers == 1) {
            for (int j = 0; j < o.h1; ++j) sg[2 * o.h1 + j] = sg[j];
        } else {
            const size_t w2 = 2 * (size_t)o.h1, w3 = w2 + (size_t)o.h2 * o.h1 + o.h2;
            for (int k = 0; k < o.h2; ++k) {
                const float q = p0[w3 + k] >= 0.0f ? 1.0f : -1.0f;
                sg[w3 + k] = q;
                for (int j = 0; j < o.h1; ++j) sg[w2 + (size_t)k * o.h1 + j] = sg[j] * q;
            }
        }
        for (size_t u = 0; u < P; ++u)
            if (sg[u] != 0.0f) p0[u] = sg[u] * std::fabs(p0[u]);
        mask = to_padded(d, pa, sg.data());
        CK(cudaMemcpyAsync(dmask, mask.data(), Pp * sizeof(float), cudaMemcpyHostToDevice, s));
    }
    const std::vector<float> pp = to_padded(d, pa, p0.data());
    CK(cudaMemcpyAsync(dp, pp.data(), Pp * sizeof(float), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(dm, 0, 2 * Pp * sizeof(float), s));
    TrainStepArgs t{};
    t.params = dp; t.m = dm; t.v = dv; t.grad = dg; t.partials = dpart; t.loss_partials = dlp;
    t.loss_out = dloss; t.x = dx; t.label = dlab; t.S = S; t.batch = o.batch;
    t.batch_seed = rng_h(o.seed, TAG_BATCH); t.loss = o.loss; t.delta = o.huber_delta;
    t.lr = o.lr; t.b1 = o.beta1; t.b2 = o.beta2; t.eps = o.adam_eps; t.P = Pp;
    t.mask = o.monotone ? dmask : nullptr;
    CK(cudaMemsetAsync(terr, 0, sizeof(uint32_t), s));
    if (pa.layers == 2 && pa.h1 == 64) {
        // every step in one cooperative launch (its blocks meet twice per step)
        std::vector<float> c12(2 * (size_t)nst);
        for (uint32_t k = 0; k < o.steps; ++k) {
            c12[k] = (float)(1.0 - std::pow((double)o.beta1, (double)(k + 1)));
            c12[o.steps + k] = (float)(1.0 - std::pow((double)o.beta2, (double)(k + 1)));
        }
        CK(cudaMemcpyAsync(dc12, c12.data(), c12.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        CK(cudaMemsetAsync(dcount, 0, sizeof(unsigned int), s));
        CK(launch_train_tc64(t, o.steps, dc12, dcount, s));
    } else {
        for (uint32_t k = 0; k < o.steps; ++k) {
            t.step = (int)k;
            CK(launch_train_step(pa, t, s));
        }
    }
    std::vector<float> hpp(Pp);
    CK(cudaMemcpyAsync(hpp.data(), dp, Pp * sizeof(float), cudaMemcpyDeviceToHost, s));
    std::vector<float> hl(std::max<uint32_t>(o.steps, 1));
    if (o.steps) CK(cudaMemcpyAsync(hl.data(), dloss, o.steps * sizeof(float), cudaMemcpyDeviceToHost, s));
    uint32_t herr = 0;
    CK(cudaMemcpyAsync(&herr, terr, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    cudaFreeAsync(dx, s);
    if (herr & ERR_TIMEOUT) return NNSORT_E_TIMEOUT;
    if (h_loss) std::memcpy(h_loss, hl.data(), o.steps * sizeof(float));
    std::vector<float> up(P);
    for (size_t u = 0; u < P; ++u) up[u] = hpp[pad_index(o.layers, o.h1, o.h2, pa, u)];
    return nnsort_model_create(&d, up.data(), out);
}

// ---- explicit forward / backward (autograd)
static int with_padded(const float *d_params, int layers, int h1, int h2, cudaStream_t s,
                       float **dpad, PadArch *pa, size_t extra_floats, float **extra) {
    if (!arch_ok(layers, h1, h2) || !d_params) return NNSORT_E_INVALID_ARG;
    *pa = pad_arch(layers, h1, h2);
    const size_t Pp = padded_param_count(*pa), P = param_count(layers, h1, h2);
    float *buf = nullptr;
    CK(cudaMallocAsync((void **)&buf, (Pp + extra_floats) * sizeof(float), s));
    CK(cudaMemsetAsync(buf, 0, Pp * sizeof(float), s));
    k_pad<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(d_params, buf, layers, h1, h2, pa->h1, pa->h2, P);
    CK(cudaGetLastError());
    note_launch(1);
    *dpad = buf;
    *extra = buf + Pp;
    return NNSORT_OK;
}

int nnsort_mlp_forward(const float *d_params, int32_t layers, int32_t h1, int32_t h2, const float *d_x,
                       uint64_t n, float *d_y, cudaStream_t s) {
    if ((n && (!d_x || !d_y))) return NNSORT_E_INVALID_ARG;
    float *pp = nullptr, *ex = nullptr;
    PadArch pa;
    int rc = with_padded(d_params, layers, h1, h2, s, &pp, &pa, 0, &ex);
    if (rc) return rc;
    CK(launch_mlp_forward(pa, pp, d_x, n, d_y, s));
    CK(cudaFreeAsync(pp, s));
    return NNSORT_OK;
}

static int backward_common(const float *d_params, int layers, int h1, int h2, const float *d_x,
                           const float *d_gy, const float *d_label, uint64_t n, int mode, int loss,
                           float delta, float *d_loss, float *d_gparams, float *d_gx, cudaStream_t s) {
    if (!d_gparams || (n && !d_x)) return NNSORT_E_INVALID_ARG;
    PadArch pa = pad_arch(layers, h1, h2);
    const size_t Pp = padded_param_count(pa), P = param_count(layers, h1, h2);
    const int blocks = train_grad_blocks(pa, n);
    float *pp = nullptr, *ex = nullptr;
    int rc = with_padded(d_params, layers, h1, h2, s, &pp, &pa, (size_t)blocks * Pp + blocks + Pp + 4, &ex);
    if (rc) return rc;
    float *part = ex, *lp = part + (size_t)blocks * Pp, *gpad = lp + blocks;
    if (n == 0) {
        CK(cudaMemsetAsync(d_gparams, 0, P * sizeof(float), s));
        if (d_loss) CK(cudaMemsetAsync(d_loss, 0, sizeof(float), s));
        CK(cudaFreeAsync(pp, s));
        return NNSORT_OK;
    }
    int nb = 0;
    CK(launch_mlp_backward(pa, pp, d_x, d_gy, d_label, n, mode, loss, delta, part, lp, d_gx, s, &nb));
    CK(launch_reduce_partials(part, nb, Pp, gpad, lp, d_loss, 1.0f / (float)n, s));
    k_unpad<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(gpad, d_gparams, layers, h1, h2, pa.h1, pa.h2, P);
    CK(cudaGetLastError());
    note_launch(1);
    CK(cudaFreeAsync(pp, s));
    return NNSORT_OK;
}

int nnsort_mlp_backward(const float *d_params, int32_t layers, int32_t h1, int32_t h2, const float *d_x,
                        const float *d_gy, uint64_t n, float *d_gparams, float *d_gx, cudaStream_t s) {
    if (n && !d_gy) return NNSORT_E_INVALID_ARG;
    return backward_common(d_params, layers, h1, h2, d_x, d_gy, nullptr, n, 0, 0, 0.0f, nullptr,
                           d_gparams, d_gx, s);
}

int nnsort_mlp_loss_grad(const float *d_params, int32_t layers, int32_t h1, int32_t h2, const float *d_x,
                         const float *d_label, uint64_t n, int32_t loss, float huber_delta, float *d_loss,
                         float *d_gparams, cudaStream_t s) {
    if ((n && !d_label) || loss < 0 || loss > 1) return NNSORT_E_INVALID_ARG;
    return backward_common(d_params, layers, h1, h2, d_x, nullptr, d_label, n, 1, loss, huber_delta,
                           d_loss, d_gparams, nullptr, s);
}

}  // extern "C"
