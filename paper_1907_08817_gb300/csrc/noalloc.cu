// noalloc.cu -- nnsort_sort_noalloc: the sort for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc (or any allocating runtime/library routine) at the point
// where they need to sort: code running under a strict memory budget that was fixed up front,
// code that must not synchronise the device (cudaFree does), or hosts whose allocator is owned by
// another framework. This entry point runs the same kernels as nnsort_sort, but every scratch
// buffer lives in one file-scope device array of fixed size that is loaded with the library. The
// caller still passes (and owns) the keys, the payload and the model.
//
// The array is shared by every call in the process on a given device and keeps the previous
// call's contents; the call clears what must start at zero. Calls whose work overlaps on the GPU
// (for example on two streams) race on the array.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace nns;

namespace {

constexpr uint64_t NA_MAX_N = NNSORT_NOALLOC_MAX_N;
constexpr uint32_t NA_MAX_BUCKETS = 1024;
constexpr uint64_t NA_MAX_TILES = (NA_MAX_N + SC_TILE - 1) / SC_TILE;
constexpr uint64_t NA_MAX_CHUNKS = (NA_MAX_TILES + SC_CHUNK - 1) / SC_CHUNK;
constexpr size_t NA_PER_ELEM = 2 * 4 + 2 * 8 + 2 * 4 + 1 + 1 + 2 * 4;  // gs, keys, payload, rank,
                                                                      // flag, two index lists
constexpr size_t NA_BYTES = NA_MAX_N * NA_PER_ELEM + (size_t)NA_MAX_BUCKETS * (4 + 2 * MAXR * 16 + 32) +
                            NA_MAX_TILES * RADIX_BINS * 2 + NA_MAX_CHUNKS * RADIX_BINS * 4 + RADIX_BINS * 4 +
                            (size_t)(NA_MAX_BUCKETS + 1) * sizeof(SeamRange) + 64 * 1024;

// the scratch: one per device that loads the library, held until the process exits
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

struct DevState {
    unsigned char *base = nullptr;  // device address of g_noalloc_scratch on this device
};
std::mutex g_na_mu;
DevState g_na_dev[64];
thread_local int g_na_cuda = 0;

#define NA_CK(x)                              \
    do {                                      \
        cudaError_t e_ = (x);                 \
        if (e_ != cudaSuccess) {              \
            g_na_cuda = (int)e_;              \
            return NNSORT_E_CUDA;             \
        }                                     \
    } while (0)

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

struct NaLayout {
    Seg *seg; SegStats *stats; uint32_t *err;
    uint32_t *gs[2]; void *key[2]; uint32_t *pay[2];
    uint8_t *rank, *flag; uint32_t *gx, *gy, *bstart;
    OKey *bmax, *carry, *blo, *bhi;
    SeamRange *ranges; uint32_t *seam_cnt;
    uint16_t *tile_hist; uint32_t *chunk, *bin_total;
    size_t end;
};

NaLayout na_carve(unsigned char *b) {
    NaLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { o = a256(o); unsigned char *p = b + o; o += bytes; return p; };
    L.seg = reinterpret_cast<Seg *>(take(sizeof(Seg)));
    L.stats = reinterpret_cast<SegStats *>(take(sizeof(SegStats)));
    L.err = reinterpret_cast<uint32_t *>(take(16));
    for (int i = 0; i < 2; ++i) {
        L.gs[i] = reinterpret_cast<uint32_t *>(take(4 * NA_MAX_N));
        L.key[i] = take(8 * NA_MAX_N);
        L.pay[i] = reinterpret_cast<uint32_t *>(take(4 * NA_MAX_N));
    }
    L.rank = take(NA_MAX_N);
    L.flag = take(NA_MAX_N);
    L.gx = reinterpret_cast<uint32_t *>(take(4 * NA_MAX_N));
    L.gy = reinterpret_cast<uint32_t *>(take(4 * NA_MAX_N));
    L.bstart = reinterpret_cast<uint32_t *>(take(4 * (NA_MAX_BUCKETS + 1)));
    L.bmax = reinterpret_cast<OKey *>(take(sizeof(OKey) * NA_MAX_BUCKETS * MAXR));
    L.carry = reinterpret_cast<OKey *>(take(sizeof(OKey) * NA_MAX_BUCKETS * MAXR));
    L.blo = reinterpret_cast<OKey *>(take(sizeof(OKey) * NA_MAX_BUCKETS));
    L.bhi = reinterpret_cast<OKey *>(take(sizeof(OKey) * NA_MAX_BUCKETS));
    L.ranges = reinterpret_cast<SeamRange *>(take(sizeof(SeamRange) * (NA_MAX_BUCKETS + 1)));
    L.seam_cnt = reinterpret_cast<uint32_t *>(take(16));
    L.tile_hist = reinterpret_cast<uint16_t *>(take(2 * NA_MAX_TILES * RADIX_BINS));
    L.chunk = reinterpret_cast<uint32_t *>(take(4 * NA_MAX_CHUNKS * RADIX_BINS));
    L.bin_total = reinterpret_cast<uint32_t *>(take(4 * RADIX_BINS));
    L.end = o;
    return L;
}

// one-time set-up on the current device: the scratch's device address
int na_setup(int dev, DevState **out) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (dev < 0 || dev >= 64) return NNSORT_E_INVALID_ARG;
    DevState &d = g_na_dev[dev];
    if (!d.base) {
        unsigned char *p = nullptr;
        NA_CK(cudaGetSymbolAddress((void **)&p, g_noalloc_scratch));
        if (na_carve(p).end > NA_BYTES) return NNSORT_E_INVALID_ARG;  // layout/size mismatch
        d.base = p;
    }
    *out = &d;
    return NNSORT_OK;
}

int na_kb(int dt) { return (dt == NNSORT_F32 || dt == NNSORT_U32) ? 4 : 8; }

}  // namespace

extern "C" int nnsort_sort_noalloc(void *d_keys, int32_t *d_payload, uint64_t n, int32_t dtype,
                                   const nnsort_model *f, const nnsort_sort_opts *op, nnsort_stats *st,
                                   cudaStream_t s) {
    nnsort_sort_opts o;
    if (op) o = *op; else nnsort_default_sort_opts(&o);
    if (dtype < NNSORT_F32 || dtype > NNSORT_U64 || !f || f->desc.dtype != dtype) return NNSORT_E_INVALID_ARG;
    if (n > NA_MAX_N) return NNSORT_E_INVALID_ARG;  // beyond the fixed scratch
    if (o.d_slots || o.d_fate) return NNSORT_E_INVALID_ARG;
    if (!(o.m > 0.0f) || o.eps < 0 || o.eps > NNSORT_MAX_ROUNDS) return NNSORT_E_INVALID_ARG;
    if (o.precision < NNSORT_PREC_FP32 || o.precision > NNSORT_PREC_BF16X2) return NNSORT_E_INVALID_ARG;
    const int wlog = o.bucket_log2 ? o.bucket_log2 : 12;
    if (wlog < 9 || wlog > 14) return NNSORT_E_INVALID_ARG;
    if (st) std::memset(st, 0, sizeof(*st));
    if (n == 0) return NNSORT_OK;
    if (!d_keys) return NNSORT_E_INVALID_ARG;

    // host scalar set-up of the paper's definitions (same as nnsort_sort); the position count
    // L = floor(n m) + 1 must fit the fixed bucket tables before anything is narrowed
    const double nm = (double)n * (double)o.m;
    if (!std::isfinite(nm) || std::floor(nm) + 1.0 > (double)((uint64_t)NA_MAX_BUCKETS << wlog))
        return NNSORT_E_INVALID_ARG;
    Seg sg;
    std::memset(&sg, 0, sizeof(sg));
    sg.keys = d_keys;
    sg.payload = d_payload;
    sg.n = n;
    sg.L = (uint64_t)std::floor(nm) + 1;
    sg.nm_hi = (float)nm;
    sg.nm_lo = (float)(nm - (double)sg.nm_hi);
    sg.nb = (uint32_t)((sg.L + (1ull << wlog) - 1) >> wlog);
    sg.ntiles = (uint32_t)((n + PRED_TILE - 1) / PRED_TILE);
    sg.eps = (uint32_t)o.eps;
    sg.tau = o.tau;
    sg.params = f->d_params;
    sg.norm.dtype = f->desc.dtype;
    sg.norm.translate = f->desc.translate;
    sg.norm.lo_bits = f->desc.lo_bits;
    sg.norm.lo_val = f->desc.lo_val;
    sg.norm.scale = f->desc.scale;
    sg.norm.lo_f = (float)f->desc.lo_val;
    sg.norm.scale_f = (float)f->desc.scale;
    if (sg.nb > NA_MAX_BUCKETS) return NNSORT_E_INVALID_ARG;  // m too large for the fixed scratch
    PassPlan pp{};
    int bits = 1;
    while ((1u << bits) < sg.nb) ++bits;
    pp.npass = (bits + RADIX_MAX_BITS - 1) / RADIX_MAX_BITS;
    pp.wlog = wlog;
    for (int p = 0, sh = wlog; p < pp.npass; ++p) {
        const int b = (bits - (sh - wlog) + (pp.npass - p) - 1) / (pp.npass - p);
        pp.shift[p] = sh;
        pp.bits[p] = b;
        sh += b;
    }

    int dev = 0;
    NA_CK(cudaGetDevice(&dev));
    DevState *ds = nullptr;
    int rc = na_setup(dev, &ds);
    if (rc) return rc;
    NaLayout L = na_carve(ds->base);
    const int kb = na_kb(dtype);
    const bool pay = d_payload != nullptr;

    NA_CK(cudaMemcpyAsync(L.seg, &sg, sizeof(Seg), cudaMemcpyHostToDevice, s));
    NA_CK(cudaMemsetAsync(L.stats, 0, sizeof(SegStats), s));
    NA_CK(cudaMemsetAsync(L.err, 0, 16, s));

    PredictArgs pa{};
    pa.segs = L.seg;
    pa.nseg = 1;
    pa.total_tiles = sg.ntiles;
    pa.gs = L.gs[0];
    pa.err = L.err;
    pa.key_bytes = kb;
    pa.dtype = dtype;
    pa.single_model = 1;  // one array whose positions come from its model, as in nnsort_sort
    pa.host_pad = f->hpad.data();
    int sms = 1;
    NA_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    {
        const cudaError_t e = launch_predict(f->pad, o.precision, pa, sms, s);
        if (e == cudaErrorNotSupported) return NNSORT_E_UNSUPPORTED;
        NA_CK(e);
    }
    for (int p = 0; p < pp.npass; ++p) {
        const int si = p & 1, di = si ^ 1;
        PartitionArgs a{};
        a.N = n;
        a.gs_in = L.gs[si];
        a.gs_out = L.gs[di];
        a.key_in = (p == 0) ? d_keys : L.key[si];
        a.key_out = L.key[di];
        if (pay) {
            a.pay_in = (p == 0) ? reinterpret_cast<const uint32_t *>(d_payload) : L.pay[si];
            a.pay_out = L.pay[di];
        }
        a.shift = pp.shift[p];
        a.bits = pp.bits[p];
        a.tile_hist = L.tile_hist;
        a.chunk = L.chunk;
        a.bin_total = L.bin_total;
        a.key_bytes = kb;
        a.dtype = dtype;
        NA_CK(launch_partition(a, s));
    }
    const int fi = pp.npass & 1, oi = fi ^ 1;
    NA_CK(launch_bucket_bounds(L.gs[fi], n, sg.nb, wlog, L.bstart, s));
    SolveArgs sa{};
    sa.segs = L.seg;
    sa.nseg = 1;
    sa.NB = sg.nb;
    sa.wlog = wlog;
    sa.bstart = L.bstart;
    sa.gs = L.gs[fi];
    sa.keys = L.key[fi];
    sa.pay = pay ? L.pay[fi] : nullptr;
    sa.rank = L.rank;
    sa.stats = L.stats;
    sa.bmax = L.bmax;
    sa.carry = L.carry;
    sa.blo = L.blo;
    sa.bhi = L.bhi;
    sa.g_flag = L.flag;
    sa.g_x = L.gx;
    sa.g_y = L.gy;
    sa.N = n;
    sa.key_scratch = L.key[oi];
    sa.pay_scratch = pay ? L.pay[oi] : nullptr;
    sa.err = L.err;
    sa.key_bytes = kb;
    sa.dtype = dtype;
    sa.polish_cap = polish_capacity(kb, pay, false, wlog, 2, &sa.polish_smem);
    sa.ranges = L.ranges;
    sa.max_ranges = sg.nb + 1;
    sa.seam_cnt = L.seam_cnt;
    sa.seam_suf = L.bmax;
    sa.seam_pre = L.bmax + sg.nb;
    sa.seam_cut = reinterpret_cast<unsigned long long *>(L.carry);
    NA_CK(launch_rounds(sa, s));
    NA_CK(launch_finalize(sa, s));
    NA_CK(launch_polish(sa, s));
    NA_CK(launch_seam_repair(sa, sms, s));

    // results: device statistics and the error word, read into host stack memory
    SegStats d;
    uint32_t err = 0;
    NA_CK(cudaMemcpyAsync(&d, L.stats, sizeof(SegStats), cudaMemcpyDeviceToHost, s));
    NA_CK(cudaMemcpyAsync(&err, L.err, 4, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
    if (st) {
        st->rounds = d.t;
        st->eps = sg.eps;
        st->n = n;
        st->L = sg.L;
        st->tau = sg.tau;
        st->w_size[0] = n;
        for (uint32_t r = 1; r <= d.t; ++r) st->w_size[r] = d.count_ge[r];
        for (uint32_t r = 0; r < d.t; ++r) {
            st->placed[r] = st->w_size[r] - st->w_size[r + 1];
            st->out_of_order[r] = d.ooo[r];
            st->sigma[r] = st->w_size[r] ? (double)st->w_size[r + 1] / (double)st->w_size[r] : 0.0;
            st->e[r] = st->placed[r] ? (double)d.ooo[r] / (double)st->placed[r] : 0.0;
        }
        st->trad_rate = (double)st->w_size[d.t] / (double)n;
        st->buckets = sg.nb;
        st->oversized_buckets = d.oversized;
        st->repaired = d.repaired;
        st->repair_ranges = d.ranges;
        st->partition_passes = (uint32_t)pp.npass;
        st->bucket_log2 = (uint32_t)wlog;
    }
    if (err & ERR_NAN) return NNSORT_E_NAN_KEY;
    if (err & ERR_TIMEOUT) return NNSORT_E_TIMEOUT;
    if (err) return NNSORT_E_INVALID_ARG;
    return NNSORT_OK;
}
