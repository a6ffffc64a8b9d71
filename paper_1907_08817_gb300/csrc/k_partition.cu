// k_partition.cu -- stable digit partition of the element space (one pass per digit, LSD order),
// used two ways:
//   * by the bucket index of each element's predicted position, so that every on-chip bucket of
//     positions ends up contiguous and in input order (which keeps the paper's first-arrival rule
//     and the conflict arrays' arrival order intact inside a bucket), and
//   * by the key's order image, as the radix sort behind the training sample (Sec. "Training").
//
// One pass reads and writes each element once. A tile ranks its elements per digit stably (a warp
// finds the lanes holding the same digit from one ballot per digit bit, then counts them with popc),
// publishes its per-digit counts, and learns its global offsets by decoupled look-back over earlier
// tiles, eight at a time (tiles are numbered by an atomic ticket, so every tile waited on has already
// started). Writes go out through a shared-memory reorder buffer in digit order, so each digit's
// run leaves as coalesced stores.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace nns {
static inline cudaError_t nns_launched(cudaError_t e, int k = 1) {
    if (e == cudaSuccess) note_launch(k);
    return e;
}
}  // namespace nns

namespace nns {

namespace {
constexpr int NW = PART_THREADS / 32;
constexpr unsigned long long FLAG_AGG = 1ull, FLAG_INCL = 2ull;
constexpr unsigned long long VAL_MASK = (1ull << 46) - 1ull;

__device__ __forceinline__ unsigned long long lb_pack(uint32_t epoch, unsigned long long flag,
                                                      unsigned long long v) {
    return ((unsigned long long)(epoch & 0xFFFFu) << 48) | (flag << 46) | (v & VAL_MASK);
}

struct PartSmem {
    uint16_t cnt[NW][RADIX_BINS];
    uint16_t dsort[PART_TILE];
    alignas(16) unsigned char buf[PART_TILE * 8];
};
}  // namespace

template <typename W, bool KEYDIG, bool PAY, bool ROW>
__global__ void __launch_bounds__(PART_THREADS, 1) k_onesweep(OnesweepArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    PartSmem &S = *reinterpret_cast<PartSmem *>(smraw);
    __shared__ uint32_t lstart[RADIX_BINS];
    __shared__ uint32_t gofs[RADIX_BINS];
    __shared__ uint32_t scratch[33];
    __shared__ uint32_t sh_tile;

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t nbins = 1u << a.bits;
    const uint32_t mask = nbins - 1u;
    if (tid == 0) sh_tile = atomicAdd(a.ticket, 1u);
    for (int i = lane; i < RADIX_BINS; i += 32) S.cnt[w][i] = 0;
    __syncthreads();
    const uint32_t tile = sh_tile;
    const uint64_t base = (uint64_t)tile * PART_TILE;
    if (base >= a.N) return;  // more blocks than tiles (never launched that way)
    const uint32_t cnt_tile = (uint32_t)std::min<uint64_t>(PART_TILE, a.N - base);

    uint32_t gsv[PART_ITEMS], pay[PART_ITEMS], row[PART_ITEMS];
    W key[PART_ITEMS];
    uint16_t dig[PART_ITEMS];
    uint16_t wr[PART_ITEMS];
    const W *kin = reinterpret_cast<const W *>(a.key_in);
    const unsigned lt = (1u << lane) - 1u;
    // all of the tile's loads first, so they are in flight together
#pragma unroll
    for (int r = 0; r < PART_ITEMS; ++r) {
        const uint32_t loc = (uint32_t)w * (32 * PART_ITEMS) + r * 32 + lane;
        const uint64_t e = base + loc;
        if (loc < cnt_tile) {
            key[r] = kin[e];
            if constexpr (!KEYDIG) gsv[r] = a.gs_in[e];
            if constexpr (PAY) pay[r] = a.pay_in[e];
            if constexpr (ROW) row[r] = a.row_in[e];
        }
    }
#pragma unroll
    for (int r = 0; r < PART_ITEMS; ++r) {
        const uint32_t loc = (uint32_t)w * (32 * PART_ITEMS) + r * 32 + lane;
        const bool valid = loc < cnt_tile;
        uint32_t d = 0xFFFFu;
        if (valid) {
            if constexpr (KEYDIG)
                d = (uint32_t)(ordbits(word64(key[r]), a.dtype) >> a.shift) & mask;
            else
                d = (gsv[r] >> a.shift) & mask;
        }
        dig[r] = (uint16_t)d;
        // lanes with the same digit: one ballot per digit bit (cheaper than a match on this part;
        // in a partial tile the invalid lanes are told apart by one more ballot)
        unsigned peers = 0xFFFFFFFFu;
        if (cnt_tile != PART_TILE) {
            peers = __ballot_sync(0xFFFFFFFFu, valid);
            if (!valid) peers = ~peers;
        }
        for (int b = 0; b < a.bits; ++b) {
            const bool bit = (d >> b) & 1u;
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, bit);
            peers &= bit ? bal : ~bal;
        }
        uint32_t c = 0;
        if (valid) c = S.cnt[w][d];
        __syncwarp();
        if (valid) {
            wr[r] = (uint16_t)(c + __popc(peers & lt));
            if ((peers & lt) == 0) S.cnt[w][d] = (uint16_t)(c + __popc(peers));
        }
        __syncwarp();
    }
    __syncthreads();
    // per-digit tile totals and warp-exclusive prefixes
    uint32_t total = 0;
    {
        const int d = tid;  // PART_THREADS == RADIX_BINS
        for (int ww = 0; ww < NW; ++ww) {
            const uint32_t c = S.cnt[ww][d];
            S.cnt[ww][d] = (uint16_t)total;
            total += c;
        }
    }
    const uint32_t ls = block_excl_sum(total, scratch, nullptr);
    lstart[tid] = ls;
    // decoupled look-back for digit tid
    if ((uint32_t)tid < nbins) {
        unsigned long long *lb = a.lookback + (size_t)tile * RADIX_BINS + tid;
        unsigned long long excl = 0;
        if (tile == 0) {
            st_release_u64(lb, lb_pack(a.epoch, FLAG_INCL, total));
        } else {
            st_release_u64(lb, lb_pack(a.epoch, FLAG_AGG, total));
            // eight predecessors per round trip: their words are read together (each word carries
            // its own flag and value, so no ordering between them is needed), then taken in order
            // until an inclusive prefix ends the walk or a tile that has not published stops it
            constexpr int LBW = 8;
            long long p = (long long)tile - 1;
            unsigned long long t0 = 0;
            uint32_t polls = 0;
            bool done = false;
            while (!done) {
                unsigned long long v[LBW];
#pragma unroll
                for (int q = 0; q < LBW; ++q)
                    v[q] = (p - q >= 0) ? ld_relaxed_u64(a.lookback + (size_t)(p - q) * RADIX_BINS + tid)
                                        : 0ull;
                int used = 0;
#pragma unroll
                for (int q = 0; q < LBW; ++q) {
                    if (used != q || p - q < 0) break;
                    const unsigned long long flag = (v[q] >> 46) & 3ull;
                    if ((uint32_t)(v[q] >> 48) != (a.epoch & 0xFFFFu) || flag == 0) break;
                    excl += v[q] & VAL_MASK;
                    used = q + 1;
                    if (flag == FLAG_INCL) { done = true; break; }
                }
                p -= used;
                if (done || p < 0) break;  // tile 0 publishes an inclusive prefix: p < 0 is not reached
                if (used) continue;
                const unsigned long long now = globaltimer_ns();
                if (t0 == 0) t0 = now;
                else if (now - t0 > SPIN_LIMIT_NS || ++polls > SPIN_LIMIT_POLLS) {
                    atomicOr(a.err, ERR_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
            st_release_u64(lb, lb_pack(a.epoch, FLAG_INCL, excl + total));
        }
        gofs[tid] = a.digit_base[tid] + (uint32_t)excl - ls;
    }
    __syncthreads();
    // local positions
    uint16_t lpos[PART_ITEMS];
#pragma unroll
    for (int r = 0; r < PART_ITEMS; ++r) {
        const uint32_t loc = (uint32_t)w * (32 * PART_ITEMS) + r * 32 + lane;
        if (loc < cnt_tile) {
            const uint32_t d = dig[r];
            lpos[r] = (uint16_t)(lstart[d] + S.cnt[w][d] + wr[r]);
            S.dsort[lpos[r]] = (uint16_t)d;
        }
    }
    // move each array through the reorder buffer
    auto emit = [&](auto *vals, auto *out) {
        using T = typename std::remove_pointer<decltype(out)>::type;
        T *b = reinterpret_cast<T *>(S.buf);
#pragma unroll
        for (int r = 0; r < PART_ITEMS; ++r) {
            const uint32_t loc = (uint32_t)w * (32 * PART_ITEMS) + r * 32 + lane;
            if (loc < cnt_tile) b[lpos[r]] = (T)vals[r];
        }
        __syncthreads();
        for (uint32_t i = tid; i < cnt_tile; i += PART_THREADS) {
            const uint32_t d = S.dsort[i];
            out[(size_t)(uint32_t)(gofs[d] + i)] = b[i];
        }
        __syncthreads();
    };
    __syncthreads();
    emit(key, reinterpret_cast<W *>(a.key_out));
    if constexpr (!KEYDIG) emit(gsv, a.gs_out);
    if constexpr (PAY) emit(pay, a.pay_out);
    if constexpr (ROW) emit(row, a.row_out);
}

template <typename W, bool KD>
static cudaError_t os_go2(const OnesweepArgs &a, cudaStream_t s) {
    const uint64_t tiles = (a.N + PART_TILE - 1) / PART_TILE;
    const size_t smem = sizeof(PartSmem);
    const bool pay = a.pay_in != nullptr, row = a.row_in != nullptr;
#define NNS_OS(P, R)                                                                              \
    {                                                                                             \
        auto kfn = k_onesweep<W, KD, P, R>;                                                       \
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,    \
                                             (int)smem);                                          \
        if (e != cudaSuccess) return e;                                                           \
        kfn<<<(unsigned)tiles, PART_THREADS, smem, s>>>(a);                                       \
        return nns_launched(cudaGetLastError());                                                                \
    }
    if (pay && row) NNS_OS(true, true)
    if (pay) NNS_OS(true, false)
    if (row) NNS_OS(false, true)
    NNS_OS(false, false)
#undef NNS_OS
}

cudaError_t launch_onesweep(const OnesweepArgs &a, cudaStream_t s) {
    if (a.N == 0) return cudaSuccess;
    if (a.key_bytes == 4)
        return a.key_digits ? os_go2<uint32_t, true>(a, s) : os_go2<uint32_t, false>(a, s);
    return a.key_digits ? os_go2<uint64_t, true>(a, s) : os_go2<uint64_t, false>(a, s);
}

// exclusive scan of each pass's histogram (one block per pass)
__global__ void k_digit_bases(const uint32_t *hist, uint32_t *bases) {
    __shared__ uint32_t scratch[33];
    const int p = blockIdx.x;
    const uint32_t v = hist[p * RADIX_BINS + threadIdx.x];
    bases[p * RADIX_BINS + threadIdx.x] = block_excl_sum(v, scratch, nullptr);
}

cudaError_t launch_digit_bases(const uint32_t *hist, uint32_t *bases, int npass, cudaStream_t s) {
    if (npass <= 0) return cudaSuccess;
    k_digit_bases<<<npass, RADIX_BINS, 0, s>>>(hist, bases);
    return nns_launched(cudaGetLastError());
}

// 8-bit key-digit histograms for every pass of a key sort
template <typename W>
__global__ void k_key_hist(const W *keys, uint64_t N, int dtype, int npass, uint32_t *hist) {
    __shared__ uint32_t h[8 * RADIX_BINS];
    for (int i = threadIdx.x; i < npass * RADIX_BINS; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t u = ordbits(word64(keys[i]), dtype);
        for (int p = 0; p < npass; ++p) atomicAdd(&h[p * RADIX_BINS + ((u >> (8 * p)) & 0xFFu)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npass * RADIX_BINS; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

cudaError_t launch_key_hist(const void *keys, uint64_t N, int key_bytes, int dtype, int npass,
                            uint32_t *hist, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    const int grid = (int)std::min<uint64_t>((N + 255) / 256, 1024);
    if (key_bytes == 4)
        k_key_hist<uint32_t><<<grid, 256, 0, s>>>(reinterpret_cast<const uint32_t *>(keys), N, dtype,
                                                  npass, hist);
    else
        k_key_hist<uint64_t><<<grid, 256, 0, s>>>(reinterpret_cast<const uint64_t *>(keys), N, dtype,
                                                  npass, hist);
    return nns_launched(cudaGetLastError());
}

// bstart[b] = first element whose global position is >= b * W (binary search; gs is sorted by
// bucket after the partition)
__global__ void k_bucket_bounds(const uint32_t *gs, uint64_t N, uint32_t nb, int wlog, uint32_t *bstart) {
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nb) return;
    uint64_t lo = 0, hi = N;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (((uint64_t)gs[mid] >> wlog) < b) lo = mid + 1; else hi = mid;
    }
    bstart[b] = (uint32_t)lo;
}

cudaError_t launch_bucket_bounds(const uint32_t *gs, uint64_t N, uint32_t nb, int wlog,
                                 uint32_t *bstart, cudaStream_t s) {
    const uint32_t th = 256, grid = (nb + 1 + th - 1) / th;
    k_bucket_bounds<<<grid, th, 0, s>>>(gs, N, nb, wlog, bstart);
    return nns_launched(cudaGetLastError());
}

}  // namespace nns
