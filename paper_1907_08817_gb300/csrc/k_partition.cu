// k_partition.cu -- stable digit partition of the element space (one pass per digit, LSD order),
// used two ways:
//   * by the bucket index of each element's predicted position, so that every on-chip bucket of
//     positions ends up contiguous and in input order (which keeps the paper's first-arrival rule
//     and the conflict arrays' arrival order intact inside a bucket), and
//   * by the key's order image, as the radix sort behind the training sample (Sec. "Training"),
//     the multi-block sorts of oversized buckets and long repairs, and the "no model" reference.
//
// One pass reads and writes each element once, in tiles of 4,096. Its offsets come from a scan
// over per-tile digit histograms (reduce, then scan, then scatter), so no block ever waits on
// another and two blocks share each SM. A tile ranks its elements per digit stably (a warp finds the
// lanes holding the same digit from one ballot per digit bit, then counts them with popc); writes
// go out through a shared-memory reorder buffer in digit order, so each digit's run leaves as
// coalesced stores.
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

// ---------------------------------------------------------------------------------------------
// The partition pass without look-back. The tiles' global offsets come from a scan over tile
// histograms instead of from waits on earlier tiles, so every block is independent: two blocks run
// on each SM and one block's loads overlap the other's ranking and stores.
namespace {
constexpr int SC_NW = SC_THREADS / 32;

template <typename W, bool KEYDIG>
__device__ __forceinline__ uint32_t sc_digit(const PartitionArgs &a, W key, uint32_t gs, uint32_t mask) {
    if constexpr (KEYDIG) return (uint32_t)(ordbits(word64(key), a.dtype) >> a.shift) & mask;
    else return (gs >> a.shift) & mask;
}
}  // namespace

// per tile: the digit histogram (per-warp counters, so that equal digits contend within a warp only)
template <typename W, bool KEYDIG>
__global__ void __launch_bounds__(SC_THREADS) k_tile_hist(PartitionArgs a) {
    __shared__ uint32_t h[SC_NW][RADIX_BINS];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = lane; i < RADIX_BINS; i += 32) h[w][i] = 0;
    __syncwarp();
    const uint64_t base = (uint64_t)blockIdx.x * SC_TILE;
    const uint32_t cnt = (uint32_t)min((uint64_t)SC_TILE, a.N - base);
    const uint32_t mask = (1u << a.bits) - 1u;
    const W *kin = reinterpret_cast<const W *>(a.key_in);
    uint32_t d[SC_ITEMS];
#pragma unroll
    for (int r = 0; r < SC_ITEMS; ++r) {
        const uint32_t loc = (uint32_t)w * (32 * SC_ITEMS) + r * 32 + lane;
        d[r] = 0xFFFFFFFFu;
        if (loc < cnt) {
            if constexpr (KEYDIG) d[r] = sc_digit<W, true>(a, kin[base + loc], 0u, mask);
            else d[r] = sc_digit<W, false>(a, W(0), a.gs_in[base + loc], mask);
        }
    }
#pragma unroll
    for (int r = 0; r < SC_ITEMS; ++r)
        if (d[r] != 0xFFFFFFFFu) atomicAdd(&h[w][d[r]], 1u);
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (int ww = 0; ww < SC_NW; ++ww) t += h[ww][tid];  // SC_THREADS == RADIX_BINS
    a.tile_hist[(size_t)blockIdx.x * RADIX_BINS + tid] = (uint16_t)t;
}

// per chunk of SC_CHUNK tiles: each tile's histogram becomes its exclusive prefix inside the chunk,
// and the chunk's totals go to chunk[c]
__global__ void __launch_bounds__(RADIX_BINS) k_chunk_prefix(PartitionArgs a, uint32_t tiles) {
    const uint32_t c = blockIdx.x, d = threadIdx.x;
    const uint32_t t0 = c * SC_CHUNK;
    uint16_t v[SC_CHUNK];
#pragma unroll
    for (int j = 0; j < SC_CHUNK; ++j)
        v[j] = (t0 + j < tiles) ? a.tile_hist[(size_t)(t0 + j) * RADIX_BINS + d] : (uint16_t)0;
    uint32_t run = 0;
#pragma unroll
    for (int j = 0; j < SC_CHUNK; ++j) {
        if (t0 + j < tiles) a.tile_hist[(size_t)(t0 + j) * RADIX_BINS + d] = (uint16_t)run;
        run += v[j];
    }
    a.chunk[(size_t)c * RADIX_BINS + d] = run;
}

// chunk totals -> chunk bases, digit_base[d] + the sum over earlier chunks, in place. Block b takes
// digits [32 b, 32 b + 32); its 32 warps take consecutive groups of chunks (lane = digit, so every
// load and store of a warp is one 128-byte line)
__global__ void __launch_bounds__(1024) k_chunk_base(PartitionArgs a, uint32_t chunks) {
    __shared__ uint32_t part[32][33];
    const int i = threadIdx.x & 31, j = threadIdx.x >> 5;
    const uint32_t d = blockIdx.x * 32 + i;
    const uint32_t G = (chunks + 31) / 32;
    const uint32_t c0 = min(chunks, (uint32_t)j * G), c1 = min(chunks, c0 + G);
    uint32_t sum = 0;
    for (uint32_t c = c0; c < c1; ++c) sum += a.chunk[(size_t)c * RADIX_BINS + d];
    part[j][i] = sum;
    __syncthreads();
    if (j == 0) {
        uint32_t run = a.digit_base[d];
        for (int q = 0; q < 32; ++q) {
            const uint32_t x = part[q][i];
            part[q][i] = run;
            run += x;
        }
    }
    __syncthreads();
    uint32_t run = part[j][i];
    for (uint32_t c = c0; c < c1; ++c) {
        const uint32_t x = a.chunk[(size_t)c * RADIX_BINS + d];
        a.chunk[(size_t)c * RADIX_BINS + d] = run;
        run += x;
    }
}

namespace {
struct ScSmem {
    uint16_t cnt[SC_NW][RADIX_BINS];
    uint16_t dsort[SC_TILE];
    alignas(16) unsigned char buf[SC_TILE * 8];
};
}  // namespace

// per tile: stable rank of every element by digit, then the scatter to its global position through
// a shared-memory reorder buffer (each digit's run leaves as coalesced stores)
template <typename W, bool KEYDIG, bool PAY, bool ROW, int MINB>
__global__ void __launch_bounds__(SC_THREADS, MINB) k_scatter(PartitionArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    ScSmem &S = *reinterpret_cast<ScSmem *>(smraw);
    __shared__ uint32_t lstart[RADIX_BINS];
    __shared__ uint32_t gofs[RADIX_BINS];
    __shared__ uint32_t scratch[33];

    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t mask = (1u << a.bits) - 1u;
    for (int i = lane; i < RADIX_BINS; i += 32) S.cnt[w][i] = 0;
    const uint32_t tile = blockIdx.x;
    const uint64_t base = (uint64_t)tile * SC_TILE;
    const uint32_t cnt_tile = (uint32_t)min((uint64_t)SC_TILE, a.N - base);
    // this tile's global digit offsets: chunk base + in-chunk prefix (read early, used late)
    const uint32_t off_in = (uint32_t)a.chunk[(size_t)(tile / SC_CHUNK) * RADIX_BINS + tid] +
                            (uint32_t)a.tile_hist[(size_t)tile * RADIX_BINS + tid];

    uint32_t gsv[SC_ITEMS], pay[SC_ITEMS], row[SC_ITEMS];
    W key[SC_ITEMS];
    uint16_t dig[SC_ITEMS], wr[SC_ITEMS];
    const W *kin = reinterpret_cast<const W *>(a.key_in);
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < SC_ITEMS; ++r) {
        const uint32_t loc = (uint32_t)w * (32 * SC_ITEMS) + r * 32 + lane;
        const uint64_t e = base + loc;
        if (loc < cnt_tile) {
            key[r] = kin[e];
            if constexpr (!KEYDIG) gsv[r] = a.gs_in[e];
            if constexpr (PAY) pay[r] = a.pay_in[e];
            if constexpr (ROW) row[r] = a.row_in[e];
        }
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < SC_ITEMS; ++r) {
        const uint32_t loc = (uint32_t)w * (32 * SC_ITEMS) + r * 32 + lane;
        const bool valid = loc < cnt_tile;
        uint32_t d = 0xFFFFu;
        if (valid) d = sc_digit<W, KEYDIG>(a, key[r], KEYDIG ? 0u : gsv[r], mask);
        dig[r] = (uint16_t)d;
        // lanes holding the same digit: one ballot per digit bit (the invalid lanes of a partial
        // tile are told apart by one more ballot)
        unsigned peers = 0xFFFFFFFFu;
        if (cnt_tile != SC_TILE) {
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
    uint32_t total = 0;
    {
        const int d = tid;  // SC_THREADS == RADIX_BINS
        for (int ww = 0; ww < SC_NW; ++ww) {
            const uint32_t c = S.cnt[ww][d];
            S.cnt[ww][d] = (uint16_t)total;
            total += c;
        }
    }
    const uint32_t ls = block_excl_sum(total, scratch, nullptr);
    lstart[tid] = ls;
    gofs[tid] = off_in - ls;
    __syncthreads();
    uint16_t lpos[SC_ITEMS];
#pragma unroll
    for (int r = 0; r < SC_ITEMS; ++r) {
        const uint32_t loc = (uint32_t)w * (32 * SC_ITEMS) + r * 32 + lane;
        if (loc < cnt_tile) {
            const uint32_t d = dig[r];
            lpos[r] = (uint16_t)(lstart[d] + S.cnt[w][d] + wr[r]);
            S.dsort[lpos[r]] = (uint16_t)d;
        }
    }
    auto emit = [&](auto *vals, auto *out) {
        using T = typename std::remove_pointer<decltype(out)>::type;
        T *b = reinterpret_cast<T *>(S.buf);
#pragma unroll
        for (int r = 0; r < SC_ITEMS; ++r) {
            const uint32_t loc = (uint32_t)w * (32 * SC_ITEMS) + r * 32 + lane;
            if (loc < cnt_tile) b[lpos[r]] = (T)vals[r];
        }
        __syncthreads();
        for (uint32_t i = tid; i < cnt_tile; i += SC_THREADS) {
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
static cudaError_t sc_go(const PartitionArgs &a, cudaStream_t s) {
    const uint64_t tiles = partition_tiles(a.N), chunks = partition_chunks(a.N);
    k_tile_hist<W, KD><<<(unsigned)tiles, SC_THREADS, 0, s>>>(a);
    cudaError_t e = nns_launched(cudaGetLastError());
    if (e != cudaSuccess) return e;
    k_chunk_prefix<<<(unsigned)chunks, RADIX_BINS, 0, s>>>(a, (uint32_t)tiles);
    if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
    k_chunk_base<<<RADIX_BINS / 32, 1024, 0, s>>>(a, (uint32_t)chunks);
    if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
    const size_t smem = sizeof(ScSmem);
    const bool pay = a.pay_in != nullptr, row = a.row_in != nullptr;
#define NNS_SC(P, R, MB)                                                                          \
    {                                                                                             \
        auto kfn = k_scatter<W, KD, P, R, MB>;                                                    \
        e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);    \
        if (e != cudaSuccess) return e;                                                           \
        kfn<<<(unsigned)tiles, SC_THREADS, smem, s>>>(a);                                         \
        return nns_launched(cudaGetLastError());                                                  \
    }
    // two resident blocks per SM where the element's registers allow it (4-byte keys)
    constexpr int MB = sizeof(W) == 4 ? 2 : 1;
    if (pay && row) NNS_SC(true, true, 1)
    if (pay) NNS_SC(true, false, MB)
    if (row) NNS_SC(false, true, MB)
    NNS_SC(false, false, MB)
#undef NNS_SC
}

cudaError_t launch_partition(const PartitionArgs &a, cudaStream_t s) {
    if (a.N == 0) return cudaSuccess;
    if (a.key_bytes == 4)
        return a.key_digits ? sc_go<uint32_t, true>(a, s) : sc_go<uint32_t, false>(a, s);
    return a.key_digits ? sc_go<uint64_t, true>(a, s) : sc_go<uint64_t, false>(a, s);
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
