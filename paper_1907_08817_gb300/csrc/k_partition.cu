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
#include <cstddef>
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
    if (blockIdx.x == 0) a.bin_total[tid] = 0;  // summed by k_chunk_prefix, which runs after
}

// per chunk of SC_CHUNK tiles: each tile's histogram becomes its exclusive prefix inside the chunk,
// the chunk's totals go to chunk[c] and are added to the digit totals
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
    if (run) atomicAdd(&a.bin_total[d], run);
}

// chunk totals -> chunk bases, the digit's base (elements of all smaller digits) plus the sum over
// earlier chunks, in place. Block b takes digits [32 b, 32 b + 32); its 32 warps take consecutive
// groups of chunks (lane = digit, so every load and store of a warp is one 128-byte line)
__global__ void __launch_bounds__(1024) k_chunk_base(PartitionArgs a, uint32_t chunks) {
    __shared__ uint32_t part[32][33];
    __shared__ uint32_t dbase[RADIX_BINS];
    __shared__ uint32_t scratch[33];
    {   // digit bases: exclusive scan of the digit totals (every block scans all of them)
        const uint32_t v = threadIdx.x < RADIX_BINS ? a.bin_total[threadIdx.x] : 0u;
        const uint32_t ex = block_excl_sum(v, scratch, nullptr);
        if (threadIdx.x < RADIX_BINS) dbase[threadIdx.x] = ex;
        __syncthreads();
    }
    const int i = threadIdx.x & 31, j = threadIdx.x >> 5;
    const uint32_t d = blockIdx.x * 32 + i;
    const uint32_t G = (chunks + 31) / 32;
    const uint32_t c0 = min(chunks, (uint32_t)j * G), c1 = min(chunks, c0 + G);
    uint32_t sum = 0;
    for (uint32_t c = c0; c < c1; ++c) sum += a.chunk[(size_t)c * RADIX_BINS + d];
    part[j][i] = sum;
    __syncthreads();
    if (j == 0) {
        uint32_t run = dbase[d];
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
    alignas(16) unsigned char buf[1];  // reorder buffer: every carried array, SC_TILE entries each
};
constexpr size_t sc_buf_offset() { return offsetof(ScSmem, buf); }

// stable rank of one item per lane inside the warp's counters: the lanes holding the same digit
// come from one ballot per digit bit (BITS > 0: a compile-time count; 0: a.bits at run time)
template <int BITS, bool FULL>
__device__ __forceinline__ uint32_t sc_peers(uint32_t d, bool valid, int bits) {
    unsigned peers = 0xFFFFFFFFu;
    if constexpr (!FULL) {
        // the invalid lanes of a partial tile are told apart by one more ballot
        peers = __ballot_sync(0xFFFFFFFFu, valid);
        if (!valid) peers = ~peers;
    }
    if constexpr (BITS > 0) {
#pragma unroll
        for (int b = 0; b < BITS; ++b) {
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bal : ~bal;
        }
    } else {
        for (int b = 0; b < bits; ++b) {
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bal : ~bal;
        }
    }
    return peers;
}
}  // namespace

// per tile: stable rank of every element by digit, then the scatter to its global position through
// a shared-memory reorder buffer that holds every carried array, so each element's digit and
// offset are read once and each digit's run leaves as coalesced stores
template <typename W, bool KEYDIG, bool PAY, bool ROW, int BITS, bool FULL>
__device__ __forceinline__ void sc_tile(const PartitionArgs &a, ScSmem &S, uint32_t *lstart, uint32_t *gofs,
                                        uint32_t *scratch, uint32_t tile, uint32_t cnt_tile) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t mask = (1u << (BITS > 0 ? BITS : a.bits)) - 1u;
    const uint64_t base = (uint64_t)tile * SC_TILE;
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
        if (FULL || loc < cnt_tile) {
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
        const bool valid = FULL || loc < cnt_tile;
        uint32_t d = 0;
        if (valid) d = sc_digit<W, KEYDIG>(a, key[r], KEYDIG ? 0u : gsv[r], mask);
        dig[r] = (uint16_t)d;
        const unsigned peers = sc_peers<BITS, FULL>(d, valid, a.bits);
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
#pragma unroll
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
    W *bk = reinterpret_cast<W *>(S.buf);
    uint32_t *bg = reinterpret_cast<uint32_t *>(bk + SC_TILE);
    uint32_t *bp = bg + (KEYDIG ? 0 : SC_TILE);
    uint32_t *br = bp + (PAY ? SC_TILE : 0);
#pragma unroll
    for (int r = 0; r < SC_ITEMS; ++r) {
        const uint32_t loc = (uint32_t)w * (32 * SC_ITEMS) + r * 32 + lane;
        if (FULL || loc < cnt_tile) {
            const uint32_t d = dig[r];
            const uint32_t lp = lstart[d] + S.cnt[w][d] + wr[r];
            S.dsort[lp] = (uint16_t)d;
            bk[lp] = key[r];
            if constexpr (!KEYDIG) bg[lp] = gsv[r];
            if constexpr (PAY) bp[lp] = pay[r];
            if constexpr (ROW) br[lp] = row[r];
        }
    }
    __syncthreads();
    W *ko = reinterpret_cast<W *>(a.key_out);
#pragma unroll 4
    for (uint32_t i = tid; i < (FULL ? (uint32_t)SC_TILE : cnt_tile); i += SC_THREADS) {
        const size_t o = (uint32_t)(gofs[S.dsort[i]] + i);
        ko[o] = bk[i];
        if constexpr (!KEYDIG) a.gs_out[o] = bg[i];
        if constexpr (PAY) a.pay_out[o] = bp[i];
        if constexpr (ROW) a.row_out[o] = br[i];
    }
}

template <typename W, bool KEYDIG, bool PAY, bool ROW, int BITS, int MINB>
__global__ void __launch_bounds__(SC_THREADS, MINB) k_scatter(PartitionArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    ScSmem &S = *reinterpret_cast<ScSmem *>(smraw);
    __shared__ uint32_t lstart[RADIX_BINS];
    __shared__ uint32_t gofs[RADIX_BINS];
    __shared__ uint32_t scratch[33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = lane; i < RADIX_BINS; i += 32) S.cnt[w][i] = 0;
    const uint32_t tile = blockIdx.x;
    const uint32_t cnt_tile = (uint32_t)min((uint64_t)SC_TILE, a.N - (uint64_t)tile * SC_TILE);
    if (cnt_tile == SC_TILE)
        sc_tile<W, KEYDIG, PAY, ROW, BITS, true>(a, S, lstart, gofs, scratch, tile, cnt_tile);
    else
        sc_tile<W, KEYDIG, PAY, ROW, BITS, false>(a, S, lstart, gofs, scratch, tile, cnt_tile);
}

template <typename W, bool KD, bool P, bool R, int MB>
static cudaError_t sc_launch(const PartitionArgs &a, uint64_t tiles, cudaStream_t s) {
    const size_t smem = sc_buf_offset() +
                        (size_t)SC_TILE * (sizeof(W) + (KD ? 0 : 4) + (P ? 4 : 0) + (R ? 4 : 0));
    auto go = [&](auto kfn) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kfn<<<(unsigned)tiles, SC_THREADS, smem, s>>>(a);
        return nns_launched(cudaGetLastError());
    };
    // the ballot loop unrolled for the digit widths the passes use (9 and 8 bits); others at run time
    if (a.bits == 9) return go(k_scatter<W, KD, P, R, 9, MB>);
    if (a.bits == 8) return go(k_scatter<W, KD, P, R, 8, MB>);
    return go(k_scatter<W, KD, P, R, 0, MB>);
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
    const bool pay = a.pay_in != nullptr, row = a.row_in != nullptr;
    // two resident blocks per SM where the element's registers allow it (4-byte keys)
    constexpr int MB = sizeof(W) == 4 ? 2 : 1;
    if (pay && row) return sc_launch<W, KD, true, true, 1>(a, tiles, s);
    if (pay) return sc_launch<W, KD, true, false, MB>(a, tiles, s);
    if (row) return sc_launch<W, KD, false, true, MB>(a, tiles, s);
    return sc_launch<W, KD, false, false, MB>(a, tiles, s);
}

cudaError_t launch_partition(const PartitionArgs &a, cudaStream_t s) {
    if (a.N == 0) return cudaSuccess;
    if (a.key_bytes == 4)
        return a.key_digits ? sc_go<uint32_t, true>(a, s) : sc_go<uint32_t, false>(a, s);
    return a.key_digits ? sc_go<uint64_t, true>(a, s) : sc_go<uint64_t, false>(a, s);
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
