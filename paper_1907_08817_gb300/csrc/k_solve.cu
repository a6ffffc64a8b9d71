// k_solve.cu -- the Sorting and Polish phases of NN-sort on buckets of positions.
//
// After the partition, the elements whose positions fall into bucket b (positions
// [b W, (b+1) W) of one array) are contiguous and in input order. Because every element keeps
// its position in every iteration (same f, same scale), the paper's iterations decompose over
// buckets exactly:
//   k_rounds   -- the iteration loop of Fig. "Algorithm NN-sort" inside one bucket: each iteration clears
//                 o_i, lets every still-unplaced element claim its position (the first to arrive,
//                 i.e. the lowest input row, wins -- "only the first element is stored"), and sends
//                 the others on to the next conflict array. Output: the iteration in which each
//                 element was stored (or eps if never), |w_i| contributions, and per-iteration
//                 maxima of the stored elements for the polish's carry across buckets.
//   k_finalize -- the loop condition "i < eps and count(w) > tau" over the array's totals
//                 gives t; exclusive prefix maxima of the per-bucket maxima give the carries.
//   k_polish   -- Fig. "Algorithm polish" inside one bucket: o_i's stored elements in position
//                 order; an element smaller than the largest earlier element of o_i (carry from
//                 earlier buckets included) is out of order and joins the leftover, the rest form
//                 a sorted run R_i (this gives the out-of-order counts and fates). The result of
//                 sorting the leftover and merging it with R_1..R_t is the bucket's elements in
//                 (key, row) order, so the bucket is sorted whole (a counting pass over bins of
//                 its key range, or a stable radix sort by key where bins crowd).
//   k_seam     -- the buckets' outputs are each sorted; where a non-monotone f lets a later
//                 bucket hold a key smaller than an earlier bucket's, the affected range is
//                 located and re-sorted (the polish Remark: out-of-order elements end up at their
//                 correct positions whatever the model's errors).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace nns {
static inline cudaError_t nns_launched(cudaError_t e, int k = 1) {
    if (e == cudaSuccess) note_launch(k);
    return e;
}
}  // namespace nns

namespace nns {

constexpr int SOLVE_THREADS = 512;
constexpr int SNW = SOLVE_THREADS / 32;
constexpr int SCAN_THREADS = 1024;  // one block per array for the scans over its buckets

__device__ __forceinline__ int seg_of_bucket(const Seg *segs, int nseg, uint32_t b) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].bbase <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename W> __device__ __forceinline__ W ldk(const void *p, size_t i) {
    return reinterpret_cast<const W *>(p)[i];
}

__device__ __forceinline__ KMax kmax_none() { KMax r; r.k = 0; r.tb = 0; r.valid = 0; return r; }
// maximum over the 32 lanes of a warp (every lane gets it)
__device__ __forceinline__ KMax warp_max_kmax(KMax v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        KMax y;
        y.k = __shfl_xor_sync(0xFFFFFFFFu, v.k, o);
        y.tb = __shfl_xor_sync(0xFFFFFFFFu, v.tb, o);
        y.valid = __shfl_xor_sync(0xFFFFFFFFu, v.valid, o);
        v = kmax(v, y);
    }
    return v;
}

// ---------------------------------------------------------------------------------------------
// Bucket order for the per-bucket kernels: blocks are dispatched roughly in index order, so heavy
// buckets listed first start first and run alongside the many light ones instead of forming a
// tail. Heavy buckets fill order[] from the front, light ones from the back.
__global__ void k_bucket_order(SolveArgs a, uint32_t heavy, uint32_t *order, uint32_t *cnt) {
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.NB) return;
    const uint32_t nbk = a.bstart[b + 1] - a.bstart[b];
    if (nbk > heavy) order[atomicAdd(&cnt[0], 1u)] = b;
    else order[a.NB - 1 - atomicAdd(&cnt[1], 1u)] = b;
    if (a.giant && nbk > POLISH_BIG) {
        BigRange r;
        r.lo = a.bstart[b]; r.hi = a.bstart[b + 1];
        r.seg = (uint32_t)seg_of_bucket(a.segs, a.nseg, b); r.off = 0; r.b = b; r.pad = 0;
        a.giant[atomicAdd(a.giant_cnt, 1u)] = r;
    }
}

cudaError_t launch_bucket_order(const SolveArgs &a, uint32_t heavy, uint32_t *order, uint32_t *cnt,
                                cudaStream_t s) {
    if (a.NB == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(cnt, 0, 2 * sizeof(uint32_t), s);
    if (e == cudaSuccess && a.giant_cnt) e = cudaMemsetAsync(a.giant_cnt, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    k_bucket_order<<<(a.NB + 255) / 256, 256, 0, s>>>(a, heavy, order, cnt);
    return nns_launched(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// Rounds of buckets above POLISH_BIG elements, spread over the whole GPU: the same first-arrival
// rule with the claims in a global table per bucket. A claim in round r stores (MAXR - r) << 32 | i,
// so one atomicMin both picks the lowest row among round-r claimants and overrides the entries of
// earlier rounds; the table is cleared once. Every kernel walks the listed buckets in turn, each
// bucket's elements spread over all threads (consecutive elements on consecutive lanes).
template <typename Fn>
__device__ __forceinline__ void giant_walk(const GiantRounds &g, Fn fn) {
    const uint32_t nb = *g.count;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t j = 0; j < nb; ++j) {
        const BigRange r = g.list[j];
        const uint64_t len = r.hi - r.lo;
        // a uniform trip count per warp, so that warp-wide intrinsics see all lanes
        for (uint64_t base = t0 & ~31ull; base < len; base += stride) fn(j, r, base + (t0 & 31), len);
    }
}

__global__ void k_giant_init(SolveArgs a, GiantRounds g) {
    const uint32_t nb = *g.count;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t Wn = 1ull << a.wlog;
    for (uint64_t q = t0; q < (uint64_t)nb * Wn; q += stride) g.table[q] = ~0ull;
    for (uint64_t q = t0; q < (uint64_t)nb * MAXR; q += stride) { g.cnt[q] = 0; g.kmax[q] = 0; g.tbmax[q] = 0; }
    giant_walk(g, [&](uint32_t, const BigRange &r, uint64_t i, uint64_t len) {
        if (i < len) a.rank[r.lo + i] = 0;
    });
}

__global__ void k_giant_claim(SolveArgs a, GiantRounds g, int r) {
    const uint32_t wm = (1u << a.wlog) - 1u;
    const unsigned lanes_below = (1u << (threadIdx.x & 31)) - 1u;
    const unsigned long long tag = (unsigned long long)(MAXR - r) << 32;
    giant_walk(g, [&](uint32_t j, const BigRange &rg, uint64_t i, uint64_t len) {
        const bool act = i < len && a.rank[rg.lo + i] == r;
        const uint32_t p = act ? (a.gs[rg.lo + i] & wm) : EMPTY32;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, p);
        if (act && (peers & lanes_below) == 0)
            atomicMin(&g.table[((uint64_t)j << a.wlog) + p], tag | (unsigned long long)i);
    });
}

__global__ void k_giant_check(SolveArgs a, GiantRounds g, int r) {
    const uint32_t wm = (1u << a.wlog) - 1u;
    const unsigned long long tag = (unsigned long long)(MAXR - r) << 32;
    giant_walk(g, [&](uint32_t j, const BigRange &rg, uint64_t i, uint64_t len) {
        if (i < len && a.rank[rg.lo + i] == r) {
            const uint32_t p = a.gs[rg.lo + i] & wm;
            if (g.table[((uint64_t)j << a.wlog) + p] != (tag | (unsigned long long)i))
                a.rank[rg.lo + i] = (uint8_t)(r + 1);
        }
    });
}

// per (bucket, round): how many elements were stored and the largest order image among them
template <typename W>
__global__ void k_giant_stats(SolveArgs a, GiantRounds g, int eps) {
    giant_walk(g, [&](uint32_t j, const BigRange &rg, uint64_t i, uint64_t len) {
        if (i >= len) return;
        const int c = a.rank[rg.lo + i];
        if (c >= eps) return;
        const unsigned long long k = ordbits(word64(ldk<W>(a.keys, rg.lo + i)), a.dtype);
        atomicAdd(&g.cnt[j * MAXR + c], 1u);
        atomicMax(&g.kmax[j * MAXR + c], k);
    });
}

// the largest tie-break among the stored elements with that order image
template <typename W>
__global__ void k_giant_stats2(SolveArgs a, GiantRounds g, int eps) {
    giant_walk(g, [&](uint32_t j, const BigRange &rg, uint64_t i, uint64_t len) {
        if (i >= len) return;
        const int c = a.rank[rg.lo + i];
        if (c >= eps) return;
        const unsigned long long k = ordbits(word64(ldk<W>(a.keys, rg.lo + i)), a.dtype);
        if (k == g.kmax[j * MAXR + c])
            atomicMax(&g.tbmax[j * MAXR + c], a.rows ? a.rows[rg.lo + i] : (uint32_t)i);
    });
}

__global__ void k_giant_fin(SolveArgs a, GiantRounds g, int eps) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= *g.count) return;
    const BigRange rg = g.list[j];
    unsigned long long ge = rg.hi - rg.lo;
    for (int r = 0; r < eps; ++r) {
        const unsigned int c = g.cnt[j * MAXR + r];
        ge -= c;
        if (ge) atomicAdd(&a.stats[rg.seg].count_ge[r + 1], ge);
        OKey o;
        o.k = c ? g.kmax[j * MAXR + r] : 0ull;
        o.tb = c ? g.tbmax[j * MAXR + r] : 0u;
        o.valid = c ? 1u : 0u;
        a.bmax[(size_t)rg.b * MAXR + r] = o;
    }
}

cudaError_t launch_giant_rounds(const SolveArgs &a, const GiantRounds &g, int eps, int sms, cudaStream_t s) {
    const unsigned grid = (unsigned)sms * 4, th = 256;
    cudaError_t e;
    k_giant_init<<<grid, th, 0, s>>>(a, g);
    if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
    for (int r = 0; r < eps; ++r) {
        k_giant_claim<<<grid, th, 0, s>>>(a, g, r);
        if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
        k_giant_check<<<grid, th, 0, s>>>(a, g, r);
        if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
    }
    if (a.key_bytes == 4) {
        k_giant_stats<uint32_t><<<grid, th, 0, s>>>(a, g, eps);
        if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
        k_giant_stats2<uint32_t><<<grid, th, 0, s>>>(a, g, eps);
    } else {
        k_giant_stats<uint64_t><<<grid, th, 0, s>>>(a, g, eps);
        if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
        k_giant_stats2<uint64_t><<<grid, th, 0, s>>>(a, g, eps);
    }
    if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
    k_giant_fin<<<(g.cap + 127) / 128, 128, 0, s>>>(a, g, eps);
    return nns_launched(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
// k_rounds: one block per bucket. A bucket of up to rounds_cap(wlog) elements keeps its local
// positions and round indices in shared memory next to the position table; larger buckets keep the
// round indices in the global rank array.
constexpr int RT = 256;  // threads of a rounds block
__host__ __device__ constexpr uint32_t rounds_cap(int wlog) {
    return wlog <= 12 ? (2u << wlog) : (1u << wlog);
}
__host__ __device__ constexpr size_t rounds_smem(int wlog) {
    return ((size_t)4 << wlog) + (size_t)3 * rounds_cap(wlog);
}

template <typename W>
__global__ void __launch_bounds__(RT, 4) k_rounds(SolveArgs a) {
    extern __shared__ uint32_t tbl[];  // Wn claims | rcap local positions (u16) | rcap round indices (u8)
    __shared__ KMax ks[RT / 32];
    __shared__ unsigned int red_cnt[RT / 32];
    __shared__ int sh_seg;
    const int tid = threadIdx.x;
    const uint32_t b = a.order ? a.order[blockIdx.x] : blockIdx.x;
    const uint32_t s0 = a.bstart[b], s1 = a.bstart[b + 1];
    const uint32_t nbk = s1 - s0;
    if (nbk == 0) {
        if (tid < MAXR) { OKey z; z.k = 0; z.tb = 0; z.valid = 0; a.bmax[(size_t)b * MAXR + tid] = z; }
        return;
    }
    if (a.giant && nbk > POLISH_BIG) return;  // launch_giant_rounds
    if (tid == 0) sh_seg = seg_of_bucket(a.segs, a.nseg, b);
    __syncthreads();
    const int seg = sh_seg;
    const int eps = (int)a.segs[seg].eps;
    const uint32_t Wn = 1u << a.wlog, wm = Wn - 1u;
    const uint32_t rcap = rounds_cap(a.wlog);
    const int dt = a.dtype;
    const bool onchip = nbk <= rcap;
    uint16_t *pos = reinterpret_cast<uint16_t *>(tbl + Wn);
    uint8_t *cur = onchip ? reinterpret_cast<uint8_t *>(pos + rcap) : a.rank + s0;
    constexpr int LB = 8;  // loads per thread issued together
    for (uint32_t i0 = 0; i0 < nbk; i0 += RT * LB) {
        uint32_t g[LB];
#pragma unroll
        for (int q = 0; q < LB; ++q) {
            const uint32_t i = i0 + q * RT + tid;
            g[q] = (onchip && i < nbk) ? a.gs[s0 + i] : 0u;
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
            const uint32_t i = i0 + q * RT + tid;
            if (i < nbk) {
                if (onchip) pos[i] = (uint16_t)(g[q] & wm);
                cur[i] = 0;
            }
        }
    }
    __syncthreads();
    auto lpos = [&](uint32_t i) -> uint32_t { return onchip ? (uint32_t)pos[i] : (a.gs[s0 + i] & wm); };
    // Algorithm NN-sort: in iteration r every element still unplaced claims its position; the
    // lowest row (first arrival) is stored, the others move on to the next conflict array. The
    // check that moves the others on also counts the stored elements and takes the largest of them
    // (for the polish carry).
    const int lane = tid & 31, wid = tid >> 5;
    unsigned long long ge = nbk;  // elements whose round index is >= r
    int r = 0;
    for (; r < eps; ++r) {
        for (uint32_t j = tid; j < Wn; j += RT) tbl[j] = EMPTY32;
        __syncthreads();
        // every claimant issues a shared-memory atomicMin of its row (the lowest row wins); a warp
        // match to let only the lowest lane of a position claim cost more than the atomics it saved,
        // except where nearly every key shares a few positions. Loads are issued LB at a time (the
        // round index and position may live in global memory).
        for (uint32_t i0 = 0; i0 < nbk; i0 += RT * LB) {
            uint32_t pv[LB];
#pragma unroll
            for (int q = 0; q < LB; ++q) {
                const uint32_t i = i0 + q * RT + tid;
                pv[q] = (i < nbk && cur[i] == r) ? lpos(i) : EMPTY32;
            }
#pragma unroll
            for (int q = 0; q < LB; ++q) {
                const uint32_t i = i0 + q * RT + tid;
                if (pv[q] != EMPTY32) atomicMin(&tbl[pv[q]], i);
            }
        }
        __syncthreads();
        int left = 0;
        unsigned int cnt = 0;
        KMax m = kmax_none();
        for (uint32_t i0 = 0; i0 < nbk; i0 += RT * LB) {
            uint32_t pv[LB];
#pragma unroll
            for (int q = 0; q < LB; ++q) {
                const uint32_t i = i0 + q * RT + tid;
                pv[q] = (i < nbk && cur[i] == r) ? lpos(i) : EMPTY32;
            }
            bool win[LB];
#pragma unroll
            for (int q = 0; q < LB; ++q) {
                const uint32_t i = i0 + q * RT + tid;
                win[q] = false;
                if (pv[q] != EMPTY32) {
                    if (tbl[pv[q]] != i) { cur[i] = (uint8_t)(r + 1); left = 1; }
                    else win[q] = true;
                }
            }
            W kv[LB];
#pragma unroll
            for (int q = 0; q < LB; ++q) kv[q] = win[q] ? ldk<W>(a.keys, s0 + i0 + q * RT + tid) : (W)0;
#pragma unroll
            for (int q = 0; q < LB; ++q) {
                if (!win[q]) continue;
                const uint32_t i = i0 + q * RT + tid;
                KMax x;
                x.k = ordbits(word64(kv[q]), dt);
                x.tb = a.rows ? a.rows[s0 + i] : i;
                x.valid = 1;
                m = kmax(m, x);
                ++cnt;
            }
        }
        cnt = __reduce_add_sync(0xFFFFFFFFu, cnt);
        m = warp_max_kmax(m);
        if (lane == 0) { red_cnt[wid] = cnt; ks[wid] = m; }
        // a barrier as well: red_cnt and ks are complete (they are written again only after the
        // next iteration's barriers)
        const bool more = __syncthreads_or(left) != 0;
        if (tid == 0) {
            unsigned int c = 0;
            KMax t = kmax_none();
            for (int w = 0; w < RT / 32; ++w) { c += red_cnt[w]; t = kmax(t, ks[w]); }
            ge -= c;
            if (ge) atomicAdd(&a.stats[seg].count_ge[r + 1], ge);
            OKey o; o.k = t.k; o.tb = t.tb; o.valid = t.valid;
            a.bmax[(size_t)b * MAXR + r] = o;
        }
        if (!more) { ++r; break; }
    }
    // iterations after the last one that stored anything store nothing
    for (; r < eps; ++r)
        if (tid == 0) { OKey z; z.k = 0; z.tb = 0; z.valid = 0; a.bmax[(size_t)b * MAXR + r] = z; }
    if (onchip)
        for (uint32_t i = tid; i < nbk; i += RT) a.rank[s0 + i] = cur[i];
}

// ---------------------------------------------------------------------------------------------
// k_finalize: one block per array
__global__ void __launch_bounds__(SCAN_THREADS) k_finalize(SolveArgs a) {
    __shared__ KMax scratch[33];
    __shared__ int sh_t;
    const int s = blockIdx.x, tid = threadIdx.x;
    const Seg &sg = a.segs[s];
    SegStats &st = a.stats[s];
    if (tid == 0) {
        uint32_t t = 0;
        unsigned long long w = sg.n;
        while (t < sg.eps && w > sg.tau) {
            ++t;
            w = st.count_ge[t];
        }
        st.count_ge[0] = sg.n;
        st.t = t;
        sh_t = (int)t;
    }
    __syncthreads();
    const int t = sh_t;
    const uint32_t nb = sg.nb, bb = sg.bbase;
    // tiles of PSI * SCAN_THREADS buckets, PSI consecutive ones per thread
    constexpr int PSI = 8;
    constexpr uint32_t PST = SCAN_THREADS * PSI;
    __shared__ KMax tot;
    for (int r = 0; r < t; ++r) {
        KMax carry = kmax_none();  // maximum stored in o_r by the buckets before the tile
        for (uint32_t t0 = 0; t0 < nb; t0 += PST) {
            KMax v[PSI];
            KMax loc = kmax_none();
#pragma unroll
            for (int k = 0; k < PSI; ++k) {
                const uint32_t c = t0 + (uint32_t)tid * PSI + k;
                v[k] = kmax_none();
                if (c < nb) {
                    const OKey o = a.bmax[(size_t)(bb + c) * MAXR + r];
                    v[k].k = o.k; v[k].tb = o.tb; v[k].valid = o.valid;
                }
                loc = kmax(loc, v[k]);
            }
            KMax run = kmax(carry, block_excl_max(loc, scratch, &tot));
#pragma unroll
            for (int k = 0; k < PSI; ++k) {
                const uint32_t c = t0 + (uint32_t)tid * PSI + k;
                if (c < nb) {
                    OKey co; co.k = run.k; co.tb = run.tb; co.valid = run.valid;
                    a.carry[(size_t)(bb + c) * MAXR + r] = co;
                }
                run = kmax(run, v[k]);
            }
            carry = kmax(carry, tot);
        }
    }
}

// One large array: the scans over its buckets (k_finalize's, k_seam_ps's) over tiles of MT_TILE
// buckets on many blocks, in three launches (tile extrema; their exclusive prefix in one block;
// each tile's scan from its prefix). Results equal the one-block scan's (the maximum is
// associative and exact).
constexpr int MT_THREADS = 256, MT_PER = 4;
constexpr uint32_t MT_TILE = MT_THREADS * MT_PER;

__device__ __forceinline__ int rounds_of(const Seg &sg, const SegStats &st) {
    uint32_t t = 0;
    unsigned long long w = sg.n;
    while (t < sg.eps && w > sg.tau) {
        ++t;
        w = st.count_ge[t];
    }
    return (int)t;
}
__device__ __forceinline__ KMax kmax_of(const OKey &o) {
    KMax x; x.k = o.k; x.tb = o.tb; x.valid = o.valid; return x;
}
__device__ __forceinline__ OKey okey_of_kmax(const KMax &x) {
    OKey o; o.k = x.k; o.tb = x.tb; o.valid = x.valid; return o;
}

// 1) tile maxima per round -> agg[tile * MAXR + r]; block 0 also records t
__global__ void __launch_bounds__(MT_THREADS) k_finalize_tiles(SolveArgs a, OKey *agg) {
    __shared__ KMax scratch[33];
    __shared__ KMax tot;
    __shared__ int sh_t;
    const int tid = threadIdx.x;
    const Seg &sg = a.segs[0];
    SegStats &st = a.stats[0];
    if (tid == 0) sh_t = rounds_of(sg, st);
    __syncthreads();
    const int t = sh_t;
    const uint32_t c0 = blockIdx.x * MT_TILE + (uint32_t)tid * MT_PER;
    for (int r = 0; r < t; ++r) {
        KMax loc = kmax_none();
#pragma unroll
        for (int k = 0; k < MT_PER; ++k)
            if (c0 + k < sg.nb) loc = kmax(loc, kmax_of(a.bmax[(size_t)(sg.bbase + c0 + k) * MAXR + r]));
        block_excl_max(loc, scratch, &tot);
        if (tid == 0) agg[(size_t)blockIdx.x * MAXR + r] = okey_of_kmax(tot);
    }
}
// 2) exclusive prefix maxima of the tile maxima (one block; at most MT_THREADS * MT_PER tiles)
__global__ void __launch_bounds__(MT_THREADS) k_finalize_prefix(SolveArgs a, OKey *agg, uint32_t ntiles) {
    __shared__ KMax scratch[33];
    __shared__ int sh_t;
    const int tid = threadIdx.x;
    const Seg &sg = a.segs[0];
    SegStats &st = a.stats[0];
    if (tid == 0) {
        const int t = rounds_of(sg, st);
        st.count_ge[0] = sg.n;
        st.t = (uint32_t)t;
        sh_t = t;
    }
    __syncthreads();
    for (int r = 0; r < sh_t; ++r) {
        KMax v[MT_PER], loc = kmax_none();
#pragma unroll
        for (int k = 0; k < MT_PER; ++k) {
            const uint32_t i = (uint32_t)tid * MT_PER + k;
            v[k] = i < ntiles ? kmax_of(agg[(size_t)i * MAXR + r]) : kmax_none();
            loc = kmax(loc, v[k]);
        }
        KMax run = block_excl_max(loc, scratch, nullptr);
#pragma unroll
        for (int k = 0; k < MT_PER; ++k) {
            const uint32_t i = (uint32_t)tid * MT_PER + k;
            if (i < ntiles) agg[(size_t)i * MAXR + r] = okey_of_kmax(run);
            run = kmax(run, v[k]);
        }
    }
}
// 3) each tile's exclusive prefix maxima from the maximum of the tiles before it
__global__ void __launch_bounds__(MT_THREADS) k_finalize_apply(SolveArgs a, const OKey *agg) {
    __shared__ KMax scratch[33];
    __shared__ int sh_t;
    const int tid = threadIdx.x;
    const Seg &sg = a.segs[0];
    if (tid == 0) sh_t = (int)a.stats[0].t;
    __syncthreads();
    const uint32_t c0 = blockIdx.x * MT_TILE + (uint32_t)tid * MT_PER;
    for (int r = 0; r < sh_t; ++r) {
        KMax v[MT_PER], loc = kmax_none();
#pragma unroll
        for (int k = 0; k < MT_PER; ++k) {
            v[k] = c0 + k < sg.nb ? kmax_of(a.bmax[(size_t)(sg.bbase + c0 + k) * MAXR + r]) : kmax_none();
            loc = kmax(loc, v[k]);
        }
        KMax run = kmax(kmax_of(agg[(size_t)blockIdx.x * MAXR + r]), block_excl_max(loc, scratch, nullptr));
#pragma unroll
        for (int k = 0; k < MT_PER; ++k) {
            if (c0 + k < sg.nb) a.carry[(size_t)(sg.bbase + c0 + k) * MAXR + r] = okey_of_kmax(run);
            run = kmax(run, v[k]);
        }
    }
}

// ---------------------------------------------------------------------------------------------
// CTA-level building blocks on index lists

// Stable LSD radix sort of an index list by a 32- or 64-bit key (kf(x)), 8-bit digits. One sweep
// builds the histograms of every digit; a digit that is constant over the list skips its pass.
// A pass moves the list in tiles of SOLVE_THREADS * SORT_ITEMS elements: warp w ranks its 256
// consecutive elements with match/popc over 8 rounds, the per-(digit, warp) counts become positions
// with the running per-digit base folded in, and each element is written straight to its place.
// Returns the buffer holding the result.
constexpr int SORT_ITEMS = 8;
constexpr uint32_t SORT_TILE = SOLVE_THREADS * SORT_ITEMS;
template <typename Idx, typename KeyFn>
__device__ Idx *cta_radix_sort(Idx *src, Idx *dst, uint32_t cnt, int keybits, KeyFn kf,
                               uint32_t *hist /*[8][256]*/, uint32_t *wcnt /*[SNW][256]*/,
                               uint32_t *scratch /*33*/) {
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int npass = keybits / 8;
    for (int i = tid; i < npass * 256; i += SOLVE_THREADS) hist[i] = 0;
    for (int i = tid; i < SNW * 256; i += SOLVE_THREADS) wcnt[i] = 0;
    __syncthreads();
    for (uint32_t i = tid; i < cnt; i += SOLVE_THREADS) {
        const unsigned long long k = kf(src[i]);
        for (int p = 0; p < npass; ++p) atomicAdd(&hist[p * 256 + (uint32_t)((k >> (8 * p)) & 0xFFu)], 1u);
    }
    __syncthreads();
    if (cnt == 0) return src;
    const unsigned long long kfirst = kf(src[0]);
    for (int p = 0; p < npass; ++p) {
        uint32_t *h = hist + p * 256;
        const int shift = 8 * p;
        if (h[(uint32_t)((kfirst >> shift) & 0xFFu)] == cnt) continue;  // same decision on every thread
        const uint32_t hv = (tid < 256) ? h[tid] : 0u;
        const uint32_t ex = block_excl_sum(hv, scratch, nullptr);
        if (tid < 256) h[tid] = ex;  // running base per digit
        __syncthreads();
        for (uint32_t t0 = 0; t0 < cnt; t0 += SORT_TILE) {
            Idx x[SORT_ITEMS];
            uint32_t d[SORT_ITEMS], wr[SORT_ITEMS];
#pragma unroll
            for (int r = 0; r < SORT_ITEMS; ++r) {
                const uint32_t i = t0 + (uint32_t)w * (32 * SORT_ITEMS) + r * 32 + lane;
                x[r] = (i < cnt) ? src[i] : (Idx)0;
            }
#pragma unroll
            for (int r = 0; r < SORT_ITEMS; ++r) {
                const uint32_t i = t0 + (uint32_t)w * (32 * SORT_ITEMS) + r * 32 + lane;
                d[r] = (i < cnt) ? (uint32_t)((kf(x[r]) >> shift) & 0xFFu) : 0x1FFu;
            }
#pragma unroll
            for (int r = 0; r < SORT_ITEMS; ++r) {
                const bool valid = d[r] < 256u;
                const unsigned peers = __match_any_sync(0xFFFFFFFFu, d[r]);
                uint32_t c = 0;
                if (valid) c = wcnt[w * 256 + d[r]];
                __syncwarp();
                if (valid) {
                    wr[r] = c + __popc(peers & lt);
                    if ((peers & lt) == 0) wcnt[w * 256 + d[r]] = c + __popc(peers);
                }
                __syncwarp();
            }
            __syncthreads();
            if (tid < 256) {
                uint32_t run = h[tid];
                for (int ww = 0; ww < SNW; ++ww) {
                    const uint32_t c = wcnt[ww * 256 + tid];
                    wcnt[ww * 256 + tid] = run;
                    run += c;
                }
                h[tid] = run;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < SORT_ITEMS; ++r)
                if (d[r] < 256u) dst[wcnt[w * 256 + d[r]] + wr[r]] = x[r];
            __syncthreads();
            for (int i = tid; i < SNW * 256; i += SOLVE_THREADS) wcnt[i] = 0;
            __syncthreads();
        }
        Idx *tmp = src; src = dst; dst = tmp;
    }
    return src;
}

// Stable sort of the element indices 0..cnt-1 by a 32- or 64-bit key in one counting pass, for
// lists whose keys spread evenly over their range (a bucket's elements under a fitted model). The
// order is that of the composite key c(i) = (key(i) - kmin) * 2^ib + i (ib = bits of cnt - 1):
// (key, index) order, i.e. a stable sort. Its range is cut into NBIN bins of 2^s consecutive
// values; when the keys span few distinct values (binary32 keys near a density peak repeat
// often) the index's top bits split each value's elements over several bins instead of crowding
// one. Every element drops into its bin (shared-memory atomics, so in arbitrary order inside
// it), and each element's place inside its bin is then the number of the bin's elements before it
// in (key, index) order -- counts that are independent of one another, so all threads rank their
// elements at once. The result is left in `src` (`dst` is scratch), and src is returned; nullptr,
// with neither list touched, when some bin would hold more than BIN_MAX elements (the caller then
// sorts by radix). For 16-bit index lists the caller may pass `pair`, room for one u32 per element,
// and `out16`: when every bin's keys differ in at most their low 16 bits, the scatter stores each
// element as (its key's offset inside the bin) * 2^16 + index -- a word whose integer order is the
// (key, index) order inside the bin -- so the ranking compares words without reading keys, and
// the result is left in out16 (returned) instead of src.
constexpr uint32_t NBIN = 4096;
constexpr int NBIN_LOG = 12;
constexpr uint32_t BIN_MAX = 24;
constexpr uint32_t BIN_SORT_MAX = 6144;  // longest list sorted this way (1.5 elements per bin)
template <typename Idx, typename KeyFn>
__device__ Idx *cta_bin_sort(Idx *src, Idx *dst, uint32_t cnt, KeyFn kf, uint32_t *bins /*[NBIN]*/,
                             unsigned long long *mm /*[2 * SNW]*/, uint32_t *scratch /*33*/,
                             uint32_t *pair = nullptr, uint16_t *out16 = nullptr) {
    static_assert(NBIN % SOLVE_THREADS == 0, "whole bins per thread");
    static_assert(NBIN == (1u << NBIN_LOG), "NBIN is 2^NBIN_LOG");
    constexpr int BPT = NBIN / SOLVE_THREADS;
    using K = decltype(kf((Idx)0));  // the key's own unsigned width
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    K lo = (K)~(K)0, hi = 0;
    for (uint32_t i = tid; i < cnt; i += SOLVE_THREADS) {
        const K k = kf((Idx)i);
        lo = k < lo ? k : lo;
        hi = k > hi ? k : hi;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const K l2 = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
        const K h2 = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
    }
    if (lane == 0) { mm[w] = lo; mm[SNW + w] = hi; }
    for (uint32_t b = tid; b < NBIN; b += SOLVE_THREADS) bins[b] = 0;
    __syncthreads();
    lo = (K)mm[0];
    hi = (K)mm[SNW];
#pragma unroll
    for (int q = 1; q < SNW; ++q) {
        lo = (K)mm[q] < lo ? (K)mm[q] : lo;
        hi = (K)mm[SNW + q] > hi ? (K)mm[SNW + q] : hi;
    }
    // c(i) < 2^(br + ib) with br = bits of (kmax - kmin); bin = c >> sh with sh = max(0, br + ib -
    // NBIN_LOG). With d = sh - ib >= 0 the index bits fall off entirely: bin = (key - kmin) >> d;
    // otherwise bin = ((key - kmin) << -d) | (i >> sh), both below NBIN.
    const K range = hi - lo;
    int br = 0;
    if constexpr (sizeof(K) == 8) br = range ? 64 - __clzll((long long)range) : 0;
    else br = range ? 32 - __clz((int)range) : 0;
    const int ib = cnt > 1 ? 32 - __clz((int)(cnt - 1)) : 0;
    const int sh = br + ib > NBIN_LOG ? br + ib - NBIN_LOG : 0;
    const int d = sh - ib;
    auto bin_of = [&](uint32_t i, K k) -> uint32_t {
        return d >= 0 ? (uint32_t)((K)(k - lo) >> d) : (((uint32_t)(k - lo) << -d) | (i >> sh));
    };
    for (uint32_t i = tid; i < cnt; i += SOLVE_THREADS) atomicAdd(&bins[bin_of(i, kf((Idx)i))], 1u);
    __syncthreads();
    uint32_t tsum = 0, tmax = 0;
#pragma unroll
    for (int q = 0; q < BPT; ++q) {
        const uint32_t c = bins[tid * BPT + q];
        tsum += c;
        tmax = c > tmax ? c : tmax;
    }
    if (__syncthreads_or(tmax > BIN_MAX)) return nullptr;
    uint32_t run = block_excl_sum(tsum, scratch, nullptr);
#pragma unroll
    for (int q = 0; q < BPT; ++q) {  // bins[b] = first slot of bin b
        const uint32_t c = bins[tid * BPT + q];
        bins[tid * BPT + q] = run;
        run += c;
    }
    __syncthreads();
    if constexpr (sizeof(Idx) == 2) {
        if (pair && out16 && d <= 16) {
            // inside bin b the keys share (key - kmin) >> d = b (d >= 0) or are all equal (d < 0).
            // When the offset's bits and the index's fit in 32 - NBIN_LOG, the word also carries
            // the bin: bin * 2^20 + offset * 2^ib + index; otherwise offset * 2^16 + index.
            const int dres = d > 0 ? d : 0;
            const bool full = dres + ib <= 32 - NBIN_LOG;
            const uint32_t rmask = dres ? (1u << dres) - 1u : 0u;
            const uint32_t imask = (1u << ib) - 1u;
            for (uint32_t i = tid; i < cnt; i += SOLVE_THREADS) {
                const K k = kf((Idx)i);
                const uint32_t b = bin_of(i, k);
                const uint32_t res = (uint32_t)(K)(k - lo) & rmask;
                pair[atomicAdd(&bins[b], 1u)] =
                    full ? (b << (32 - NBIN_LOG)) | (res << ib) | i : (res << 16) | i;
            }
            __syncthreads();
            for (uint32_t j = tid; j < cnt; j += SOLVE_THREADS) {
                const uint32_t c = pair[j];
                uint32_t x, b;
                if (full) {
                    x = c & imask;
                    b = c >> (32 - NBIN_LOG);
                } else {
                    x = c & 0xFFFFu;
                    b = bin_of(x, kf((Idx)x));
                }
                const uint32_t st = b ? bins[b - 1] : 0u, e = bins[b];
                uint32_t r = 0;
                for (uint32_t i = st; i < e; ++i) r += pair[i] < c ? 1u : 0u;
                out16[st + r] = (uint16_t)x;
            }
            __syncthreads();
            return reinterpret_cast<Idx *>(out16);
        }
    }
    for (uint32_t i = tid; i < cnt; i += SOLVE_THREADS)
        dst[atomicAdd(&bins[bin_of(i, kf((Idx)i))], 1u)] = (Idx)i;
    __syncthreads();
    // bins[b] is now one past the last slot of bin b; each element's rank inside its bin gives its
    // slot in src
    for (uint32_t j = tid; j < cnt; j += SOLVE_THREADS) {
        const Idx x = dst[j];
        const K kx = kf(x);
        const uint32_t b = bin_of((uint32_t)x, kx);
        const uint32_t st = b ? bins[b - 1] : 0u, e = bins[b];
        uint32_t r = 0;
        if (e - st > 1) {
            for (uint32_t i = st; i < e; ++i) {
                const Idx y = dst[i];
                const K ky = kf(y);
                r += (ky < kx || (ky == kx && y < x)) ? 1u : 0u;
            }
        }
        src[st + r] = x;
    }
    __syncthreads();
    return src;
}

// ---------------------------------------------------------------------------------------------
// k_polish
struct PolishSmem {
    union {
        struct {
            uint32_t hist[8 * 256];
            uint32_t wcnt[SNW * 256];
        };
        uint32_t bins[NBIN];  // cta_bin_sort
    };
    unsigned long long mm[2 * SNW];
    uint32_t scratch[33];
    KMax kscratch[33];
    KMax carry[MAXR];
    unsigned int ooo[MAXR];
    int seg, t;
};

// order image of a key whose type is known at compile time (FL: IEEE float, else unsigned)
// (in the key's own width, so that 32-bit keys are compared and binned in 32-bit arithmetic)
template <typename W, bool FL>
__device__ __forceinline__ W okey_of(W w) {
    if constexpr (!FL) {
        return w;
    } else if constexpr (sizeof(W) == 4) {
        return (w & 0x80000000u) ? (W)~w : (W)(w | 0x80000000u);
    } else {
        return (w >> 63) ? (W)~w : (W)(w | 0x8000000000000000ull);
    }
}

template <typename W, typename Idx, bool FL>
struct BucketView {
    // element accessors (generic pointers: shared memory on chip, global memory otherwise)
    const W *K;        // keys
    const uint16_t *S16;  // on-chip local positions (or null)
    const uint32_t *G;    // global positions (when S16 is null)
    const uint8_t *R;     // iteration index
    uint8_t *F;           // 1: sorted as leftover (last conflict array or out of order)
    const uint32_t *P;    // payload (nullable)
    const uint32_t *T;    // rows (nullable)
    Idx *X, *Y, *TB;
    uint32_t wm;
    __device__ __forceinline__ uint32_t ls(uint32_t i) const { return S16 ? S16[i] : (G[i] & wm); }
    __device__ __forceinline__ W ok(uint32_t i) const { return okey_of<W, FL>(K[i]); }
    __device__ __forceinline__ uint32_t tb(uint32_t i) const { return T ? T[i] : i; }
    __device__ __forceinline__ bool less(uint32_t a, uint32_t b) const {
        const unsigned long long ka = ok(a), kb = ok(b);
        return ka < kb || (ka == kb && tb(a) < tb(b));
    }
};

// Block-wide exclusive prefix maximum of one u64 per thread (0 where no thread before holds
// more). Ends without a barrier: the caller passes at least one __syncthreads() before it writes
// `scratch` again.
__device__ __forceinline__ unsigned long long block_excl_max_u64(unsigned long long v,
                                                                 unsigned long long *scratch /*SNW*/) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x = y > x ? y : x;
    }
    unsigned long long ex = __shfl_up_sync(0xFFFFFFFFu, x, 1);
    if (lane == 0) ex = 0;
    if (lane == 31) scratch[wid] = x;
    __syncthreads();
    // every warp folds the totals of the warps before it
    unsigned long long m = lane < wid ? scratch[lane] : 0ull;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, m, o);
        m = y > m ? y : m;
    }
    return m > ex ? m : ex;
}

// Fig. "Algorithm polish", first part: for each o_r its stored elements in position order and the
// out-of-order split against the running maximum (carry from earlier buckets first); the in-order
// rest is the run R_r. Sets v.F for leftover elements (last conflict array and out-of-order ones)
// and counts the out-of-order ones in sm.ooo.
template <typename W, typename Idx, bool FL>
__device__ void polish_runs(const SolveArgs &a, PolishSmem &sm, const BucketView<W, Idx, FL> &v,
                            uint32_t b, uint32_t nbk) {
    const int tid = threadIdx.x;
    const int t = sm.t;
    const uint32_t Wn = v.wm + 1u;
    const Idx EMPTY = (Idx)~(Idx)0;
    constexpr int LB = 8;  // element loads issued together (the view may be in global memory)
    for (uint32_t i0 = 0; i0 < nbk; i0 += SOLVE_THREADS * LB) {
        uint8_t rv[LB];
#pragma unroll
        for (int q = 0; q < LB; ++q) {
            const uint32_t i = i0 + q * SOLVE_THREADS + tid;
            rv[q] = i < nbk ? v.R[i] : 0;
        }
#pragma unroll
        for (int q = 0; q < LB; ++q) {
            const uint32_t i = i0 + q * SOLVE_THREADS + tid;
            if (i < nbk) v.F[i] = (rv[q] >= t) ? 1 : 0;
        }
    }
    if (tid < MAXR) sm.ooo[tid] = 0;
    if (tid < t) {
        const OKey cr = a.carry[(size_t)b * MAXR + tid];
        sm.carry[tid].k = cr.k;
        sm.carry[tid].tb = cr.tb;
        sm.carry[tid].valid = cr.valid;
    }
    __syncthreads();
    // 32-bit keys with a position table of at most NBIN entries keep each stored element's order
    // image beside its index in the table (the bin counters, idle until the bucket sort)
    const bool packed = sizeof(W) == 4 && Wn <= NBIN;
    uint32_t *TK = sm.bins;
    for (int r = 0; r < t; ++r) {
        // o_r: stored elements in position order
        for (uint32_t j = tid; j < Wn; j += SOLVE_THREADS) v.TB[j] = EMPTY;
        __syncthreads();
        for (uint32_t i0 = 0; i0 < nbk; i0 += SOLVE_THREADS * LB) {
            uint32_t pv[LB];
#pragma unroll
            for (int q = 0; q < LB; ++q) {
                const uint32_t i = i0 + q * SOLVE_THREADS + tid;
                pv[q] = (i < nbk && v.R[i] == r) ? v.ls(i) : 0xFFFFFFFFu;
            }
#pragma unroll
            for (int q = 0; q < LB; ++q)
                if (pv[q] != 0xFFFFFFFFu) {
                    const uint32_t i = i0 + q * SOLVE_THREADS + tid;
                    v.TB[pv[q]] = (Idx)i;
                    if (packed) TK[pv[q]] = (uint32_t)v.ok(i);
                }
        }
        __syncthreads();
        // out-of-order split against the running maximum (carry from earlier buckets first), run
        // over the position table itself: each thread takes a contiguous range of positions, so
        // thread order is position order
        const uint32_t per_s = (Wn + SOLVE_THREADS - 1) / SOLVE_THREADS;
        const uint32_t p0 = std::min(Wn, tid * per_s), p1 = std::min(Wn, p0 + per_s);
        if (packed) {
            // (order image, tie-break) packed as order image * 2^32 + tie-break: the pair order is
            // the integer order, and (0, 0) -- the least pair -- stands for "none", which leaves
            // every maximum and every out-of-order test unchanged
            unsigned long long loc = 0;
#pragma unroll 8
            for (uint32_t j = p0; j < p1; ++j) {
                const Idx x = v.TB[j];
                if (x == EMPTY) continue;
                const unsigned long long e = ((unsigned long long)TK[j] << 32) | v.tb(x);
                loc = e > loc ? e : loc;
            }
            unsigned long long run =
                block_excl_max_u64(loc, reinterpret_cast<unsigned long long *>(sm.kscratch));
            const KMax cr = sm.carry[r];
            const unsigned long long cp = cr.valid ? ((cr.k << 32) | cr.tb) : 0ull;
            run = cp > run ? cp : run;
            uint32_t evicted = 0;
#pragma unroll 8
            for (uint32_t j = p0; j < p1; ++j) {
                const Idx x = v.TB[j];
                if (x == EMPTY) continue;
                const unsigned long long e = ((unsigned long long)TK[j] << 32) | v.tb(x);
                if (e < run) {
                    v.F[x] = 1;
                    ++evicted;
                } else {
                    run = e;
                }
            }
            if (evicted) atomicAdd(&sm.ooo[r], evicted);
            __syncthreads();
            continue;
        }
        KMax loc = kmax_none();
        for (uint32_t j = p0; j < p1; ++j) {
            const Idx x = v.TB[j];
            if (x == EMPTY) continue;
            KMax e; e.k = v.ok(x); e.tb = v.tb(x); e.valid = 1;
            loc = kmax(loc, e);
        }
        KMax run = block_excl_max(loc, sm.kscratch, nullptr);
        run = kmax(sm.carry[r], run);
        uint32_t evicted = 0;
        for (uint32_t j = p0; j < p1; ++j) {
            const Idx x = v.TB[j];
            if (x == EMPTY) continue;
            const unsigned long long xk = v.ok(x);
            const uint32_t xt = v.tb(x);
            if (run.valid && okey_less(xk, xt, run.k, run.tb)) {
                v.F[x] = 1;
                ++evicted;
            } else {
                run.k = xk; run.tb = xt; run.valid = 1;
            }
        }
        if (evicted) atomicAdd(&sm.ooo[r], evicted);
        __syncthreads();
    }
}

template <typename W, typename Idx, bool FL>
__device__ void polish_bucket(const SolveArgs &a, PolishSmem &sm, const BucketView<W, Idx, FL> &v,
                              uint32_t b, uint32_t s0, uint32_t nbk, const Seg &sg,
                              uint32_t *pair, uint16_t *out16) {
    const int tid = threadIdx.x;
    const int t = sm.t;
    const int keybits = (a.key_bytes == 4) ? 32 : 64;
    polish_runs<W, Idx, FL>(a, sm, v, b, nbk);
    // The bucket's output -- the leftover (the last conflict array and every out-of-order element)
    // sorted by QuickSort(w) and merged with the in-order runs R_1..R_t of Fig. "Algorithm polish" --
    // is all of its elements in (key, row) order, so it is computed as one stable sort of the whole
    // bucket; the runs above supply the out-of-order counts and the fates.
    auto kf = [&](Idx x) { return v.ok(x); };
    Idx *A = nbk <= BIN_SORT_MAX ? cta_bin_sort<Idx>(v.X, v.Y, nbk, kf, sm.bins, sm.mm, sm.scratch, pair, out16)
                                 : nullptr;
    if (!A) {
        for (uint32_t i = tid; i < nbk; i += SOLVE_THREADS) v.X[i] = (Idx)i;
        __syncthreads();
        A = cta_radix_sort<Idx>(v.X, v.Y, nbk, keybits, kf, sm.hist, sm.wcnt, sm.scratch);
    }
    __syncthreads();
    // write the bucket's sorted run in place of the caller's array
    const uint64_t off = (uint64_t)s0 - sg.ebase;
    W *outk = reinterpret_cast<W *>(sg.keys) + off;
    int32_t *outp = sg.payload ? sg.payload + off : nullptr;
    for (uint32_t p = tid; p < nbk; p += SOLVE_THREADS) {
        const uint32_t x = A[p];
        outk[p] = v.K[x];
        if (outp) outp[p] = (int32_t)v.P[x];
        if (a.out_rows) a.out_rows[s0 + p] = v.T[x];
        if (a.fate) {
            const int rr = v.R[x];
            const int8_t f = (rr < t) ? (int8_t)(v.F[x] ? -(rr + 1) : (rr + 1)) : (int8_t)0;
            a.fate[v.T[x]] = f;
        }
    }
    if (tid < t && sm.ooo[tid]) atomicAdd(&a.stats[sm.seg].ooo[tid], (unsigned long long)sm.ooo[tid]);
    if (tid == 0) {
        const uint32_t xf = A[0], xl = A[nbk - 1];
        OKey lo, hi;
        lo.k = v.ok(xf); lo.tb = v.T ? v.T[xf] : 0u; lo.valid = 1;
        hi.k = v.ok(xl); hi.tb = v.T ? v.T[xl] : 0u; hi.valid = 1;
        a.blo[b] = lo;
        a.bhi[b] = hi;
    }
}

int polish_capacity(int key_bytes, bool payload, bool rows, int wlog, int blocks_per_sm,
                    size_t *smem_bytes) {
    const size_t fixed = sizeof(PolishSmem) + 256;
    const size_t tbl = ((size_t)2 << wlog);  // on chip the position table holds 16-bit indices
    const size_t per = key_bytes + 2 + 1 + 1 + (payload ? 4 : 0) + (rows ? 4 : 0) + 2 * 2;
    // shared memory per SM is 228 KB (227 KB usable by one block); each resident block reserves
    // 1 KB. When the position table leaves no room at this many blocks per SM, fewer blocks share
    // the SM; with no room even for one block every bucket takes the global-memory path.
    long cap = 0;
    for (int pb = std::max(1, blocks_per_sm); pb >= 1; --pb) {
        const long budget = (pb == 1) ? 227L * 1024 : (228L * 1024) / pb - 1024 - 512;
        cap = (budget - (long)fixed - (long)tbl - 64) / (long)per;
        if (cap >= 256) break;
    }
    cap = std::max<long>(0, std::min<long>(cap, 65534));
    cap &= ~15L;
    if (smem_bytes) *smem_bytes = fixed + tbl + (size_t)cap * per + 64;
    return (int)cap;
}

template <typename W, bool FL>
__global__ void __launch_bounds__(SOLVE_THREADS) k_polish(SolveArgs a) {
    extern __shared__ __align__(16) unsigned char praw[];
    PolishSmem &sm = *reinterpret_cast<PolishSmem *>(praw);
    unsigned char *dyn = praw + ((sizeof(PolishSmem) + 15) & ~(size_t)15);
    const int tid = threadIdx.x;
    const uint32_t b = a.order ? a.order[blockIdx.x] : blockIdx.x;
    const uint32_t s0 = a.bstart[b], s1 = a.bstart[b + 1];
    const uint32_t nbk = s1 - s0;
    if (nbk == 0) return;
    if (*a.err) return;  // NaN keys / bad positions: leave the caller's arrays untouched
    if (tid == 0) {
        sm.seg = seg_of_bucket(a.segs, a.nseg, b);
        sm.t = (int)a.stats[sm.seg].t;
    }
    __syncthreads();
    const Seg &sg = a.segs[sm.seg];
    const uint32_t Wn = 1u << a.wlog;
    const uint32_t cap = (uint32_t)a.polish_cap;
    if (a.big && nbk > POLISH_BIG) {
        // the runs of o_1..o_t are split here (out-of-order counts); the bucket's output -- the
        // merge of the sorted leftover with the runs, i.e. its elements in (key, row) order -- is
        // left to the multi-block sort of all such buckets
        if (tid == 0) atomicAdd(&a.stats[sm.seg].oversized, 1u);
        uint32_t *TB = reinterpret_cast<uint32_t *>(dyn);
        BucketView<W, uint32_t, FL> v{reinterpret_cast<const W *>(a.keys) + s0, nullptr, a.gs + s0,
                                      a.rank + s0, a.g_flag + s0, nullptr, nullptr, a.g_x + s0,
                                      a.g_y + s0, TB, Wn - 1u};
        polish_runs<W, uint32_t, FL>(a, sm, v, b, nbk);
        if (tid < sm.t && sm.ooo[tid]) atomicAdd(&a.stats[sm.seg].ooo[tid], (unsigned long long)sm.ooo[tid]);
        if (tid == 0) {
            BigRange r;
            r.lo = s0; r.hi = s1; r.seg = (uint32_t)sm.seg; r.off = 0; r.b = b; r.pad = 0;
            a.big[atomicAdd(a.big_cnt, 1u)] = r;
        }
        return;
    }
    if (nbk <= cap) {
        // on-chip: stage the bucket in shared memory
        unsigned char *p = dyn;
        uint16_t *TB = reinterpret_cast<uint16_t *>(p); p += (size_t)2 * Wn;  // 16-bit element indices
        W *K = reinterpret_cast<W *>(p); p += (size_t)sizeof(W) * cap;
        uint32_t *P = nullptr, *T = nullptr;
        if (a.pay) { P = reinterpret_cast<uint32_t *>(p); p += (size_t)4 * cap; }
        if (a.rows) { T = reinterpret_cast<uint32_t *>(p); p += (size_t)4 * cap; }
        uint16_t *S16 = reinterpret_cast<uint16_t *>(p); p += (size_t)2 * cap;
        uint16_t *X = reinterpret_cast<uint16_t *>(p); p += (size_t)2 * cap;
        uint16_t *Y = reinterpret_cast<uint16_t *>(p); p += (size_t)2 * cap;
        uint8_t *R = p; p += cap;
        uint8_t *F = p; p += cap;
        const W *gk = reinterpret_cast<const W *>(a.keys) + s0;
        const uint32_t *gg = a.gs + s0;
        const uint8_t *gr = a.rank + s0;
        constexpr int LB = 8;  // items per thread whose loads are issued together
        for (uint32_t b0 = 0; b0 < nbk; b0 += SOLVE_THREADS * LB) {
            W kr[LB];
            uint32_t sr[LB], pr[LB], tr[LB];
            uint8_t rr[LB];
#pragma unroll
            for (int q = 0; q < LB; ++q) {
                const uint32_t i = b0 + q * SOLVE_THREADS + tid;
                if (i < nbk) {
                    kr[q] = gk[i];
                    sr[q] = gg[i];
                    rr[q] = gr[i];
                    if (P) pr[q] = a.pay[s0 + i];
                    if (T) tr[q] = a.rows[s0 + i];
                }
            }
#pragma unroll
            for (int q = 0; q < LB; ++q) {
                const uint32_t i = b0 + q * SOLVE_THREADS + tid;
                if (i < nbk) {
                    K[i] = kr[q];
                    S16[i] = (uint16_t)(sr[q] & (Wn - 1u));
                    R[i] = rr[q];
                    if (P) P[i] = pr[q];
                    if (T) T[i] = tr[q];
                }
            }
        }
        __syncthreads();
        BucketView<W, uint16_t, FL> v{K, S16, nullptr, R, F, P, T, X, Y, TB, Wn - 1u};
        // X and Y are adjacent: together one u32 per element for the bucket sort's packed words;
        // the result goes to S16, idle once the runs are split
        polish_bucket<W, uint16_t, FL>(a, sm, v, b, s0, nbk, sg, reinterpret_cast<uint32_t *>(X), S16);
    } else {
        if (tid == 0) atomicAdd(&a.stats[sm.seg].oversized, 1u);
        uint32_t *TB = reinterpret_cast<uint32_t *>(dyn);
        BucketView<W, uint32_t, FL> v{reinterpret_cast<const W *>(a.keys) + s0, nullptr, a.gs + s0,
                                      a.rank + s0, a.g_flag + s0, a.pay ? a.pay + s0 : nullptr,
                                      a.rows ? a.rows + s0 : nullptr, a.g_x + s0, a.g_y + s0,
                                      TB, Wn - 1u};
        polish_bucket<W, uint32_t, FL>(a, sm, v, b, s0, nbk, sg, nullptr, nullptr);
    }
}

// ---------------------------------------------------------------------------------------------
// Seam repair. Every bucket's output is sorted; across buckets a non-monotone f can leave elements
// on the wrong side of a bucket boundary. Call the boundary before output position p a cut; it is
// sound when every element before it is <= every element after it (in (key, row) order when rows
// are carried). The array is sorted exactly when every cut is sound, and sorting each maximal run
// of elements between consecutive sound cuts, independently, sorts the array. Inside a bucket with
// sorted elements e_0 <= ... <= e_{len-1}, preceded by elements whose maximum is P and followed by
// elements whose minimum is S, the cut before e_j is sound iff P <= S and P <= e_j and
// e_{j-1} <= S; with P <= S these hold for j in [#{e < P}, #{e <= S}], a non-empty interval.
//   k_seam_ps / k_seam_cuts / k_seam_emit -- per bucket the largest element before it and the
//                   smallest after it, its first and last sound cut, then the runs between
//                   consecutive sound cuts that hold two or more elements.
//   k_seam_fix   -- blocks take the runs of at most SEAM_CTA_MAX elements one by one and sort each
//                   on chip; longer runs go to the multi-block sort on the host's side (or are
//                   sorted here too when rows are carried or deferral is off).
__device__ __forceinline__ KMax kinv(const KMax &x) {
    KMax r; r.k = ~x.k; r.tb = ~x.tb; r.valid = x.valid; return r;
}

// Scans over an array's buckets walk tiles of SOLVE_THREADS consecutive buckets (one per thread,
// coalesced loads) with the running value carried from tile to tile; a backward scan gives thread
// t the bucket tile_end - 1 - t, so that an exclusive scan over threads runs over later buckets.
// 1) k_seam_ps (one block per array): S(b) = the smallest element of the buckets after b,
//    P(b) = the largest element of the buckets before b.
__global__ void __launch_bounds__(SCAN_THREADS) k_seam_ps(SolveArgs a) {
    // tiles of PSI * SCAN_THREADS buckets, PSI consecutive ones per thread: a thread folds its own
    // buckets in order and one block scan per tile carries the rest
    constexpr int PSI = 8;
    constexpr uint32_t PST = SCAN_THREADS * PSI;
    __shared__ KMax ks[33];
    __shared__ KMax tot;
    const int s = blockIdx.x, tid = threadIdx.x;
    if (*a.err) return;
    const Seg &sg = a.segs[s];
    const uint32_t nb = sg.nb, bb = sg.bbase;
    auto okey = [&](const OKey &o) { KMax x; x.k = o.k; x.tb = o.tb; x.valid = o.valid; return x; };
    KMax v[PSI];
    KMax carry = kmax_none();  // inverted minimum of the buckets after the current tile
    for (uint32_t t1 = nb; t1 > 0;) {
        const uint32_t t0 = t1 > PST ? t1 - PST : 0;
        KMax loc = kmax_none();
        uint32_t nem = 0;  // bit k: this thread's bucket k is non-empty
#pragma unroll
        for (int k = 0; k < PSI; ++k) {  // this thread's buckets, later ones first
            const uint32_t r = (uint32_t)tid * PSI + k;
            const bool own = r < t1 - t0;
            const uint32_t bi = bb + (own ? t1 - 1 - r : 0u);
            // bounds and key read together; the key of an empty bucket is read but not used
            const uint32_t s0 = a.bstart[bi], s1 = a.bstart[bi + 1];
            const OKey o = a.blo[bi];
            const bool ne = own && s1 > s0;
            nem |= (ne ? 1u : 0u) << k;
            v[k] = ne ? kinv(okey(o)) : kmax_none();
            loc = kmax(loc, v[k]);
        }
        KMax run = kmax(carry, block_excl_max(loc, ks, &tot));
#pragma unroll
        for (int k = 0; k < PSI; ++k) {
            if ((nem >> k) & 1u) {
                const uint32_t bi = bb + (t1 - 1 - ((uint32_t)tid * PSI + k));
                const KMax sv = kinv(run);
                OKey o; o.k = sv.k; o.tb = sv.tb; o.valid = sv.valid;
                a.seam_suf[bi] = o;
                run = kmax(run, v[k]);
            }
        }
        carry = kmax(carry, tot);
        t1 = t0;
    }
    carry = kmax_none();  // maximum of the buckets before the current tile
    for (uint32_t t0 = 0; t0 < nb; t0 += PST) {
        KMax loc = kmax_none();
        uint32_t nem = 0;
#pragma unroll
        for (int k = 0; k < PSI; ++k) {
            const uint32_t c = t0 + (uint32_t)tid * PSI + k;
            const bool own = c < nb;
            const uint32_t bi = bb + (own ? c : 0u);
            const uint32_t s0 = a.bstart[bi], s1 = a.bstart[bi + 1];
            const OKey o = a.bhi[bi];
            const bool ne = own && s1 > s0;
            nem |= (ne ? 1u : 0u) << k;
            v[k] = ne ? okey(o) : kmax_none();
            loc = kmax(loc, v[k]);
        }
        KMax run = kmax(carry, block_excl_max(loc, ks, &tot));
#pragma unroll
        for (int k = 0; k < PSI; ++k) {
            if ((nem >> k) & 1u) {
                const uint32_t bi = bb + t0 + (uint32_t)tid * PSI + k;
                OKey o; o.k = run.k; o.tb = run.tb; o.valid = run.valid;
                a.seam_pre[bi] = o;
                run = kmax(run, v[k]);
            }
        }
        carry = kmax(carry, tot);
    }
}

// One large array: k_seam_ps over tiles of MT_TILE buckets on many blocks (tile extrema; their
// exclusive suffix minimum / prefix maximum in one block; each tile's scans from them).
// agg[2 i] = inverted minimum of tile i's non-empty buckets (blo), agg[2 i + 1] = their maximum (bhi)
__global__ void __launch_bounds__(MT_THREADS) k_seam_tiles(SolveArgs a, OKey *agg) {
    __shared__ KMax scratch[33];
    __shared__ KMax tot;
    if (*a.err) return;
    const int tid = threadIdx.x;
    const Seg &sg = a.segs[0];
    const uint32_t c0 = blockIdx.x * MT_TILE + (uint32_t)tid * MT_PER;
    KMax lo = kmax_none(), hi = kmax_none();
#pragma unroll
    for (int k = 0; k < MT_PER; ++k) {
        const uint32_t c = c0 + k;
        if (c < sg.nb) {
            const uint32_t bi = sg.bbase + c;
            if (a.bstart[bi + 1] > a.bstart[bi]) {
                lo = kmax(lo, kinv(kmax_of(a.blo[bi])));
                hi = kmax(hi, kmax_of(a.bhi[bi]));
            }
        }
    }
    block_excl_max(lo, scratch, &tot);
    if (tid == 0) agg[2 * (size_t)blockIdx.x] = okey_of_kmax(tot);
    block_excl_max(hi, scratch, &tot);
    if (tid == 0) agg[2 * (size_t)blockIdx.x + 1] = okey_of_kmax(tot);
}
// agg[2 i] <- inverted minimum over the tiles after i; agg[2 i + 1] <- maximum over the tiles before i
__global__ void __launch_bounds__(MT_THREADS) k_seam_prefix(SolveArgs a, OKey *agg, uint32_t ntiles) {
    __shared__ KMax scratch[33];
    if (*a.err) return;
    const int tid = threadIdx.x;
    {   // suffix: thread tid takes tiles ntiles - 1 - (tid * MT_PER + k)
        KMax v[MT_PER], loc = kmax_none();
#pragma unroll
        for (int k = 0; k < MT_PER; ++k) {
            const uint32_t r = (uint32_t)tid * MT_PER + k;
            v[k] = r < ntiles ? kmax_of(agg[2 * (size_t)(ntiles - 1 - r)]) : kmax_none();
            loc = kmax(loc, v[k]);
        }
        KMax run = block_excl_max(loc, scratch, nullptr);
#pragma unroll
        for (int k = 0; k < MT_PER; ++k) {
            const uint32_t r = (uint32_t)tid * MT_PER + k;
            if (r < ntiles) agg[2 * (size_t)(ntiles - 1 - r)] = okey_of_kmax(run);
            run = kmax(run, v[k]);
        }
    }
    {
        KMax v[MT_PER], loc = kmax_none();
#pragma unroll
        for (int k = 0; k < MT_PER; ++k) {
            const uint32_t i = (uint32_t)tid * MT_PER + k;
            v[k] = i < ntiles ? kmax_of(agg[2 * (size_t)i + 1]) : kmax_none();
            loc = kmax(loc, v[k]);
        }
        KMax run = block_excl_max(loc, scratch, nullptr);
#pragma unroll
        for (int k = 0; k < MT_PER; ++k) {
            const uint32_t i = (uint32_t)tid * MT_PER + k;
            if (i < ntiles) agg[2 * (size_t)i + 1] = okey_of_kmax(run);
            run = kmax(run, v[k]);
        }
    }
}
__global__ void __launch_bounds__(MT_THREADS) k_seam_apply(SolveArgs a, const OKey *agg) {
    __shared__ KMax scratch[33];
    if (*a.err) return;
    const int tid = threadIdx.x;
    const Seg &sg = a.segs[0];
    const uint32_t t0 = blockIdx.x * MT_TILE;
    const uint32_t t1 = std::min<uint32_t>(sg.nb, t0 + MT_TILE);
    {   // S(b): thread tid takes the tile's buckets t1 - 1 - (tid * MT_PER + k), later ones first
        KMax v[MT_PER], loc = kmax_none();
        uint32_t nem = 0;
#pragma unroll
        for (int k = 0; k < MT_PER; ++k) {
            const uint32_t r = (uint32_t)tid * MT_PER + k;
            const bool own = r < t1 - t0;
            const uint32_t bi = sg.bbase + (own ? t1 - 1 - r : 0u);
            const bool ne = own && a.bstart[bi + 1] > a.bstart[bi];
            nem |= (ne ? 1u : 0u) << k;
            v[k] = ne ? kinv(kmax_of(a.blo[bi])) : kmax_none();
            loc = kmax(loc, v[k]);
        }
        KMax run = kmax(kmax_of(agg[2 * (size_t)blockIdx.x]), block_excl_max(loc, scratch, nullptr));
#pragma unroll
        for (int k = 0; k < MT_PER; ++k) {
            if ((nem >> k) & 1u) {
                a.seam_suf[sg.bbase + t1 - 1 - ((uint32_t)tid * MT_PER + k)] = okey_of_kmax(kinv(run));
                run = kmax(run, v[k]);
            }
        }
    }
    {   // P(b)
        KMax v[MT_PER], loc = kmax_none();
        uint32_t nem = 0;
#pragma unroll
        for (int k = 0; k < MT_PER; ++k) {
            const uint32_t c = t0 + (uint32_t)tid * MT_PER + k;
            const bool own = c < t1;
            const uint32_t bi = sg.bbase + (own ? c : 0u);
            const bool ne = own && a.bstart[bi + 1] > a.bstart[bi];
            nem |= (ne ? 1u : 0u) << k;
            v[k] = ne ? kmax_of(a.bhi[bi]) : kmax_none();
            loc = kmax(loc, v[k]);
        }
        KMax run = kmax(kmax_of(agg[2 * (size_t)blockIdx.x + 1]), block_excl_max(loc, scratch, nullptr));
#pragma unroll
        for (int k = 0; k < MT_PER; ++k) {
            if ((nem >> k) & 1u) {
                a.seam_pre[sg.bbase + t0 + (uint32_t)tid * MT_PER + k] = okey_of_kmax(run);
                run = kmax(run, v[k]);
            }
        }
    }
}

// 2) k_seam_cuts (one thread per bucket of every array): the bucket's first and last sound cut.
template <typename W>
__global__ void k_seam_cuts(SolveArgs a) {
    const uint32_t bi = blockIdx.x * blockDim.x + threadIdx.x;
    if (bi >= a.NB || *a.err) return;
    const unsigned long long NONE = ~0ull;
    if (a.bstart[bi + 1] == a.bstart[bi]) {
        a.seam_cut[2 * (size_t)bi] = NONE;
        a.seam_cut[2 * (size_t)bi + 1] = NONE;
        return;
    }
    const Seg &sg = a.segs[seg_of_bucket(a.segs, a.nseg, bi)];
    const W *outk = reinterpret_cast<const W *>(sg.keys);
    auto okey = [&](const OKey &o) { KMax x; x.k = o.k; x.tb = o.tb; x.valid = o.valid; return x; };
    auto elem = [&](unsigned long long pos, unsigned long long &k, uint32_t &tb) {
        k = ordbits(word64(outk[pos]), a.dtype);
        tb = a.out_rows ? a.out_rows[sg.ebase + pos] : 0u;
    };
    const KMax P = okey(a.seam_pre[bi]), S = okey(a.seam_suf[bi]);
    const unsigned long long b0 = a.bstart[bi] - sg.ebase, b1 = a.bstart[bi + 1] - sg.ebase;
    unsigned long long fg = NONE, lg = NONE;
    if (!(P.valid && S.valid && okey_less(S.k, S.tb, P.k, P.tb))) {
        unsigned long long l = b0, h = b1;  // A = #{e < P}
        if (P.valid) {
            while (l < h) {
                const unsigned long long mid = (l + h) >> 1;
                unsigned long long k; uint32_t tb;
                elem(mid, k, tb);
                if (okey_less(k, tb, P.k, P.tb)) l = mid + 1; else h = mid;
            }
        }
        fg = l;
        l = fg; h = b1;  // B = #{e <= S}
        if (S.valid) {
            while (l < h) {
                const unsigned long long mid = (l + h) >> 1;
                unsigned long long k; uint32_t tb;
                elem(mid, k, tb);
                if (!okey_less(S.k, S.tb, k, tb)) l = mid + 1; else h = mid;
            }
        } else {
            l = b1;
        }
        lg = l;
    }
    a.seam_cut[2 * (size_t)bi] = fg;
    a.seam_cut[2 * (size_t)bi + 1] = lg;
}

// 3) k_seam_emit (one block per array): the runs between consecutive sound cuts that hold two or
//    more elements (backward: the next bucket's first sound cut).
__global__ void __launch_bounds__(SCAN_THREADS) k_seam_emit(SolveArgs a) {
    constexpr int NW = SCAN_THREADS / 32;
    __shared__ unsigned long long wmin[NW];
    const int s = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (*a.err) return;
    const Seg &sg = a.segs[s];
    const uint32_t nb = sg.nb, bb = sg.bbase;
    // a sound cut is a position below n, so NONE (all ones) is the identity of the minimum
    const unsigned long long n = sg.n, NONE = ~0ull;
    auto emit = [&](unsigned long long lo, unsigned long long hi) {
        if (hi - lo < 2) return;
        atomicAdd(&a.stats[s].repaired, hi - lo);
        atomicAdd(&a.stats[s].ranges, 1u);
        SeamRange r; r.lo = lo; r.hi = hi; r.seg = (uint32_t)s; r.pad = 0;
        if (a.allow_defer && !a.out_rows && hi - lo > SEAM_CTA_MAX) {
            const uint32_t i = atomicAdd(&a.seam_cnt[1], 1u);
            a.ranges[a.max_ranges - 1 - i] = r;
        } else {
            a.ranges[atomicAdd(&a.seam_cnt[0], 1u)] = r;
        }
    };
    auto umin = [](unsigned long long x, unsigned long long y) { return y < x ? y : x; };
    // tiles of PSI * SCAN_THREADS buckets, PSI consecutive ones per thread (later ones first)
    constexpr int PSI = 8;
    constexpr uint32_t PST = SCAN_THREADS * PSI;
    unsigned long long carry = NONE;  // smallest first sound cut after the current tile
    for (uint32_t t1 = nb; t1 > 0;) {
        const uint32_t t0 = t1 > PST ? t1 - PST : 0;
        unsigned long long fg[PSI], lg[PSI];
        unsigned long long loc = NONE;
#pragma unroll
        for (int k = 0; k < PSI; ++k) {
            const uint32_t r = (uint32_t)tid * PSI + k;
            const bool own = r < t1 - t0;
            const uint32_t bi = bb + (t1 - 1 - r);
            fg[k] = own ? a.seam_cut[2 * (size_t)bi] : NONE;
            lg[k] = own ? a.seam_cut[2 * (size_t)bi + 1] : NONE;
            loc = umin(loc, fg[k]);
        }
        // exclusive minimum over the threads before this one (they hold later buckets)
        unsigned long long x = loc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= o) x = umin(x, y);
        }
        unsigned long long ex = __shfl_up_sync(0xFFFFFFFFu, x, 1);
        if (lane == 0) ex = NONE;
        if (lane == 31) wmin[wid] = x;
        __syncthreads();
        unsigned long long before = lane < wid ? wmin[lane] : NONE;
        unsigned long long all = lane < NW ? wmin[lane] : NONE;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            before = umin(before, __shfl_xor_sync(0xFFFFFFFFu, before, o));
            all = umin(all, __shfl_xor_sync(0xFFFFFFFFu, all, o));
        }
        __syncthreads();  // wmin is written again by the next tile
        unsigned long long run = umin(carry, umin(before, ex));
#pragma unroll
        for (int k = 0; k < PSI; ++k) {
            if (lg[k] != NONE) emit(lg[k], run != NONE ? run : n);
            run = umin(run, fg[k]);
        }
        carry = umin(carry, all);
        t1 = t0;
    }
    if (tid == 0) emit(0, carry != NONE ? carry : n);  // before the first sound cut
}

// re-sort out[lo, lo + len) of one array by (key, row): the range is a union of sorted runs. The
// two index lists of the sort live in shared memory (sX, sY: SEAM_SMEM_IDX entries each) when the
// range fits, else in the global scratch.
constexpr uint32_t SEAM_SMEM_IDX = 8192;
template <typename W>
__device__ void repair_range(const SolveArgs &a, PolishSmem &sm, const Seg &sg, uint64_t lo,
                             uint32_t len, uint32_t *sX, uint32_t *sY) {
    const int tid = threadIdx.x, dt = a.dtype;
    W *outk = reinterpret_cast<W *>(sg.keys);
    const bool onchip = len <= SEAM_SMEM_IDX;
    uint32_t *X = onchip ? sX : a.g_x + sg.ebase + lo, *Y = onchip ? sY : a.g_y + sg.ebase + lo;
    for (uint32_t i = tid; i < len; i += SOLVE_THREADS) X[i] = i;
    __syncthreads();
    const W *rk = outk + lo;
    const uint32_t *rr = a.out_rows ? a.out_rows + sg.ebase + lo : nullptr;
    uint32_t *res = X;
    if (rr) {
        auto rkf = [&](uint32_t x) -> unsigned long long { return rr[x]; };
        res = cta_radix_sort<uint32_t>(X, Y, len, 32, rkf, sm.hist, sm.wcnt, sm.scratch);
    }
    uint32_t *oth = (res == X) ? Y : X;
    auto kkf = [&](uint32_t x) -> unsigned long long { return ordbits(word64(rk[x]), dt); };
    res = cta_radix_sort<uint32_t>(res, oth, len, a.key_bytes * 8, kkf, sm.hist, sm.wcnt, sm.scratch);
    __syncthreads();
    // gather through scratch, then copy back
    W *tk = reinterpret_cast<W *>(a.key_scratch) + sg.ebase + lo;
    uint32_t *tp = a.pay_scratch ? a.pay_scratch + sg.ebase + lo : nullptr;
    uint32_t *tr = a.row_scratch ? a.row_scratch + sg.ebase + lo : nullptr;
    int32_t *op = sg.payload ? sg.payload + lo : nullptr;
    for (uint32_t i = tid; i < len; i += SOLVE_THREADS) {
        const uint32_t x = res[i];
        tk[i] = rk[x];
        if (op && tp) tp[i] = (uint32_t)op[x];
        if (rr && tr) tr[i] = rr[x];
    }
    __syncthreads();
    for (uint32_t i = tid; i < len; i += SOLVE_THREADS) {
        outk[lo + i] = tk[i];
        if (op && tp) op[i] = (int32_t)tp[i];
        if (rr && tr) a.out_rows[sg.ebase + lo + i] = tr[i];
    }
    __syncthreads();
}

template <typename W>
__global__ void __launch_bounds__(SOLVE_THREADS) k_seam_fix(SolveArgs a) {
    extern __shared__ __align__(16) unsigned char sraw[];
    PolishSmem &sm = *reinterpret_cast<PolishSmem *>(sraw);
    uint32_t *sX = reinterpret_cast<uint32_t *>(sraw + ((sizeof(PolishSmem) + 15) & ~(size_t)15));
    uint32_t *sY = sX + SEAM_SMEM_IDX;
    __shared__ uint32_t sh_r;
    if (*a.err) return;
    const uint32_t nr = a.seam_cnt[0];
    for (;;) {
        if (threadIdx.x == 0) sh_r = atomicAdd(&a.seam_cnt[2], 1u);
        __syncthreads();
        const uint32_t r = sh_r;
        __syncthreads();
        if (r >= nr) break;
        const SeamRange R = a.ranges[r];
        repair_range<W>(a, sm, a.segs[R.seg], R.lo, (uint32_t)(R.hi - R.lo), sX, sY);
    }
}

// Buckets above POLISH_BIG: k_big_pack copies their partitioned elements (br sorted by position,
// br[j].off = packed offset) into the packed buffers with the bucket's list index j, or, with
// unpack = 1, the sorted packed elements to the bucket's output positions; k_big_bounds records
// each such bucket's first and last output element for the seam.
template <typename W>
__global__ void k_big_pack(const BigRange *br, uint32_t nr, const Seg *segs, uint64_t total, const W *sk,
                           const uint32_t *sp, W *pk, uint32_t *pp, uint32_t *pj, int unpack) {
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = nr - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (br[mid].off <= q) lo = mid; else hi = mid - 1;
        }
        const BigRange r = br[lo];
        if (!unpack) {
            const uint64_t e = r.lo + (q - r.off);
            pk[q] = sk[e];
            if (pp && sp) pp[q] = sp[e];
            if (pj) pj[q] = lo;
        } else {
            const Seg &sg = segs[r.seg];
            const uint64_t e = r.lo - sg.ebase + (q - r.off);
            reinterpret_cast<W *>(sg.keys)[e] = pk[q];
            if (pp && sg.payload) sg.payload[e] = (int32_t)pp[q];
        }
    }
}

template <typename W>
__global__ void k_big_bounds(const BigRange *br, uint32_t nr, const Seg *segs, int dtype, OKey *blo,
                             OKey *bhi) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nr) return;
    const BigRange r = br[j];
    const Seg &sg = segs[r.seg];
    const W *k = reinterpret_cast<const W *>(sg.keys);
    OKey lo, hi;
    lo.k = ordbits(word64(k[r.lo - sg.ebase]), dtype); lo.tb = 0; lo.valid = 1;
    hi.k = ordbits(word64(k[r.hi - 1 - sg.ebase]), dtype); hi.tb = 0; hi.valid = 1;
    blo[r.b] = lo;
    bhi[r.b] = hi;
}

cudaError_t launch_big_pack(const BigRange *br, uint32_t nr, const Seg *segs, uint64_t total, int key_bytes,
                            const void *src_k, const uint32_t *src_p, void *pk, uint32_t *pp, uint32_t *pj,
                            int unpack, int sms, cudaStream_t s) {
    if (total == 0 || nr == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, (uint64_t)sms * 8);
    if (key_bytes == 4)
        k_big_pack<uint32_t><<<grid, 256, 0, s>>>(br, nr, segs, total, (const uint32_t *)src_k, src_p,
                                                  (uint32_t *)pk, pp, pj, unpack);
    else
        k_big_pack<uint64_t><<<grid, 256, 0, s>>>(br, nr, segs, total, (const uint64_t *)src_k, src_p,
                                                  (uint64_t *)pk, pp, pj, unpack);
    return nns_launched(cudaGetLastError());
}

cudaError_t launch_big_bounds(const BigRange *br, uint32_t nr, const Seg *segs, int key_bytes, int dtype,
                              OKey *blo, OKey *bhi, cudaStream_t s) {
    if (nr == 0) return cudaSuccess;
    if (key_bytes == 4) k_big_bounds<uint32_t><<<(nr + 127) / 128, 128, 0, s>>>(br, nr, segs, dtype, blo, bhi);
    else k_big_bounds<uint64_t><<<(nr + 127) / 128, 128, 0, s>>>(br, nr, segs, dtype, blo, bhi);
    return nns_launched(cudaGetLastError());
}

// Long seam ranges are sorted together: the cut between two ranges is sound, so every element of
// one range is <= every element of the next, and one stable sort by key of all the ranges' elements,
// packed in output order, leaves each range's elements (equal keys included) in its own stretch.
// k_seam_pack copies the ranges (rg sorted by array and position, rg[j].pad = packed offset) into
// the packed buffers or, with unpack = 1, back.
template <typename W>
__global__ void k_seam_pack(const SeamRange *rg, uint32_t nr, const Seg *segs, uint64_t total, W *pk,
                            uint32_t *pp, uint32_t *ps, int unpack) {
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = nr - 1;
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (rg[mid].pad <= q) lo = mid; else hi = mid - 1;
        }
        const SeamRange r = rg[lo];
        const Seg &sg = segs[r.seg];
        const uint64_t e = r.lo + (q - r.pad);
        W *k = reinterpret_cast<W *>(sg.keys) + e;
        if (!unpack) {
            pk[q] = *k;
            if (pp && sg.payload) pp[q] = (uint32_t)sg.payload[e];
            if (ps) ps[q] = r.seg;
        } else {
            *k = pk[q];
            if (pp && sg.payload) sg.payload[e] = (int32_t)pp[q];
        }
    }
}

cudaError_t launch_seam_pack(const SeamRange *rg, uint32_t nr, const Seg *segs, uint64_t total,
                             int key_bytes, void *pk, uint32_t *pp, uint32_t *ps, int unpack, int sms,
                             cudaStream_t s) {
    if (total == 0 || nr == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, (uint64_t)sms * 8);
    if (key_bytes == 4)
        k_seam_pack<uint32_t><<<grid, 256, 0, s>>>(rg, nr, segs, total, (uint32_t *)pk, pp, ps, unpack);
    else
        k_seam_pack<uint64_t><<<grid, 256, 0, s>>>(rg, nr, segs, total, (uint64_t *)pk, pp, ps, unpack);
    return nns_launched(cudaGetLastError());
}

// ---------------------------------------------------------------------------------------------
template <typename W> static cudaError_t rounds_go(const SolveArgs &a, cudaStream_t s) {
    const size_t smem = rounds_smem(a.wlog);
    cudaError_t e = cudaFuncSetAttribute(k_rounds<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_rounds<W><<<a.NB, RT, smem, s>>>(a);
    return nns_launched(cudaGetLastError());
}
cudaError_t launch_rounds(const SolveArgs &a, cudaStream_t s) {
    if (a.NB == 0) return cudaSuccess;
    return a.key_bytes == 4 ? rounds_go<uint32_t>(a, s) : rounds_go<uint64_t>(a, s);
}

// the scans of one array of more than one tile of buckets run on many blocks
constexpr uint32_t MT_MIN_BUCKETS = MT_TILE + 1;

cudaError_t launch_finalize(const SolveArgs &a, cudaStream_t s) {
    const uint32_t nt = (a.NB + MT_TILE - 1) / MT_TILE;
    if (a.nseg == 1 && a.NB >= MT_MIN_BUCKETS && nt <= MT_TILE &&
        (uint64_t)nt * MAXR * sizeof(OKey) <= a.N * sizeof(uint32_t)) {
        // tile maxima in the g_y scratch (free between the rounds and the polish)
        OKey *agg = reinterpret_cast<OKey *>(a.g_y);
        k_finalize_tiles<<<nt, MT_THREADS, 0, s>>>(a, agg);
        cudaError_t e = nns_launched(cudaGetLastError());
        if (e != cudaSuccess) return e;
        k_finalize_prefix<<<1, MT_THREADS, 0, s>>>(a, agg, nt);
        if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
        k_finalize_apply<<<nt, MT_THREADS, 0, s>>>(a, agg);
        return nns_launched(cudaGetLastError());
    }
    k_finalize<<<a.nseg, SCAN_THREADS, 0, s>>>(a);
    return nns_launched(cudaGetLastError());
}

template <typename W> static cudaError_t polish_go(const SolveArgs &a, cudaStream_t s) {
    const size_t smem = std::max(a.polish_smem, sizeof(PolishSmem) + 16 + ((size_t)4 << a.wlog));
    // the key's order image with its type fixed at compile time (IEEE float or unsigned)
    auto kfn = (a.dtype == NNSORT_F32 || a.dtype == NNSORT_F64) ? k_polish<W, true> : k_polish<W, false>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kfn<<<a.NB, SOLVE_THREADS, smem, s>>>(a);
    return nns_launched(cudaGetLastError());
}
cudaError_t launch_polish(const SolveArgs &a, cudaStream_t s) {
    if (a.NB == 0) return cudaSuccess;
    return a.key_bytes == 4 ? polish_go<uint32_t>(a, s) : polish_go<uint64_t>(a, s);
}

template <typename W> static cudaError_t seam_go(const SolveArgs &a, int sms, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(a.seam_cnt, 0, 4 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const uint32_t nt = (a.NB + MT_TILE - 1) / MT_TILE;
    if (a.nseg == 1 && a.NB >= MT_MIN_BUCKETS && nt <= MT_TILE) {
        // tile extrema in the cut scratch (free until k_seam_cuts): 2 nt <= 2 NB entries of 16 bytes
        OKey *agg = reinterpret_cast<OKey *>(a.seam_cut);
        k_seam_tiles<<<nt, MT_THREADS, 0, s>>>(a, agg);
        if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
        k_seam_prefix<<<1, MT_THREADS, 0, s>>>(a, agg, nt);
        if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
        k_seam_apply<<<nt, MT_THREADS, 0, s>>>(a, agg);
    } else {
        k_seam_ps<<<a.nseg, SCAN_THREADS, 0, s>>>(a);
    }
    if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
    k_seam_cuts<W><<<(a.NB + 255) / 256, 256, 0, s>>>(a);
    if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
    k_seam_emit<<<a.nseg, SCAN_THREADS, 0, s>>>(a);
    if ((e = nns_launched(cudaGetLastError())) != cudaSuccess) return e;
    const size_t fix_smem = ((sizeof(PolishSmem) + 15) & ~(size_t)15) + 2 * sizeof(uint32_t) * SEAM_SMEM_IDX;
    if ((e = cudaFuncSetAttribute(k_seam_fix<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fix_smem)) !=
        cudaSuccess)
        return e;
    k_seam_fix<W><<<2 * sms, SOLVE_THREADS, fix_smem, s>>>(a);
    return nns_launched(cudaGetLastError());
}
cudaError_t launch_seam_repair(const SolveArgs &a, int sms, cudaStream_t s) {
    return a.key_bytes == 4 ? seam_go<uint32_t>(a, sms, s) : seam_go<uint64_t>(a, sms, s);
}

}  // namespace nns
