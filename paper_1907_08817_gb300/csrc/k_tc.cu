// k_tc.cu -- w_pos <- w.map(f) with the hidden-to-hidden layer of a two-hidden-layer f on the
// fifth-generation tensor cores (tcgen05): BF16 operands, FP32 accumulation in tensor memory.
//
// Per sub-tile of KPT x 128 keys (KPT keys per thread, 4 warps):
//   layer 1 (1 -> H)  binary32 FFMA, ReLU, rounded to BF16 and stored as the A operand
//                     (128 x H, K-major, no swizzle: 8x8 core matrices of 128 bytes); the split form
//                     stores ReLU(h) truncated to BF16 and the (exact, non-negative) rest rounded to
//                     FP16 as a second A tile, multiplied by an FP16 copy of W2;
//   layer 2 (H -> H)  tcgen05.mma.kind::f16, M = 128, N = H, K = H in steps of 16, issued by one
//                     thread; B = W2 (H x H, K-major) staged once per block; D in TMEM (the split
//                     form accumulates A_hi W2^T + A_lo W2^T into the same D);
//                     b2 enters the same accumulator as one more K-step (a constant slab of ones
//                     times b2 split exactly into three BF16 parts);
//   epilogue          tcgen05.ld (thread t reads TMEM lane t = its key's row), ReLU, output layer
//                     in binary32 FFMA, position rounding as in the binary32 path.
// The MMA completion is signalled through an mbarrier that the issuing thread waits on (the
// others wait in a barrier behind it); the wait gives up after a time limit (the kernel then raises
// ERR_TIMEOUT, still frees its tensor memory and returns).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"
#include "tc05.cuh"

namespace nns {
static inline cudaError_t nns_launched(cudaError_t e, int k = 1) {
    if (e == cudaSuccess) note_launch(k);
    return e;
}

namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_M = 128;

using namespace tc05;

// The second layer's bias enters the MMA as one more K-step of 16: a constant A slab whose first
// three columns are 1 (every row) and a B slab whose first three columns hold b2 split exactly into
// three BF16 parts (hi = b2 truncated to 8 significant bits, mid and lo the truncated rests), so
// D = [1 1 1 0 ..] [b2_hi b2_mid b2_lo 0 ..]^T + A W2^T with b2 carried to binary32 precision.
// Both slabs use the canonical K-major layout of a 16-wide K block (two 8x8 core matrices along K,
// LBO = 128 bytes; 8-row groups SBO = 256 bytes apart).
constexpr uint32_t SLAB_LBO = 128, SLAB_SBO = 256;
__device__ __forceinline__ uint32_t slab_off(int row, int k) {
    return (uint32_t)(row / 8) * SLAB_SBO + (uint32_t)(k / 8) * SLAB_LBO + (uint32_t)(row % 8) * 16 +
           (uint32_t)(k % 8) * 2;
}
__device__ __forceinline__ float bf16_trunc(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFF0000u); }
// ones: TC_M x 16; bias: H x 16 (row = output unit)
template <int H>
__device__ __forceinline__ void fill_bias_slabs(unsigned char *ones, unsigned char *bias, const float *b2,
                                                int tid, int nthreads) {
    for (int e = tid; e < TC_M * 16; e += nthreads) {
        const int r = e / 16, k = e % 16;
        *reinterpret_cast<__nv_bfloat16 *>(ones + slab_off(r, k)) = __float2bfloat16_rn(k < 3 ? 1.0f : 0.0f);
    }
    for (int e = tid; e < H * 16; e += nthreads) {
        const int r = e / 16, k = e % 16;
        const float v = b2[r];
        const float hi = bf16_trunc(v), mid = bf16_trunc(v - hi), lo = (v - hi) - mid;
        const float piece = k == 0 ? hi : (k == 1 ? mid : (k == 2 ? lo : 0.0f));
        *reinterpret_cast<__nv_bfloat16 *>(bias + slab_off(r, k)) = __float2bfloat16_rn(piece);
    }
}

__device__ __forceinline__ int seg_of_tile_tc(const Seg *segs, int nseg, uint32_t tile) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].tbase <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace

// A block of 128 threads walks sub-tiles of KPT * 128 keys (thread t handles keys t, t + 128, ...);
// the predict tile map (tbase, ntiles) is in units of PRED_TILE keys. Key group g of a sub-tile has
// its own A tile(s) and its own accumulator (TMEM columns [g H, (g+1) H)), so every parameter
// loaded from shared memory serves KPT keys. Parameters are read as float4 (broadcast).
__host__ __device__ constexpr int tc_ncol(int H, int KPT) {
    return KPT * H <= 32 ? 32 : (KPT * H <= 64 ? 64 : (KPT * H <= 128 ? 128 : 256));
}
template <int H, bool SPLIT, int KPT>
__host__ __device__ constexpr size_t tc_smem_bytes() {
    return (size_t)KPT * (SPLIT ? 2 : 1) * TC_M * H * 2 + (size_t)(SPLIT ? 2 : 1) * H * H * 2 +
           (size_t)TC_M * 16 * 2 + (size_t)H * 16 * 2 + (size_t)(4 * H + 4) * 4;
}

template <int H, typename W, bool SPLIT, int KPT>
__global__ void __launch_bounds__(TC_THREADS) k_predict_bf16(PredictArgs a) {
    static_assert(H == 16 || H == 32 || H == 64, "tensor path widths");
    static_assert(PRED_TILE % (KPT * TC_M) == 0, "sub-tiles tile the predict tile");
    constexpr int NT = SPLIT ? 2 : 1;          // A tiles per key group: hi (and lo)
    constexpr uint32_t TILE_B = TC_M * H * 2;  // bytes of one 128 x H BF16 tile
    constexpr int NCOL = tc_ncol(H, KPT);
    constexpr uint32_t LBO = 128;              // next core matrix along K
    constexpr uint32_t SBO = (H / 8) * 128;    // next 8-row group
    constexpr int SUB = KPT * TC_M;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sB = sm + KPT * NT * TILE_B;                       // H x H bf16
    unsigned char *sB16 = sB + H * H * 2;                             // H x H fp16 (split form)
    unsigned char *sOnes = sB + (SPLIT ? 2 : 1) * H * H * 2;          // TC_M x 16 bf16
    unsigned char *sBias = sOnes + TC_M * 16 * 2;                     // H x 16 bf16
    float *pf = reinterpret_cast<float *>(sBias + H * 16 * 2);      // W1 | b1 | b2 | W3 | b3
    const float4 *pv = reinterpret_cast<const float4 *>(pf);
    __shared__ __align__(8) unsigned long long bar;
    __shared__ uint32_t tmem_base;
    __shared__ int sh_seg;

    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tmem_alloc<NCOL>(smem_u32(&tmem_base));
    if (tid == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base;
    const uint32_t idesc = idesc_bf16(TC_M, H);
    const uint32_t idesc_lo = idesc_f16(TC_M, H);
    uint32_t phase = 0;
    uint32_t err = 0;
    bool dead = false;  // set once a wait gave up: no further MMAs are issued
    uint32_t dead_parity = 0;
    int loaded = -1;
    const uint32_t sub_per_tile = PRED_TILE / SUB;
    const uint64_t total = (uint64_t)a.total_tiles * sub_per_tile;
    const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
    const uint32_t aoff = (tid / 8) * SBO + (tid % 8) * 16;  // this thread's row in an A tile
    // the next sub-tile's keys are loaded while this one is computed (when it lies in the same array)
    uint64_t pre[KPT];
    uint64_t pre_st = ~0ull;

    for (uint64_t st = blockIdx.x; st < total; st += gridDim.x) {
        const uint32_t tile = (uint32_t)(st / sub_per_tile), sub = (uint32_t)(st % sub_per_tile);
        __syncthreads();
        if (tid == 0) sh_seg = seg_of_tile_tc(a.segs, a.nseg, tile);
        __syncthreads();
        const int si = sh_seg;
        const Seg &sg = a.segs[si];
        const uint64_t n = sg.n;
        const uint64_t r0 = (uint64_t)(tile - sg.tbase) * PRED_TILE + (uint64_t)sub * SUB;
        if (r0 >= n) continue;  // whole sub-tile past the end of its array
        const bool model = sg.slots == nullptr;
        if (model && si != loaded) {
            // W2 (row k = output unit, K = input unit j) -> bf16 canonical K-major layout
            const float *W2 = sg.params + 2 * H;
            for (int e = tid; e < H * H; e += TC_THREADS) {
                const int nrow = e / H, k = e % H;
                const uint32_t off = (nrow / 8) * SBO + (k / 8) * LBO + (nrow % 8) * 16 + (k % 8) * 2;
                *reinterpret_cast<__nv_bfloat16 *>(sB + off) = __float2bfloat16_rn(W2[e]);
                if (SPLIT) *reinterpret_cast<__half *>(sB16 + off) = __float2half_rn(W2[e]);
            }
            for (int e = tid; e < H; e += TC_THREADS) {
                pf[e] = sg.params[e];                          // W1
                pf[H + e] = sg.params[H + e];                  // b1
                pf[2 * H + e] = sg.params[2 * H + H * H + e];  // b2
                pf[3 * H + e] = sg.params[3 * H + H * H + e];  // W3
            }
            if (tid == 0) pf[4 * H] = sg.params[4 * H + H * H];  // b3
            fill_bias_slabs<H>(sOnes, sBias, sg.params + 2 * H + H * H, tid, TC_THREADS);
            loaded = si;
            fence_async_smem();
            __syncthreads();
        }
        const W *keys = reinterpret_cast<const W *>(sg.keys);
        uint64_t wv[KPT];
        bool valid[KPT];
#pragma unroll
        for (int g = 0; g < KPT; ++g) {
            const uint64_t i = r0 + (uint64_t)g * TC_M + tid;
            valid[g] = i < n;
            wv[g] = !valid[g] ? 0ull : (pre_st == st ? pre[g] : word64(keys[i]));
            if (valid[g] && key_is_nan(wv[g], a.dtype)) err |= ERR_NAN;
        }
        {
            const uint64_t st2 = st + gridDim.x;
            const uint32_t tile2 = (uint32_t)(st2 / sub_per_tile), sub2 = (uint32_t)(st2 % sub_per_tile);
            if (st2 < total && tile2 < sg.tbase + sg.ntiles) {
                const uint64_t q0 = (uint64_t)(tile2 - sg.tbase) * PRED_TILE + (uint64_t)sub2 * SUB;
#pragma unroll
                for (int g = 0; g < KPT; ++g) {
                    const uint64_t i = q0 + (uint64_t)g * TC_M + tid;
                    pre[g] = i < n ? word64(keys[i]) : 0ull;
                }
                pre_st = st2;
            }
        }
        float y[KPT];
        uint32_t slot[KPT];
#pragma unroll
        for (int g = 0; g < KPT; ++g) { y[g] = 0.0f; slot[g] = 0; }
        if (model) {
            float x[KPT];
#pragma unroll
            for (int g = 0; g < KPT; ++g) x[g] = valid[g] ? translate_x(wv[g], sg.norm) : 0.0f;
            // layer 1 -> row `tid` of key group g's A tile(s)
#pragma unroll
            for (int j0 = 0; j0 < H; j0 += 8) {
                const float4 wa = pv[j0 / 4], wb = pv[j0 / 4 + 1];
                const float4 ba = pv[H / 4 + j0 / 4], bb = pv[H / 4 + j0 / 4 + 1];
                const float w8[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
                const float b8[8] = {ba.x, ba.y, ba.z, ba.w, bb.x, bb.y, bb.z, bb.w};
#pragma unroll
                for (int g = 0; g < KPT; ++g) {
                    uint32_t hi[4], lo[4];
                    const unsigned long long xx = pk2(x[g], x[g]);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        // pre-activations of units 2q, 2q+1 in one packed FMA; the conversions apply
                        // the ReLU (negative results become 0)
                        const unsigned long long hh =
                            fma2_rn(pk2(w8[2 * q], w8[2 * q + 1]), xx, pk2(b8[2 * q], b8[2 * q + 1]));
                        float h0, h1;
                        upk2(hh, h0, h1);
                        if (!SPLIT) {
                            hi[q] = cvt_bf16x2_rn_relu(h0, h1);  // RN(ReLU(h))
                        } else {
                            // ReLU(h) = hi + lo: hi = ReLU(h) truncated to BF16 (8 significant bits),
                            // lo = the rest (non-negative, exact in binary32) rounded to FP16 (11
                            // bits); for h <= 0 both parts are 0
                            hi[q] = cvt_bf16x2_rz_relu(h0, h1);
                            const unsigned long long tr =
                                pk2(__uint_as_float(__float_as_uint(h0) & 0xFFFF0000u),
                                    __uint_as_float(__float_as_uint(h1) & 0xFFFF0000u));
                            float r0, r1;
                            upk2(sub2_rn(hh, tr), r0, r1);
                            lo[q] = cvt_f16x2_rn_relu(r0, r1);
                        }
                    }
                    unsigned char *t0 = sm + (g * NT) * TILE_B + aoff + (j0 / 8) * LBO;
                    *reinterpret_cast<uint4 *>(t0) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    if (SPLIT) *reinterpret_cast<uint4 *>(t0 + TILE_B) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0 && !dead) {
                const uint32_t b0 = smem_u32(sB);
#pragma unroll
                for (int g = 0; g < KPT; ++g) {
                    const uint32_t a0 = smem_u32(sm + (g * NT) * TILE_B);
                    // the bias slab first (it starts the accumulator), then A_hi W2^T (and A_lo W2^T)
                    mma_bf16(tbase + g * H, mdesc(smem_u32(sOnes), SLAB_LBO, SLAB_SBO),
                             mdesc(smem_u32(sBias), SLAB_LBO, SLAB_SBO), idesc, 0u);
#pragma unroll
                    for (int ks = 0; ks < H / 16; ++ks)
                        mma_bf16(tbase + g * H, mdesc(a0 + ks * 2 * LBO, LBO, SBO),
                                 mdesc(b0 + ks * 2 * LBO, LBO, SBO), idesc, 1u);
                    if (SPLIT) {
#pragma unroll
                        for (int ks = 0; ks < H / 16; ++ks)
                            mma_bf16(tbase + g * H, mdesc(a0 + TILE_B + ks * 2 * LBO, LBO, SBO),
                                     mdesc(smem_u32(sB16) + ks * 2 * LBO, LBO, SBO), idesc_lo, 1u);
                    }
                }
                mma_commit(smem_u32(&bar));
                // one thread waits for the MMAs; the others sleep in the barrier below
                if (!mbar_wait(smem_u32(&bar), phase)) {
                    dead = true;
                    dead_parity = phase;
                    err |= ERR_TIMEOUT;
                }
                tc_fence_before();
            }
            phase ^= 1u;
            dead = __syncthreads_or(dead);
            tc_fence_after();
            // output layer in two packed partial sums (even and odd hidden units), added at the end
            unsigned long long yy[KPT];
#pragma unroll
            for (int g = 0; g < KPT; ++g) yy[g] = pk2(pf[4 * H], 0.0f);
#pragma unroll
            for (int c0 = 0; c0 < H; c0 += 16) {
                float w3[16];
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float4 wq = pv[3 * H / 4 + c0 / 4 + v];
                    w3[4 * v] = wq.x; w3[4 * v + 1] = wq.y; w3[4 * v + 2] = wq.z; w3[4 * v + 3] = wq.w;
                }
#pragma unroll
                for (int g = 0; g < KPT; ++g) {
                    float acc[16];
                    if (!dead) {
                        tmem_ld16(lane_addr + g * H + c0, acc);
                        tmem_wait_ld();
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
                    }
#pragma unroll
                    for (int q = 0; q < 16; q += 2)
                        yy[g] = fma2_rn(pk2(w3[q], w3[q + 1]), pk2(relu_f(acc[q]), relu_f(acc[q + 1])), yy[g]);
                }
            }
#pragma unroll
            for (int g = 0; g < KPT; ++g) {
                float ye, yo;
                upk2(yy[g], ye, yo);
                y[g] = __fadd_rn(ye, yo);
                slot[g] = slot_of(y[g], sg.nm_hi, sg.nm_lo, sg.L);
            }
            tc_fence_before();
        } else {
#pragma unroll
            for (int g = 0; g < KPT; ++g) {
                if (!valid[g]) continue;
                slot[g] = sg.slots[r0 + (uint64_t)g * TC_M + tid];
                if ((uint64_t)slot[g] >= sg.L) { err |= ERR_SLOT; slot[g] = 0; }
            }
        }
#pragma unroll
        for (int g = 0; g < KPT; ++g) {
            if (!valid[g]) continue;
            const uint64_t i = r0 + (uint64_t)g * TC_M + tid;
            const uint64_t e = sg.ebase + i;
            const uint32_t gpos = (uint32_t)(sg.gs_base + slot[g]);
            if (a.gs) a.gs[e] = gpos;
            if (a.key_copy) reinterpret_cast<W *>(a.key_copy)[e] = (W)wv[g];
            if (a.pay_copy && sg.payload) a.pay_copy[e] = (uint32_t)sg.payload[i];
            if (a.row_init) a.row_init[e] = (uint32_t)i;
            if (a.slots_out) a.slots_out[e] = slot[g];
            if (a.y_out) a.y_out[e] = y[g];
        }
    }
    if (err) atomicOr(a.err, err);
    // an MMA whose completion was not seen may still be running: wait for it (bounded) before the
    // tensor memory it writes is released
    if (dead && tid == 0) mbar_wait(smem_u32(&bar), dead_parity);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free<NCOL>(tbase);
}

// ---------------------------------------------------------------------------------------------
// One array, one model: NG independent groups of 4 warps per block and one block per SM. Group g
// has its own A tile(s), accumulator columns [g H, (g + 1) H), mbarrier and named barrier (1 + g)
// and walks its own sub-tiles of 128 keys; the B tile(s) and the parameters are staged once per
// block and shared. The A tiles are then the only per-group shared memory, so NG = 6 groups fit
// on an SM (24 warps, against 16 for blocks that each hold a W2 copy), and no block-wide barrier
// separates one sub-tile from the next.
constexpr int TC_NG = 6;

__device__ __forceinline__ void grp_sync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(TC_THREADS) : "memory");
}
// OR of v over the 128 threads of named barrier id (a barrier as well)
__device__ __forceinline__ bool grp_or(int id, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "n"(TC_THREADS)
        : "memory");
    return r != 0;
}

// the first and last layers' parameters as launch constants: every thread reads them through the
// constant cache (one broadcast per warp instruction, no shared-memory traffic)
struct TcConst {
    float w1[64], b1[64], w3[64], b3;
};

template <int H, bool SPLIT, int NG>
__host__ __device__ constexpr size_t tcmg_smem_bytes() {
    return (size_t)NG * (SPLIT ? 2 : 1) * TC_M * H * 2 + (size_t)(SPLIT ? 2 : 1) * H * H * 2 +
           (size_t)TC_M * 16 * 2 + (size_t)H * 16 * 2 + (size_t)(4 * H + 4) * 4;
}

template <int H, typename W, bool SPLIT, int NG>
__global__ void __launch_bounds__(NG * TC_THREADS, 1) k_predict_bf16_mg(PredictArgs a, const TcConst cst) {
    static_assert(H == 16 || H == 32 || H == 64, "tensor path widths");
    static_assert(NG * H <= 512, "accumulators fit in tensor memory");
    constexpr int NT = SPLIT ? 2 : 1;
    constexpr uint32_t TILE_B = TC_M * H * 2;
    constexpr uint32_t LBO = 128;
    constexpr uint32_t SBO = (H / 8) * 128;
    constexpr int NCOL = NG * H <= 128 ? 128 : (NG * H <= 256 ? 256 : 512);
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sB = sm + NG * NT * TILE_B;
    unsigned char *sB16 = sB + H * H * 2;
    unsigned char *sOnes = sB + NT * H * H * 2;                       // TC_M x 16 bf16
    unsigned char *sBias = sOnes + TC_M * 16 * 2;                     // H x 16 bf16
    __shared__ __align__(8) unsigned long long bar[NG];
    __shared__ uint32_t tmem_base;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int grp = tid / TC_THREADS, gt = tid % TC_THREADS;
    if (warp == 0) tmem_alloc<NCOL>(smem_u32(&tmem_base));
    if (tid == 0) {
        for (int g = 0; g < NG; ++g) mbar_init(smem_u32(&bar[g]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const Seg &sg = a.segs[0];
    {   // W2 (row = output unit, K = input unit) -> canonical K-major layout; bias slabs
        const float *W2 = sg.params + 2 * H;
        for (int e = tid; e < H * H; e += NG * TC_THREADS) {
            const int nrow = e / H, k = e % H;
            const uint32_t off = (nrow / 8) * SBO + (k / 8) * LBO + (nrow % 8) * 16 + (k % 8) * 2;
            *reinterpret_cast<__nv_bfloat16 *>(sB + off) = __float2bfloat16_rn(W2[e]);
            if (SPLIT) *reinterpret_cast<__half *>(sB16 + off) = __float2half_rn(W2[e]);
        }
        fill_bias_slabs<H>(sOnes, sBias, sg.params + 2 * H + H * H, tid, NG * TC_THREADS);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base;
    const uint32_t dcol = tbase + (uint32_t)(grp * H);
    const uint32_t lane_addr = dcol + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t aoff = (gt / 8) * SBO + (gt % 8) * 16;
    unsigned char *myA = sm + grp * NT * TILE_B;
    const uint32_t mybar = smem_u32(&bar[grp]);
    const int bid = 1 + grp;
    const uint32_t idesc = idesc_bf16(TC_M, H);
    const uint32_t idesc_lo = idesc_f16(TC_M, H);
    uint32_t phase = 0, err = 0, dead_parity = 0;
    bool dead = false;
    const uint64_t n = sg.n;
    const uint64_t total = (n + TC_M - 1) / TC_M;
    const uint64_t stride = (uint64_t)gridDim.x * NG;
    const W *keys = reinterpret_cast<const W *>(sg.keys);
    uint64_t pre = 0, pre_st = ~0ull;
    for (uint64_t st = (uint64_t)blockIdx.x * NG + grp; st < total; st += stride) {
        const uint64_t i = st * TC_M + gt;
        const bool valid = i < n;
        const uint64_t wv = !valid ? 0ull : (pre_st == st ? pre : word64(keys[i]));
        if (valid && key_is_nan(wv, a.dtype)) err |= ERR_NAN;
        {   // the group's next sub-tile's keys, loaded while this one is computed
            const uint64_t st2 = st + stride;
            if (st2 < total) {
                const uint64_t i2 = st2 * TC_M + gt;
                pre = i2 < n ? word64(keys[i2]) : 0ull;
                pre_st = st2;
            }
        }
        const float x = valid ? translate_x(wv, sg.norm) : 0.0f;
        const unsigned long long xx = pk2(x, x);
#pragma unroll
        for (int j0 = 0; j0 < H; j0 += 8) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = j0 + 2 * q;
                const unsigned long long hh =
                    fma2_rn(pk2(cst.w1[j], cst.w1[j + 1]), xx, pk2(cst.b1[j], cst.b1[j + 1]));
                float h0, h1;
                upk2(hh, h0, h1);
                if (!SPLIT) {
                    hi[q] = cvt_bf16x2_rn_relu(h0, h1);
                } else {
                    hi[q] = cvt_bf16x2_rz_relu(h0, h1);
                    const unsigned long long tr = pk2(__uint_as_float(__float_as_uint(h0) & 0xFFFF0000u),
                                                      __uint_as_float(__float_as_uint(h1) & 0xFFFF0000u));
                    float r0, r1;
                    upk2(sub2_rn(hh, tr), r0, r1);
                    lo[q] = cvt_f16x2_rn_relu(r0, r1);
                }
            }
            unsigned char *t0 = myA + aoff + (j0 / 8) * LBO;
            *reinterpret_cast<uint4 *>(t0) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            if (SPLIT) *reinterpret_cast<uint4 *>(t0 + TILE_B) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        fence_async_smem();
        tc_fence_before();
        grp_sync(bid);
        tc_fence_after();
        if (gt == 0 && !dead) {
            const uint32_t a0 = smem_u32(myA), b0 = smem_u32(sB);
            // the bias slab first (it starts the accumulator), then A_hi W2^T (and A_lo W2^T)
            mma_bf16(dcol, mdesc(smem_u32(sOnes), SLAB_LBO, SLAB_SBO), mdesc(smem_u32(sBias), SLAB_LBO, SLAB_SBO),
                     idesc, 0u);
#pragma unroll
            for (int ks = 0; ks < H / 16; ++ks)
                mma_bf16(dcol, mdesc(a0 + ks * 2 * LBO, LBO, SBO), mdesc(b0 + ks * 2 * LBO, LBO, SBO), idesc, 1u);
            if (SPLIT) {
#pragma unroll
                for (int ks = 0; ks < H / 16; ++ks)
                    mma_bf16(dcol, mdesc(a0 + TILE_B + ks * 2 * LBO, LBO, SBO),
                             mdesc(smem_u32(sB16) + ks * 2 * LBO, LBO, SBO), idesc_lo, 1u);
            }
            mma_commit(mybar);
            // one thread of the group waits for the MMAs; the others sleep in the barrier below
            if (!mbar_wait(mybar, phase)) {
                dead = true;
                dead_parity = phase;
                err |= ERR_TIMEOUT;
            }
            tc_fence_before();
        }
        phase ^= 1u;
        dead = grp_or(bid, dead);
        tc_fence_after();
        unsigned long long yy = pk2(cst.b3, 0.0f);
#pragma unroll
        for (int c0 = 0; c0 < H; c0 += 16) {
            float acc[16];
            if (!dead) {
                tmem_ld16(lane_addr + c0, acc);
                tmem_wait_ld();
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 16; q += 2)
                yy = fma2_rn(pk2(cst.w3[c0 + q], cst.w3[c0 + q + 1]), pk2(relu_f(acc[q]), relu_f(acc[q + 1])), yy);
        }
        tc_fence_before();
        if (!valid) continue;
        float ye, yo;
        upk2(yy, ye, yo);
        const float y = __fadd_rn(ye, yo);
        const uint32_t slot = slot_of(y, sg.nm_hi, sg.nm_lo, sg.L);
        const uint64_t e = sg.ebase + i;
        const uint32_t gpos = (uint32_t)(sg.gs_base + slot);
        if (a.gs) a.gs[e] = gpos;
        if (a.key_copy) reinterpret_cast<W *>(a.key_copy)[e] = (W)wv;
        if (a.pay_copy && sg.payload) a.pay_copy[e] = (uint32_t)sg.payload[i];
        if (a.row_init) a.row_init[e] = (uint32_t)i;
        if (a.slots_out) a.slots_out[e] = slot;
        if (a.y_out) a.y_out[e] = y;
    }
    if (err) atomicOr(a.err, err);
    // an MMA whose completion was not seen may still be running: wait for it (bounded) before the
    // tensor memory it writes is released
    if (dead && gt == 0) mbar_wait(mybar, dead_parity);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free<NCOL>(tbase);
}

template <int H, bool SPLIT>
static cudaError_t bf16_mg_go(const PredictArgs &p, int sms, cudaStream_t s) {
    // padded layout: W1[H] b1[H] W2[H * H] b2[H] W3[H] b3
    TcConst c{};
    for (int j = 0; j < H; ++j) {
        c.w1[j] = p.host_pad[j];
        c.b1[j] = p.host_pad[H + j];
        c.w3[j] = p.host_pad[3 * H + H * H + j];
    }
    c.b3 = p.host_pad[4 * H + H * H];
    const uint64_t n_sub = (uint64_t)p.total_tiles * (PRED_TILE / TC_M);
    const size_t smem = tcmg_smem_bytes<H, SPLIT, TC_NG>();
    const int grid = (int)std::min<uint64_t>((n_sub + TC_NG - 1) / TC_NG, (uint64_t)sms);
    if (grid == 0) return cudaSuccess;
    auto k4 = k_predict_bf16_mg<H, uint32_t, SPLIT, TC_NG>;
    auto k8 = k_predict_bf16_mg<H, uint64_t, SPLIT, TC_NG>;
    cudaError_t e = cudaFuncSetAttribute(p.key_bytes == 4 ? k4 : k8,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (p.key_bytes == 4) k4<<<grid, TC_NG * TC_THREADS, smem, s>>>(p, c);
    else k8<<<grid, TC_NG * TC_THREADS, smem, s>>>(p, c);
    return nns_launched(cudaGetLastError());
}

template <int H, bool SPLIT, int KPT>
static cudaError_t bf16_go(const PredictArgs &p, int sms, cudaStream_t s) {
    const uint64_t subtiles = (uint64_t)p.total_tiles * (PRED_TILE / (KPT * TC_M));
    // resident blocks per SM: bounded by tensor memory (512 columns) and by shared memory (228 KB,
    // 1 KB reserved per block); the request is raised so that shared memory never admits more
    // blocks than tensor memory can serve (a block waiting in tcgen05.alloc would hold its slot)
    constexpr int NCOL = tc_ncol(H, KPT);
    const int by_tmem = std::min(512 / NCOL, 2048 / TC_THREADS);
    size_t smem = tc_smem_bytes<H, SPLIT, KPT>();
    const size_t floor_req = (size_t)(228 * 1024) / (size_t)(by_tmem + 1) - 1024 + 64;
    smem = std::max(smem, floor_req);
    const int by_smem = (int)((size_t)(228 * 1024) / (smem + 1024));
    const int per_sm = std::max(1, std::min(by_tmem, by_smem));
    const int grid = (int)std::min<uint64_t>(subtiles, (uint64_t)sms * per_sm);
    if (grid == 0) return cudaSuccess;
    auto k4 = k_predict_bf16<H, uint32_t, SPLIT, KPT>;
    auto k8 = k_predict_bf16<H, uint64_t, SPLIT, KPT>;
    cudaError_t e = cudaFuncSetAttribute(p.key_bytes == 4 ? k4 : k8,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (p.key_bytes == 4) k4<<<grid, TC_THREADS, smem, s>>>(p);
    else k8<<<grid, TC_THREADS, smem, s>>>(p);
    return nns_launched(cudaGetLastError());
}

// keys per thread per sub-tile: two for the plain form (parameter reads shared by two keys, 4 blocks
// per SM); one for the split form, whose second A tile would otherwise halve the resident blocks
// (measured at 2^28 keys, H = 64: split 12.1 ms at one key vs 15.9 ms at two; plain 8.1 vs 8.3 ms)
constexpr int TC_KPT = 2, TC_KPT_SPLIT = 1;

cudaError_t launch_predict_bf16(const PadArch &a, const PredictArgs &p, bool split, int sms, cudaStream_t s) {
    if (a.layers != 2) return cudaErrorNotSupported;
    if (p.nseg == 1 && p.single_model && p.host_pad) {
        switch (a.h1) {
        case 16: return split ? bf16_mg_go<16, true>(p, sms, s) : bf16_mg_go<16, false>(p, sms, s);
        case 32: return split ? bf16_mg_go<32, true>(p, sms, s) : bf16_mg_go<32, false>(p, sms, s);
        case 64: return split ? bf16_mg_go<64, true>(p, sms, s) : bf16_mg_go<64, false>(p, sms, s);
        }
    }
    switch (a.h1) {
    case 16: return split ? bf16_go<16, true, TC_KPT_SPLIT>(p, sms, s) : bf16_go<16, false, TC_KPT>(p, sms, s);
    case 32: return split ? bf16_go<32, true, TC_KPT_SPLIT>(p, sms, s) : bf16_go<32, false, TC_KPT>(p, sms, s);
    case 64: return split ? bf16_go<64, true, TC_KPT_SPLIT>(p, sms, s) : bf16_go<64, false, TC_KPT>(p, sms, s);
    }
    return cudaErrorNotSupported;  // widths below 16 stay on the binary32 path
}

}  // namespace nns
