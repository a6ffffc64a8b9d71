// k_tc.cu -- w_pos <- w.map(f) with the hidden-to-hidden layer of a two-hidden-layer f on the
// fifth-generation tensor cores (tcgen05): BF16 operands, FP32 accumulation in tensor memory.
//
// Per tile of 128 keys (one key per thread, 4 warps):
//   layer 1 (1 -> H)  binary32 FFMA, ReLU, rounded to BF16 and stored as the A operand
//                     (128 x H, K-major, no swizzle: 8x8 core matrices of 128 bytes); with the
//                     split form also the rounding residual, rounded to BF16, as a second A tile;
//   layer 2 (H -> H)  tcgen05.mma.kind::f16, M = 128, N = H, K = H in steps of 16, issued by one
//                     thread; B = W2 (H x H, K-major) staged once per block; D in TMEM (the split
//                     form accumulates A_hi W2^T + A_lo W2^T into the same D);
//   epilogue          tcgen05.ld (thread t reads TMEM lane t = its key's row), + b2, ReLU, output
//                     layer in binary32 FFMA, position rounding as in the binary32 path.
// The MMA completion is signalled through an mbarrier whose wait gives up after a time limit
// (the kernel then raises ERR_TIMEOUT, still frees its tensor memory and returns).
#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"

namespace nns {
static inline cudaError_t nns_launched(cudaError_t e, int k = 1) {
    if (e == cudaSuccess) note_launch(k);
    return e;
}

namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_M = 128;
constexpr size_t TC_SMEM = 32 * 1024;  // also caps residency at 7 blocks per SM (TMEM: 7 x 64 <= 512 columns)
constexpr size_t TC_SMEM_SPLIT = 48 * 1024;  // second A tile; 4 blocks per SM

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle, K-major:
// start >> 4 in [0,14), leading-dimension byte offset >> 4 in [16,30), stride-dimension byte offset
// >> 4 in [32,46), descriptor version 1 in [46,48), base offset 0, layout SWIZZLE_NONE (0) in [61,64)
__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = BF16 (bits 7-9 = 1),
// B = BF16 (bits 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in bits 24-28
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false when the limit expired
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = globaltimer_ns();
    while (!mbar_try(bar, parity)) {
        if (globaltimer_ns() - t0 > SPIN_LIMIT_NS) return false;
    }
    return true;
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <int NCOL> __device__ __forceinline__ void tmem_alloc(uint32_t dst_smem) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
                 "n"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
template <int NCOL> __device__ __forceinline__ void tmem_free(uint32_t taddr) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(NCOL) : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ int seg_of_tile_tc(const Seg *segs, int nseg, uint32_t tile) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].tbase <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace

// Tiles here are 128 keys; the predict tile map (tbase, ntiles) is in units of PRED_TILE keys, so
// a block walks PRED_TILE / 128 sub-tiles of each predict tile.
template <int H, typename W, bool SPLIT>
__global__ void __launch_bounds__(TC_THREADS) k_predict_bf16(PredictArgs a) {
    static_assert(H == 16 || H == 32 || H == 64, "tensor path widths");
    constexpr int NCOL = H < 32 ? 32 : H;
    constexpr uint32_t LBO = 128;              // next core matrix along K
    constexpr uint32_t SBO_A = (H / 8) * 128;  // next 8-row group
    constexpr uint32_t SBO_B = (H / 8) * 128;
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char *sA = sm;                          // 128 x H bf16
    unsigned char *sA2 = sA + TC_M * H * 2;          // 128 x H bf16 residuals (split form)
    unsigned char *sB = sA + (SPLIT ? 2 : 1) * TC_M * H * 2;  // H x H bf16
    float *sP = reinterpret_cast<float *>(sB + H * H * 2);  // W1 b1 b2 W3 b3
    __shared__ __align__(8) unsigned long long bar;
    __shared__ uint32_t tmem_base;
    __shared__ int sh_seg;
    __shared__ uint32_t sh_hist[MAX_PASSES * RADIX_BINS];

    const int tid = threadIdx.x, warp = tid >> 5;
    const int npass = a.hist ? a.plan.npass : 0;
    for (int i = tid; i < npass * RADIX_BINS; i += TC_THREADS) sh_hist[i] = 0;
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
    uint32_t phase = 0;
    uint32_t err = 0;
    bool dead = false;  // set once a wait gave up: no further MMAs are issued
    uint32_t dead_parity = 0;
    int loaded = -1;
    const uint32_t sub_per_tile = PRED_TILE / TC_M;
    const uint64_t total = (uint64_t)a.total_tiles * sub_per_tile;

    for (uint64_t st = blockIdx.x; st < total; st += gridDim.x) {
        const uint32_t tile = (uint32_t)(st / sub_per_tile), sub = (uint32_t)(st % sub_per_tile);
        __syncthreads();
        if (tid == 0) sh_seg = seg_of_tile_tc(a.segs, a.nseg, tile);
        __syncthreads();
        const int si = sh_seg;
        const Seg &sg = a.segs[si];
        const uint64_t n = sg.n;
        const uint64_t i = (uint64_t)(tile - sg.tbase) * PRED_TILE + (uint64_t)sub * TC_M + tid;
        if ((uint64_t)(tile - sg.tbase) * PRED_TILE + (uint64_t)sub * TC_M >= n) continue;  // whole sub-tile past the end
        const bool model = sg.slots == nullptr;
        if (model && si != loaded) {
            // W2 (row k = output unit, K = input unit j) -> bf16 canonical K-major layout
            const float *W2 = sg.params + 2 * H;
            for (int e = tid; e < H * H; e += TC_THREADS) {
                const int nrow = e / H, k = e % H;
                const uint32_t off = (nrow / 8) * SBO_B + (k / 8) * LBO + (nrow % 8) * 16 + (k % 8) * 2;
                *reinterpret_cast<__nv_bfloat16 *>(sB + off) = __float2bfloat16_rn(W2[e]);
            }
            for (int e = tid; e < H; e += TC_THREADS) {
                sP[e] = sg.params[e];                          // W1
                sP[H + e] = sg.params[H + e];                  // b1
                sP[2 * H + e] = sg.params[2 * H + H * H + e];  // b2
                sP[3 * H + e] = sg.params[3 * H + H * H + e];  // W3
            }
            if (tid == 0) sP[4 * H] = sg.params[4 * H + H * H];  // b3
            loaded = si;
            fence_async_smem();
            __syncthreads();
        }
        const bool valid = i < n;
        const W *keys = reinterpret_cast<const W *>(sg.keys);
        const uint64_t w = valid ? word64(keys[i]) : 0ull;
        if (valid && key_is_nan(w, a.dtype)) err |= ERR_NAN;
        float y = 0.0f;
        uint32_t slot = 0;
        if (model) {
            const float x = valid ? translate_x(w, sg.norm) : 0.0f;
            // layer 1 -> A row `tid`
#pragma unroll
            for (int j0 = 0; j0 < H; j0 += 8) {
                __align__(16) __nv_bfloat16 hb[8];
                __align__(16) __nv_bfloat16 lb[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float h = relu_f(__fmaf_rn(sP[j0 + q], x, sP[H + j0 + q]));
                    hb[q] = __float2bfloat16_rn(h);
                    if (SPLIT) lb[q] = __float2bfloat16_rn(__fsub_rn(h, __bfloat162float(hb[q])));
                }
                const uint32_t off = (tid / 8) * SBO_A + (j0 / 8) * LBO + (tid % 8) * 16;
                *reinterpret_cast<uint4 *>(sA + off) = *reinterpret_cast<const uint4 *>(hb);
                if (SPLIT) *reinterpret_cast<uint4 *>(sA2 + off) = *reinterpret_cast<const uint4 *>(lb);
            }
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0 && !dead) {
                const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
                for (int ks = 0; ks < H / 16; ++ks)
                    mma_bf16(tbase, mdesc(a0 + ks * 2 * LBO, LBO, SBO_A), mdesc(b0 + ks * 2 * LBO, LBO, SBO_B),
                             idesc, ks > 0 ? 1u : 0u);
                if (SPLIT) {
                    const uint32_t a1 = smem_u32(sA2);
#pragma unroll
                    for (int ks = 0; ks < H / 16; ++ks)
                        mma_bf16(tbase, mdesc(a1 + ks * 2 * LBO, LBO, SBO_A),
                                 mdesc(b0 + ks * 2 * LBO, LBO, SBO_B), idesc, 1u);
                }
                mma_commit(smem_u32(&bar));
            }
            if (!dead && !mbar_wait(smem_u32(&bar), phase)) {
                dead = true;
                dead_parity = phase;
                err |= ERR_TIMEOUT;
            }
            phase ^= 1u;
            dead = __syncthreads_or(dead);
            tc_fence_after();
            float acc[16];
            float yy = sP[4 * H];
            const uint32_t lane_addr = tbase + ((uint32_t)(warp * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < H; c0 += 16) {
                if (!dead) {
                    tmem_ld16(lane_addr + c0, acc);
                    tmem_wait_ld();
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) acc[q] = 0.0f;
                }
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    yy = __fmaf_rn(sP[3 * H + c0 + q], relu_f(__fadd_rn(acc[q], sP[2 * H + c0 + q])), yy);
            }
            y = yy;
            slot = slot_of(y, sg.nm_hi, sg.nm_lo, sg.L);
            tc_fence_before();
        } else if (valid) {
            slot = sg.slots[i];
            if ((uint64_t)slot >= sg.L) { err |= ERR_SLOT; slot = 0; }
        }
        if (valid) {
            const uint64_t e = sg.ebase + i;
            const uint32_t g = (uint32_t)(sg.gs_base + slot);
            if (a.gs) a.gs[e] = g;
            if (a.key_copy) reinterpret_cast<W *>(a.key_copy)[e] = (W)w;
            if (a.pay_copy && sg.payload) a.pay_copy[e] = (uint32_t)sg.payload[i];
            if (a.row_init) a.row_init[e] = (uint32_t)i;
            if (a.slots_out) a.slots_out[e] = slot;
            if (a.y_out) a.y_out[e] = y;
#pragma unroll
            for (int p = 0; p < MAX_PASSES; ++p) {
                if (p >= npass) break;
                const uint32_t d = (g >> a.plan.shift[p]) & ((1u << a.plan.bits[p]) - 1u);
                atomicAdd(&sh_hist[p * RADIX_BINS + d], 1u);
            }
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
    for (int i = tid; i < npass * RADIX_BINS; i += TC_THREADS)
        if (sh_hist[i]) atomicAdd(&a.hist[i], sh_hist[i]);
}

template <int H, bool SPLIT>
static cudaError_t bf16_go(const PredictArgs &p, int sms, cudaStream_t s) {
    const uint64_t subtiles = (uint64_t)p.total_tiles * (PRED_TILE / TC_M);
    constexpr size_t smem = SPLIT ? TC_SMEM_SPLIT : TC_SMEM;
    const int grid = (int)std::min<uint64_t>(subtiles, (uint64_t)sms * (SPLIT ? 4 : 7));
    if (grid == 0) return cudaSuccess;
    auto k4 = k_predict_bf16<H, uint32_t, SPLIT>;
    auto k8 = k_predict_bf16<H, uint64_t, SPLIT>;
    cudaError_t e = cudaFuncSetAttribute(p.key_bytes == 4 ? k4 : k8,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (p.key_bytes == 4) k4<<<grid, TC_THREADS, smem, s>>>(p);
    else k8<<<grid, TC_THREADS, smem, s>>>(p);
    return nns_launched(cudaGetLastError());
}

cudaError_t launch_predict_bf16(const PadArch &a, const PredictArgs &p, bool split, int sms, cudaStream_t s) {
    if (a.layers != 2) return cudaErrorNotSupported;
    switch (a.h1) {
    case 16: return split ? bf16_go<16, true>(p, sms, s) : bf16_go<16, false>(p, sms, s);
    case 32: return split ? bf16_go<32, true>(p, sms, s) : bf16_go<32, false>(p, sms, s);
    case 64: return split ? bf16_go<64, true>(p, sms, s) : bf16_go<64, false>(p, sms, s);
    }
    return cudaErrorNotSupported;  // widths below 16 stay on the binary32 path
}

}  // namespace nns
