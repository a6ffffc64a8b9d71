// k_train_block.cu -- training many small models at once (Sec. "Training"), one thread block per
// model, entirely on chip: the block draws its array's sample, sorts it, labels it, initialises the
// network and runs every Adam step without leaving the kernel.
//
// For a model with one hidden layer of at most 32 units and a sample of at most TB_MAX_S keys the
// whole training set fits in shared memory and the gradient is a few hundred numbers, so launching
// two kernels per step over the whole GPU (the path of nnsort_train for large models) would spend
// its time on launches. Here:
//   * sample: S draws with replacement from the SplitMix64 stream (seed, 1), as nnsort_train;
//   * sort: a bitonic sort of the sample's order images in shared memory (equal keys give equal
//     inputs and consecutive labels, so the order among them does not change the training data);
//   * normaliser, inputs and labels: the sample's extremes, x_j = translate(key_j), label_j = j / S;
//   * initial weights: stream (seed, 2) in the same order and binary64 arithmetic as nnsort_train;
//   * each step: every thread runs forward and backward over its samples (full batch, or the
//     minibatch drawn from stream (seed, 3)), keeping its share of the gradient in registers; the
//     shares meet in a fixed shuffle tree and a fixed warp order, then Adam in binary32.
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace nns {
static inline cudaError_t nns_launched(cudaError_t e, int k = 1) {
    if (e == cudaSuccess) note_launch(k);
    return e;
}

namespace {
constexpr int TB_THREADS = 256;
constexpr int TB_WARPS = TB_THREADS / 32;

__device__ __forceinline__ double tb_unit53(uint64_t u) {
    return __dmul_rn((double)(u >> 11), 1.0 / 9007199254740992.0);
}

// the key word whose order image is u (the inverse of ordbits)
__device__ __forceinline__ uint64_t key_of_image(uint64_t u, int dtype) {
    if (dtype == NNSORT_F32) {
        const uint32_t b = (uint32_t)u;
        return (b & 0x80000000u) ? (uint64_t)(b & 0x7FFFFFFFu) : (uint64_t)(uint32_t)~b;
    }
    if (dtype == NNSORT_F64) return (u >> 63) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
    return u;
}
__device__ __forceinline__ double value_of_key(uint64_t w, int dtype) {
    if (dtype == NNSORT_F32) return (double)__uint_as_float((uint32_t)w);
    if (dtype == NNSORT_F64) return __longlong_as_double((long long)w);
    if (dtype == NNSORT_U32) return (double)(uint32_t)w;
    return __ull2double_rn(w);
}

// fixed-order sum of v over the 32 lanes (the result in lane 0)
__device__ __forceinline__ float tb_warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_down_sync(0xFFFFFFFFu, v, o));
    return v;
}
}  // namespace

// the gradient's 3 H + 1 partial sums live in registers: two blocks per SM up to 16 hidden units
template <typename W, int H>
__global__ void __launch_bounds__(TB_THREADS, H >= 32 ? 1 : 2) k_train_block(TrainBlockArgs a) {
    constexpr int P = 3 * H + 1;  // W1[H] b1[H] W3[H] b3 (padded layout of one hidden layer)
    extern __shared__ __align__(16) unsigned long long tb_buf[];  // [cap]: images, then (x, label)
    __shared__ float sp[P], sm_[P], sv[P];
    __shared__ float red[TB_WARPS][P + 1];
    __shared__ Norm nm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t m = a.ids[blockIdx.x];
    const uint64_t n = a.n[m], S = a.S[m];
    const W *keys = reinterpret_cast<const W *>(a.keys[m]);
    const uint64_t seed = a.seed0 + m;
    uint32_t err = 0;

    // sample and its order images; the rest of the buffer sorts last
    const uint64_t ss = rng_draw(seed, 1);
    for (uint32_t i = tid; i < a.cap; i += TB_THREADS) {
        unsigned long long u = ~0ull;
        if (i < S) {
            const uint64_t r = __umul64hi(rng_draw(ss, i), n);
            const uint64_t w = word64(keys[r]);
            if (key_is_nan(w, a.dtype)) err |= ERR_NAN;
            u = ordbits(w, a.dtype);
        }
        tb_buf[i] = u;
    }
    __syncthreads();
    // bitonic sort of the cap images, ascending
    for (uint32_t k = 2; k <= a.cap; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = tid; i < a.cap; i += TB_THREADS) {
                const uint32_t p = i ^ j;
                if (p > i) {
                    const unsigned long long x = tb_buf[i], y = tb_buf[p];
                    if ((x > y) == ((i & k) == 0)) { tb_buf[i] = y; tb_buf[p] = x; }
                }
            }
            __syncthreads();
        }
    }
    // normaliser from the sample's extremes (as nnsort_sample_labels computes it)
    if (tid == 0) {
        const uint64_t lo = tb_buf[0], hi = tb_buf[S - 1];
        Norm q;
        q.dtype = a.dtype;
        q.translate = a.translate;
        q.lo_bits = lo;
        q.lo_val = value_of_key(key_of_image(lo, a.dtype), a.dtype);
        const bool ob = a.translate == NNSORT_TRANSLATE_ORDBITS || a.dtype == NNSORT_U32 || a.dtype == NNSORT_U64;
        if (ob) {
            q.scale = (hi > lo) ? __ddiv_rn(1.0, __ull2double_rn(hi - lo)) : 1.0;
        } else {
            const double hv = value_of_key(key_of_image(hi, a.dtype), a.dtype);
            q.scale = (hv > q.lo_val) ? __ddiv_rn(1.0, __dsub_rn(hv, q.lo_val)) : 1.0;
        }
        q.lo_f = __double2float_rn(q.lo_val);
        q.scale_f = __double2float_rn(q.scale);
        nm = q;
        a.norm_out[m] = q;
        // initial weights: W1_j in (-sqrt 6, sqrt 6), kink c_j in [0, 1) (b1_j = -W1_j c_j),
        // output weights in (-sqrt(6/h1), sqrt(6/h1)), b3 = 0; padding units stay 0
        const uint64_t si = rng_draw(seed, 2);
        uint64_t c = 0;
        const double r1 = __dsqrt_rn(6.0), r3 = __dsqrt_rn(__ddiv_rn(6.0, (double)a.h1));
        for (int u = 0; u < P; ++u) { sp[u] = 0.0f; sm_[u] = 0.0f; sv[u] = 0.0f; }
        for (int j = 0; j < a.h1; ++j)
            sp[j] = __double2float_rn(__dmul_rn(__dsub_rn(__dmul_rn(2.0, tb_unit53(rng_draw(si, c++))), 1.0), r1));
        for (int j = 0; j < a.h1; ++j)
            sp[H + j] = __double2float_rn(__dmul_rn(-(double)sp[j], tb_unit53(rng_draw(si, c++))));
        for (int j = 0; j < a.h1; ++j)
            sp[2 * H + j] = __double2float_rn(__dmul_rn(__dsub_rn(__dmul_rn(2.0, tb_unit53(rng_draw(si, c++))), 1.0), r3));
    }
    __syncthreads();
    // inputs and labels in place of the sorted images
    float2 *xl = reinterpret_cast<float2 *>(tb_buf);
    for (uint32_t j = tid; j < S; j += TB_THREADS) {
        const float x = translate_x(key_of_image(tb_buf[j], a.dtype), nm);
        const float lab = __double2float_rn(__ddiv_rn((double)j, (double)S));
        xl[j] = make_float2(x, lab);  // the same 8 bytes this thread just read
    }
    __syncthreads();

    const uint64_t B = a.batch ? a.batch : S;
    const float inv_n = 1.0f / (float)B;
    const uint64_t bseed = rng_draw(seed, 3);
    for (int step = 0; step < a.steps; ++step) {
        float g[P];
#pragma unroll
        for (int u = 0; u < P; ++u) g[u] = 0.0f;
        float lsum = 0.0f;
        for (uint64_t i = tid; i < B; i += TB_THREADS) {
            const uint64_t src = a.batch ? __umul64hi(rng_draw(bseed, (uint64_t)step * B + i), S) : i;
            const float2 v = xl[src];
            // hidden activations are recomputed in the backward loop rather than kept in registers
            float y = sp[3 * H];
#pragma unroll
            for (int j = 0; j < H; ++j) y = __fmaf_rn(sp[2 * H + j], relu_f(__fmaf_rn(sp[j], v.x, sp[H + j])), y);
            const float r = __fsub_rn(y, v.y);
            float gy, lv;
            if (a.loss == NNSORT_LOSS_HUBER) {
                const float ar = fabsf(r);
                lv = (ar <= a.delta) ? 0.5f * r * r : a.delta * ar - 0.5f * a.delta * a.delta;
                gy = (r > a.delta) ? a.delta : ((r < -a.delta) ? -a.delta : r);
            } else {
                lv = __fmul_rn(r, r);
                gy = __fmul_rn(2.0f, r);
            }
            gy = __fmul_rn(gy, inv_n);
            lsum = __fadd_rn(lsum, lv);
#pragma unroll
            for (int j = 0; j < H; ++j) {
                const float h = relu_f(__fmaf_rn(sp[j], v.x, sp[H + j]));
                const float d1 = (h > 0.0f) ? __fmul_rn(gy, sp[2 * H + j]) : 0.0f;
                g[j] = __fmaf_rn(d1, v.x, g[j]);
                g[H + j] = __fadd_rn(g[H + j], d1);
                g[2 * H + j] = __fmaf_rn(gy, h, g[2 * H + j]);
            }
            g[3 * H] = __fadd_rn(g[3 * H], gy);
        }
        // fixed-order reduction: shuffle tree inside each warp, then the warps in order
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const float t = tb_warp_sum(g[u]);
            if (lane == 0) red[warp][u] = t;
        }
        {
            const float t = tb_warp_sum(lsum);
            if (lane == 0) red[warp][P] = t;
        }
        __syncthreads();
        if (tid < P) {
            float gs = 0.0f;
#pragma unroll
            for (int w = 0; w < TB_WARPS; ++w) gs = __fadd_rn(gs, red[w][tid]);
            const float c1 = a.c1[step], c2 = a.c2[step];
            const float mm = a.b1 * sm_[tid] + (1.0f - a.b1) * gs;
            const float vv = a.b2 * sv[tid] + (1.0f - a.b2) * gs * gs;
            sm_[tid] = mm;
            sv[tid] = vv;
            const float mh = mm / c1, vh = vv / c2;
            sp[tid] = sp[tid] - a.lr * mh / (sqrtf(vh) + a.eps);
        } else if (tid == P && a.loss_out) {
            float l = 0.0f;
#pragma unroll
            for (int w = 0; w < TB_WARPS; ++w) l = __fadd_rn(l, red[w][P]);
            a.loss_out[(size_t)m * a.steps + step] = l * inv_n;
        }
        __syncthreads();
    }
    for (int u = tid; u < P; u += TB_THREADS) a.params_out[(size_t)m * P + u] = sp[u];
    if (err) atomicOr(a.err, err);
}

template <typename W>
static cudaError_t tb_go(const TrainBlockArgs &a, int H, uint32_t blocks, cudaStream_t s) {
    const size_t smem = (size_t)a.cap * 8;
    auto go = [&](auto kfn) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kfn<<<blocks, TB_THREADS, smem, s>>>(a);
        return nns_launched(cudaGetLastError());
    };
    switch (H) {
    case 8: return go(k_train_block<W, 8>);
    case 16: return go(k_train_block<W, 16>);
    case 32: return go(k_train_block<W, 32>);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_train_block(const TrainBlockArgs &a, int key_bytes, int padded_h, uint32_t blocks,
                               cudaStream_t s) {
    if (blocks == 0) return cudaSuccess;
    if (a.cap < 2 || a.cap > TB_MAX_S || (a.cap & (a.cap - 1))) return cudaErrorInvalidValue;
    return key_bytes == 4 ? tb_go<uint32_t>(a, padded_h, blocks, s) : tb_go<uint64_t>(a, padded_h, blocks, s);
}

}  // namespace nns
