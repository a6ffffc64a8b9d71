// k_train.cu -- training the model f on the device (Sec. "Training"; Sec. "Experimental Study /
// Training details"; Eq. (loss)).
//
//   * sampling: S draws with replacement from the SplitMix64 stream of the training seed;
//   * labels: after a stable radix sort of the sample, label_j = j / S (the empirical CDF);
//   * gradient: each block takes a fixed chunk of the batch, runs the binary32 forward pass,
//     the loss derivative and backpropagation per sample, and reduces the chunk's parameter
//     gradient as small matrix products over its samples in a fixed order (no atomics);
//     block partials are then summed in block order, so gradients are reproducible;
//   * Adam (Kingma & Ba), bias-corrected, in binary32.
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

constexpr int TR_THREADS = 256;
constexpr int TR_CHUNK = 64;  // samples whose activations a block stages at once

// ---- sampling
template <typename W>
__global__ void k_sample(const W *keys, uint64_t n, int dtype, uint64_t S, uint64_t seed, W *out,
                         uint32_t *rows, uint32_t *err) {
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < S;
         j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r = __umul64hi(rng_draw(seed, j), n);
        const W k = keys[r];
        if (key_is_nan(word64(k), dtype)) atomicOr(err, ERR_NAN);
        out[j] = k;
        rows[j] = (uint32_t)r;
    }
}

cudaError_t launch_sample(const void *keys, uint64_t n, int key_bytes, int dtype, uint64_t S,
                          uint64_t stream_seed, void *sample_keys, uint32_t *sample_rows,
                          uint32_t *err, cudaStream_t s) {
    const int grid = (int)std::min<uint64_t>((S + 255) / 256, 4096);
    if (key_bytes == 4)
        k_sample<uint32_t><<<grid, 256, 0, s>>>(reinterpret_cast<const uint32_t *>(keys), n, dtype, S,
                                                stream_seed, reinterpret_cast<uint32_t *>(sample_keys),
                                                sample_rows, err);
    else
        k_sample<uint64_t><<<grid, 256, 0, s>>>(reinterpret_cast<const uint64_t *>(keys), n, dtype, S,
                                                stream_seed, reinterpret_cast<uint64_t *>(sample_keys),
                                                sample_rows, err);
    return nns_launched(cudaGetLastError());
}

template <typename W>
__global__ void k_make_xy(const W *sorted, uint64_t S, const Norm *nm, float *x, float *label) {
    const Norm N = *nm;
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < S;
         j += (uint64_t)gridDim.x * blockDim.x) {
        x[j] = translate_x(word64(sorted[j]), N);
        label[j] = __double2float_rn(__ddiv_rn((double)j, (double)S));
    }
}

cudaError_t launch_make_xy(const void *sorted_keys, uint64_t S, int key_bytes, const Norm *nm_dev,
                           float *x, float *label, cudaStream_t s) {
    const int grid = (int)std::min<uint64_t>((S + 255) / 256, 4096);
    if (key_bytes == 4)
        k_make_xy<uint32_t><<<grid, 256, 0, s>>>(reinterpret_cast<const uint32_t *>(sorted_keys), S,
                                                 nm_dev, x, label);
    else
        k_make_xy<uint64_t><<<grid, 256, 0, s>>>(reinterpret_cast<const uint64_t *>(sorted_keys), S,
                                                 nm_dev, x, label);
    return nns_launched(cudaGetLastError());
}

// ---- forward pass for explicit inputs
template <int H1, int H2>
__global__ void k_mlp_forward(const float *params, const float *x, uint64_t n, float *y) {
    extern __shared__ __align__(16) float sp[];
    constexpr int P = (H2 == 0) ? (3 * H1 + 1) : (2 * H1 + H2 * H1 + 2 * H2 + 1);
    for (int i = threadIdx.x; i < P; i += blockDim.x) sp[i] = params[i];
    __syncthreads();
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        y[i] = mlp_fwd_f32<H1, H2>(sp, x[i]);
}

// ---- gradient of a sum over samples (GradArgs: internal.h)
template <int H1, int H2>
__global__ void __launch_bounds__(TR_THREADS) k_grad(GradArgs g) {
    constexpr int HL = (H2 == 0) ? H1 : H2;
    constexpr int P = (H2 == 0) ? (3 * H1 + 1) : (2 * H1 + H2 * H1 + 2 * H2 + 1);
    extern __shared__ __align__(16) float sm[];
    float *sp = sm;                               // parameters (P, padded to 4)
    float *sx = sp + ((P + 3) & ~3);              // [CH] inputs
    float *sgy = sx + TR_CHUNK;                   // [CH] dL/dy
    float *sh1 = sgy + TR_CHUNK;                  // [CH][H1] hidden 1 activations
    float *sd1 = sh1 + TR_CHUNK * H1;             // [CH][H1] delta at hidden-1 pre-activations
    float *sh2 = sd1 + TR_CHUNK * H1;             // [CH][H2]
    float *sd2 = sh2 + TR_CHUNK * (H2 ? H2 : 1);  // [CH][H2]
    float *sloss = sd2 + TR_CHUNK * (H2 ? H2 : 1);  // [CH]
    const int tid = threadIdx.x;
    for (int i = tid; i < P; i += blockDim.x) sp[i] = g.params[i];
    __syncthreads();
    const float *W1 = sp, *b1 = sp + H1;
    const float *W2 = sp + 2 * H1, *b2 = W2 + H2 * H1;
    const float *W3 = (H2 == 0) ? sp + 2 * H1 : b2 + H2;
    // each block owns a contiguous range of the batch
    const uint64_t per = (g.n + gridDim.x - 1) / gridDim.x;
    const uint64_t i0 = std::min<uint64_t>(g.n, (uint64_t)blockIdx.x * per);
    const uint64_t i1 = std::min<uint64_t>(g.n, i0 + per);
    float acc[(P + TR_THREADS - 1) / TR_THREADS];
#pragma unroll
    for (int q = 0; q < (P + TR_THREADS - 1) / TR_THREADS; ++q) acc[q] = 0.0f;
    float lacc = 0.0f;
    for (uint64_t c0 = i0; c0 < i1; c0 += TR_CHUNK) {
        const int cn = (int)std::min<uint64_t>(TR_CHUNK, i1 - c0);
        // phase A: one sample per thread (threads >= cn idle)
        if (tid < cn) {
            const uint64_t i = c0 + tid;
            uint64_t src = i;
            if (g.mode == 2) src = __umul64hi(rng_draw(g.bseed, g.bofs + i), g.S);
            const float x = g.x[src];
            float h1[H1];
#pragma unroll
            for (int j = 0; j < H1; ++j) h1[j] = relu_f(__fmaf_rn(W1[j], x, b1[j]));
            float y;
            if constexpr (H2 == 0) {
                y = W3[H1];
#pragma unroll
                for (int k = 0; k < H1; ++k) y = __fmaf_rn(W3[k], h1[k], y);
            } else {
                y = W3[H2];
                for (int k = 0; k < H2; ++k) {
                    float z = b2[k];
#pragma unroll
                    for (int j = 0; j < H1; ++j) z = __fmaf_rn(W2[k * H1 + j], h1[j], z);
                    sd2[tid * H2 + k] = z;  // pre-activation, replaced by its delta below
                    const float h = relu_f(z);
                    sh2[tid * H2 + k] = h;
                    y = __fmaf_rn(W3[k], h, y);
                }
            }
            float gy, lv = 0.0f;
            if (g.mode == 0) {
                gy = g.gy[i];
            } else {
                const float r = y - g.label[src];
                if (g.loss == NNSORT_LOSS_HUBER) {
                    const float ar = fabsf(r);
                    lv = (ar <= g.delta) ? 0.5f * r * r : g.delta * ar - 0.5f * g.delta * g.delta;
                    gy = (r > g.delta) ? g.delta : ((r < -g.delta) ? -g.delta : r);
                } else {
                    lv = r * r;
                    gy = 2.0f * r;
                }
                gy *= g.inv_n;
            }
            sx[tid] = x;
            sgy[tid] = gy;
            sloss[tid] = lv;
            float d1[H1];
            if constexpr (H2 == 0) {
#pragma unroll
                for (int j = 0; j < H1; ++j) d1[j] = (h1[j] > 0.0f) ? gy * W3[j] : 0.0f;
            } else {
#pragma unroll
                for (int j = 0; j < H1; ++j) d1[j] = 0.0f;
                for (int k = 0; k < H2; ++k) {
                    const float d2 = (sd2[tid * H2 + k] > 0.0f) ? gy * W3[k] : 0.0f;
                    sd2[tid * H2 + k] = d2;
#pragma unroll
                    for (int j = 0; j < H1; ++j) d1[j] = __fmaf_rn(d2, W2[k * H1 + j], d1[j]);
                }
#pragma unroll
                for (int j = 0; j < H1; ++j) d1[j] = (h1[j] > 0.0f) ? d1[j] : 0.0f;
            }
            float gx = 0.0f;
#pragma unroll
            for (int j = 0; j < H1; ++j) {
                sh1[tid * H1 + j] = h1[j];
                sd1[tid * H1 + j] = d1[j];
                gx = __fmaf_rn(d1[j], W1[j], gx);
            }
            if (g.gx) g.gx[i] = gx;
        }
        __syncthreads();
        // phase B: every parameter sums its chunk contributions in sample order
#pragma unroll
        for (int q = 0; q < (P + TR_THREADS - 1) / TR_THREADS; ++q) {
            const int p = q * TR_THREADS + tid;
            if (p >= P) break;
            float s = 0.0f;
            if (p < H1) {                                  // W1_j: d1_j * x
                for (int c = 0; c < cn; ++c) s = __fmaf_rn(sd1[c * H1 + p], sx[c], s);
            } else if (p < 2 * H1) {                       // b1_j: d1_j
                const int j = p - H1;
                for (int c = 0; c < cn; ++c) s = __fadd_rn(s, sd1[c * H1 + j]);
            } else if (H2 != 0 && p < 2 * H1 + H2 * H1) {  // W2_kj: d2_k * h1_j
                const int kj = p - 2 * H1, k = kj / (H1 ? H1 : 1), j = kj - k * H1;
                for (int c = 0; c < cn; ++c) s = __fmaf_rn(sd2[c * (H2 ? H2 : 1) + k], sh1[c * H1 + j], s);
            } else if (H2 != 0 && p < 2 * H1 + H2 * H1 + H2) {  // b2_k: d2_k
                const int k = p - 2 * H1 - H2 * H1;
                for (int c = 0; c < cn; ++c) s = __fadd_rn(s, sd2[c * (H2 ? H2 : 1) + k]);
            } else if (p < P - 1) {                        // W3_k: gy * h_k
                const int k = p - (P - 1 - HL);
                if constexpr (H2 == 0)
                    for (int c = 0; c < cn; ++c) s = __fmaf_rn(sgy[c], sh1[c * H1 + k], s);
                else
                    for (int c = 0; c < cn; ++c) s = __fmaf_rn(sgy[c], sh2[c * (H2 ? H2 : 1) + k], s);
            } else {                                       // b3: gy
                for (int c = 0; c < cn; ++c) s = __fadd_rn(s, sgy[c]);
            }
            acc[q] = __fadd_rn(acc[q], s);
        }
        if (tid == 0)
            for (int c = 0; c < cn; ++c) lacc = __fadd_rn(lacc, sloss[c]);
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < (P + TR_THREADS - 1) / TR_THREADS; ++q) {
        const int p = q * TR_THREADS + tid;
        if (p < P) g.partials[(size_t)blockIdx.x * P + p] = acc[q];
    }
    if (tid == 0 && g.loss_partials) g.loss_partials[blockIdx.x] = lacc;
}

// Two hidden layers of width H (32 or 64): the per-chunk work as three register-tiled block
// products over all threads (C = 64 samples per chunk, 4 x TN outputs per thread):
//   Z  = b2 + H1 W2^T        (forward, accumulated over j in the oracle's order)
//   D1 = [H1 > 0] (D2 W2)    (backward), D2 = [Z > 0] gy W3
//   dW2 += D2^T H1           (kept in registers across the block's chunks)
// Every operand a thread reads in an inner step is a contiguous run of 4 (or 2) floats, one vector
// load: the products' left operands are staged transposed (H1^T, D2^T: [unit][sample]) next to
// the row-major copies the dW2 product reads. Every sum runs in a fixed order, so the gradient is
// reproducible.
constexpr int GC = 64;          // samples per chunk
template <int H> struct GemmSmem {
    static constexpr int LD = H + 4;   // row-major [sample][unit] stride (16-byte rows)
    static constexpr int LDT = GC + 4; // transposed [unit][sample] stride
    static constexpr int P = 2 * H + H * H + 2 * H + 1;
    static constexpr int OFF_W2T = (P + 3) & ~3;
    static constexpr int OFF_H1 = OFF_W2T + H * LD;     // H1 [s][j]
    static constexpr int OFF_H1T = OFF_H1 + GC * LD;    // H1^T [j][s]; then D1 [s][j] for gx
    static_assert(GC * H <= H * LDT, "D1 fits the H1^T buffer");
    static constexpr int OFF_HD = OFF_H1T + H * LDT;    // H2 [s][k], then D2 [s][k]
    static constexpr int OFF_D2T = OFF_HD + GC * LD;    // D2^T [k][s]
    static constexpr int OFF_X = OFF_D2T + H * LDT;
    static constexpr int OFF_GY = OFF_X + GC;
    static constexpr int OFF_L = OFF_GY + GC;
    static constexpr int FLOATS = OFF_L + GC;
};

template <int TN> struct VecT;
template <> struct VecT<4> { using T = ulonglong2; };
template <> struct VecT<2> { using T = unsigned long long; };
// the TN/2 packed column pairs of a contiguous run of TN floats
template <int TN>
__device__ __forceinline__ void load_pairs(const float *p, unsigned long long *b) {
    if constexpr (TN == 4) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p);
        b[0] = v.x;
        b[1] = v.y;
    } else {
        b[0] = *reinterpret_cast<const unsigned long long *>(p);
    }
}

template <int H>
__global__ void __launch_bounds__(TR_THREADS, 2) k_grad_gemm(GradArgs g) {
    using S = GemmSmem<H>;
    constexpr int LD = S::LD, LDT = S::LDT, P = S::P;
    constexpr int TN = H / 16;  // outputs per thread along the width (4 for H = 64, 2 for H = 32)
    static_assert(H == 32 || H == 64, "block-product gradient widths");
    extern __shared__ __align__(16) float sm[];
    float *sp = sm, *W2T = sm + S::OFF_W2T, *sH1 = sm + S::OFF_H1, *sH1T = sm + S::OFF_H1T;
    float *sHD = sm + S::OFF_HD, *sD2T = sm + S::OFF_D2T, *sX = sm + S::OFF_X, *sGY = sm + S::OFF_GY;
    const int tid = threadIdx.x;
    for (int i = tid; i < P; i += TR_THREADS) sp[i] = g.params[i];
    __syncthreads();
    const float *W1 = sp, *b1 = sp + H, *W2 = sp + 2 * H, *b2 = W2 + H * H, *W3 = b2 + H;
    const float b3 = W3[H];
    for (int e = tid; e < H * H; e += TR_THREADS) {  // W2T[j][k] = W2[k][j]
        const int k = e / H, j = e % H;
        W2T[j * LD + k] = W2[e];
    }
    // thread tiles: rows m0..m0+3 (samples), columns n0..n0+TN-1
    const int tm = tid / 16, tn = tid % 16;
    const int m0 = 4 * tm, n0 = TN * tn;
    // dW2 tile: rows k0..k0+TK-1, columns j0..j0+TN-1 over the H x H gradient
    constexpr int TK = (H * H) / (TR_THREADS * TN);  // 4 for H = 64, 2 for H = 32
    const int k0 = TK * tm, j0 = TN * tn;
    // accumulators hold column pairs (q, q+1) for the packed two-lane FMA: each lane is rounded as a
    // scalar FMA would be, so the sums are those of the scalar loop
    constexpr int TP = TN / 2;
    unsigned long long aW2[TK][TP];
#pragma unroll
    for (int i = 0; i < TK; ++i)
#pragma unroll
        for (int q = 0; q < TP; ++q) aW2[i][q] = 0ull;
    // vector gradients as per-thread partial sums, combined in a fixed order after the last chunk:
    // the D2 pass gives thread t the fixed column t % H (db2, dW3) over every (TR_THREADS / H)-th
    // sample; the D1 product's epilogue gives it columns n0..n0+TN-1 over rows m0..m0+3 (db1, dW1);
    // threads t < GC see sample t of every chunk (db3, loss)
    static_assert(TR_THREADS % H == 0, "fixed D2 column per thread");
    float pb2 = 0.0f, pw3 = 0.0f, pgy = 0.0f, plv = 0.0f;
    float pb1[TN], pw1[TN];
#pragma unroll
    for (int q = 0; q < TN; ++q) { pb1[q] = 0.0f; pw1[q] = 0.0f; }
    const uint64_t per = (g.n + gridDim.x - 1) / gridDim.x;
    const uint64_t i0 = std::min<uint64_t>(g.n, (uint64_t)blockIdx.x * per);
    const uint64_t i1 = std::min<uint64_t>(g.n, i0 + per);
    __syncthreads();
    for (uint64_t c0 = i0; c0 < i1; c0 += GC) {
        const int cn = (int)std::min<uint64_t>(GC, i1 - c0);
        uint64_t src = 0;
        if (tid < GC) {
            float x = 0.0f;
            if (tid < cn) {
                src = c0 + tid;
                if (g.mode == 2) src = __umul64hi(rng_draw(g.bseed, g.bofs + c0 + tid), g.S);
                x = g.x[src];
            }
            sX[tid] = x;
        }
        __syncthreads();
        for (int e = tid; e < GC * H; e += TR_THREADS) {
            const int s = e / H, j = e % H;
            const float h = (s < cn) ? relu_f(__fmaf_rn(W1[j], sX[s], b1[j])) : 0.0f;
            sH1[s * LD + j] = h;
            sH1T[j * LDT + s] = h;
        }
        __syncthreads();
        {   // Z = b2 + H1 W2^T, then H2 = relu(Z)
            unsigned long long acc[4][TP];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < TP; ++q) acc[i][q] = pk2(b2[n0 + 2 * q], b2[n0 + 2 * q + 1]);
#pragma unroll 8
            for (int j = 0; j < H; ++j) {
                unsigned long long b[TP];
                load_pairs<TN>(W2T + j * LD + n0, b);
                const float4 a4 = *reinterpret_cast<const float4 *>(sH1T + j * LDT + m0);
                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const unsigned long long a2 = pk2(av[i], av[i]);
#pragma unroll
                    for (int q = 0; q < TP; ++q) acc[i][q] = fma2_rn(b[q], a2, acc[i][q]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < TP; ++q) {
                    float z0, z1;
                    upk2(acc[i][q], z0, z1);
                    sHD[(m0 + i) * LD + n0 + 2 * q] = relu_f(z0);
                    sHD[(m0 + i) * LD + n0 + 2 * q + 1] = relu_f(z1);
                }
        }
        __syncthreads();
        if (tid < GC) {  // output, loss, upstream gradient per sample
            float gy = 0.0f, lv = 0.0f;
            if (tid < cn) {
                float y = b3;
                for (int k = 0; k < H; ++k) y = __fmaf_rn(W3[k], sHD[tid * LD + k], y);
                if (g.mode == 0) {
                    gy = g.gy[c0 + tid];
                } else {
                    const float r = y - g.label[src];
                    if (g.loss == NNSORT_LOSS_HUBER) {
                        const float ar = fabsf(r);
                        lv = (ar <= g.delta) ? 0.5f * r * r : g.delta * ar - 0.5f * g.delta * g.delta;
                        gy = (r > g.delta) ? g.delta : ((r < -g.delta) ? -g.delta : r);
                    } else {
                        lv = r * r;
                        gy = 2.0f * r;
                    }
                    gy *= g.inv_n;
                }
            }
            sGY[tid] = gy;
            pgy = __fadd_rn(pgy, gy);
            plv = __fadd_rn(plv, lv);
        }
        __syncthreads();
        for (int e = tid; e < GC * H; e += TR_THREADS) {
            const int s = e / H, k = e % H;  // k = tid % H on every iteration
            const float h2 = sHD[s * LD + k];
            const float d = (h2 > 0.0f) ? sGY[s] * W3[k] : 0.0f;
            sHD[s * LD + k] = d;
            sD2T[k * LDT + s] = d;
            pb2 = __fadd_rn(pb2, d);
            pw3 = __fmaf_rn(sGY[s], h2, pw3);
        }
        __syncthreads();
        {   // D1 = [H1 > 0] (D2 W2)
            unsigned long long acc[4][TP];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < TP; ++q) acc[i][q] = 0ull;
#pragma unroll 8
            for (int k = 0; k < H; ++k) {
                unsigned long long b[TP];
                load_pairs<TN>(W2 + k * H + n0, b);
                const float4 a4 = *reinterpret_cast<const float4 *>(sD2T + k * LDT + m0);
                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const unsigned long long a2 = pk2(av[i], av[i]);
#pragma unroll
                    for (int q = 0; q < TP; ++q) acc[i][q] = fma2_rn(a2, b[q], acc[i][q]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < TP; ++q) {
                    float d0, d1;
                    upk2(acc[i][q], d0, d1);
                    const int c = (m0 + i) * LD + n0 + 2 * q;
                    const float e0 = (sH1[c] > 0.0f) ? d0 : 0.0f, e1 = (sH1[c + 1] > 0.0f) ? d1 : 0.0f;
                    if (g.gx) {  // D1 [s][j] (stride H) over the (now free) H1^T buffer
                        sH1T[(m0 + i) * H + n0 + 2 * q] = e0;
                        sH1T[(m0 + i) * H + n0 + 2 * q + 1] = e1;
                    }
                    const float xs = sX[m0 + i];
                    pb1[2 * q] = __fadd_rn(pb1[2 * q], e0);
                    pb1[2 * q + 1] = __fadd_rn(pb1[2 * q + 1], e1);
                    pw1[2 * q] = __fmaf_rn(e0, xs, pw1[2 * q]);
                    pw1[2 * q + 1] = __fmaf_rn(e1, xs, pw1[2 * q + 1]);
                }
        }
        __syncthreads();
        if (g.gx && tid < cn) {
            float gx = 0.0f;
            for (int j = 0; j < H; ++j) gx = __fmaf_rn(sH1T[tid * H + j], W1[j], gx);
            g.gx[c0 + tid] = gx;
        }
        // dW2 += D2^T H1 over this chunk's samples
#pragma unroll 4
        for (int s = 0; s < cn; ++s) {
            unsigned long long b[TP];
            load_pairs<TN>(sH1 + s * LD + j0, b);
            float av[TK];
            if constexpr (TK == 4) {
                const float4 a4 = *reinterpret_cast<const float4 *>(sHD + s * LD + k0);
                av[0] = a4.x; av[1] = a4.y; av[2] = a4.z; av[3] = a4.w;
            } else {
                const float2 a2v = *reinterpret_cast<const float2 *>(sHD + s * LD + k0);
                av[0] = a2v.x; av[1] = a2v.y;
            }
#pragma unroll
            for (int i = 0; i < TK; ++i) {
                const unsigned long long a2 = pk2(av[i], av[i]);
#pragma unroll
                for (int q = 0; q < TP; ++q) aW2[i][q] = fma2_rn(a2, b[q], aW2[i][q]);
            }
        }
        __syncthreads();
    }
    // combine the partial sums (the activation tiles are free now)
    float *R2b = sH1, *R2w = R2b + TR_THREADS, *R1b = R2w + TR_THREADS, *R1w = R1b + TR_THREADS * TN;
    float *Rg = R1w + TR_THREADS * TN, *Rl = Rg + GC;
    static_assert((2 + 2 * TN) * TR_THREADS + 2 * GC <= GC * LD + H * LDT, "partials fit the activation tiles");
    R2b[tid] = pb2;
    R2w[tid] = pw3;
#pragma unroll
    for (int q = 0; q < TN; ++q) { R1b[tid * TN + q] = pb1[q]; R1w[tid * TN + q] = pw1[q]; }
    if (tid < GC) { Rg[tid] = pgy; Rl[tid] = plv; }
    __syncthreads();
    float *out = g.partials + (size_t)blockIdx.x * P;
#pragma unroll
    for (int i = 0; i < TK; ++i)
#pragma unroll
        for (int q = 0; q < TP; ++q) {
            float w0, w1;
            upk2(aW2[i][q], w0, w1);
            out[2 * H + (k0 + i) * H + j0 + 2 * q] = w0;
            out[2 * H + (k0 + i) * H + j0 + 2 * q + 1] = w1;
        }
    if (tid < H) {  // column tid of D2: threads tid, tid + H, ...
        float b = 0.0f, w = 0.0f;
        for (int ph = 0; ph < TR_THREADS / H; ++ph) {
            b = __fadd_rn(b, R2b[ph * H + tid]);
            w = __fadd_rn(w, R2w[ph * H + tid]);
        }
        out[2 * H + H * H + tid] = b;        // b2
        out[3 * H + H * H + tid] = w;        // W3
    } else if (tid < 2 * H) {  // column j of D1: thread (tm, j / TN), slot j % TN, for every tm
        const int j = tid - H, tn2 = j / TN, q = j % TN;
        float b = 0.0f, w = 0.0f;
        for (int tm2 = 0; tm2 < TR_THREADS / 16; ++tm2) {
            b = __fadd_rn(b, R1b[(tm2 * 16 + tn2) * TN + q]);
            w = __fadd_rn(w, R1w[(tm2 * 16 + tn2) * TN + q]);
        }
        out[H + j] = b;                      // b1
        out[j] = w;                          // W1
    } else if (tid == 2 * H) {
        float b = 0.0f;
        for (int t2 = 0; t2 < GC; ++t2) b = __fadd_rn(b, Rg[t2]);
        out[P - 1] = b;                      // b3
    } else if (tid == 2 * H + 1 && g.loss_partials) {
        float l = 0.0f;
        for (int t2 = 0; t2 < GC; ++t2) l = __fadd_rn(l, Rl[t2]);
        g.loss_partials[blockIdx.x] = l;
    }
}

template <int H1, int H2> static size_t grad_smem() {
    constexpr int P = (H2 == 0) ? (3 * H1 + 1) : (2 * H1 + H2 * H1 + 2 * H2 + 1);
    constexpr int H2e = H2 ? H2 : 1;
    return sizeof(float) * (((P + 3) & ~3) + TR_CHUNK * (3 + 2 * H1 + 2 * H2e));
}

int train_grad_blocks(const PadArch &a, uint64_t nsamples) {
    // width 64: the tensor-core kernel
    if (a.layers == 2 && a.h1 == 64) return grad_tc64_blocks(nsamples);
    // the block-product kernel (two hidden layers of 32) takes four chunks per block, so its
    // thousands of per-block partial gradients stay few; the per-sample kernel of the small shapes
    // takes one chunk per block, so small batches still spread over the GPU; at most 1024 blocks
    const bool gemm = a.layers == 2 && a.h1 == 32;
    const uint64_t per = gemm ? 4 * TR_CHUNK : TR_CHUNK;
    const uint64_t b = (nsamples + per - 1) / per;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>(b, 1024));
}

template <int H1, int H2>
static cudaError_t grad_go(const GradArgs &g, int blocks, cudaStream_t s) {
    const size_t smem = grad_smem<H1, H2>();
    cudaError_t e = cudaFuncSetAttribute(k_grad<H1, H2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_grad<H1, H2><<<blocks, TR_THREADS, smem, s>>>(g);
    return nns_launched(cudaGetLastError());
}

template <int H>
static cudaError_t grad_gemm_go(const GradArgs &g, int blocks, cudaStream_t s) {
    const size_t smem = sizeof(float) * GemmSmem<H>::FLOATS;
    cudaError_t e = cudaFuncSetAttribute(k_grad_gemm<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_grad_gemm<H><<<blocks, TR_THREADS, smem, s>>>(g);
    return nns_launched(cudaGetLastError());
}

static cudaError_t grad_dispatch(const PadArch &a, const GradArgs &g, int blocks, cudaStream_t s) {
    if (a.layers == 1) {
        switch (a.h1) {
        case 8: return grad_go<8, 0>(g, blocks, s);
        case 16: return grad_go<16, 0>(g, blocks, s);
        case 32: return grad_go<32, 0>(g, blocks, s);
        case 64: return grad_go<64, 0>(g, blocks, s);
        }
    } else {
        switch (a.h1) {
        case 8: return grad_go<8, 8>(g, blocks, s);
        case 16: return grad_go<16, 16>(g, blocks, s);
        case 32: return grad_gemm_go<32>(g, blocks, s);
        case 64: return launch_grad_tc64(g, s);
        }
    }
    return cudaErrorInvalidValue;
}

// ---- fixed-order reduction of block partials (+ optional Adam step)
struct ReduceArgs {
    const float *partials;
    int blocks;
    size_t P;
    float *out;                 // gradient (nullable when Adam consumes it directly)
    const float *loss_partials;
    float *loss_out;
    float loss_scale;
    // Adam
    float *params, *m, *v;
    const float *mask;  // nullable: +1/-1 sign a parameter must keep, 0 free
    float lr, b1, b2, eps, c1, c2;
};

// A block takes 32 parameters (lane l: parameter 32 b + l) and its warp w adds partial rows w, w + 16,
// ... in order, issuing eight row loads before the first add (each load one coalesced 128-byte row
// segment); the sixteen warp sums then meet in warp order. One more block sums the loss partials
// the same way. The result does not depend on timing.
constexpr int RD_WARPS = 16;
__device__ __forceinline__ float rows_sum(const float *col, size_t stride, int rows, int w, bool active) {
    float acc = 0.0f;
    for (int b0 = w; b0 < rows; b0 += RD_WARPS * 8) {
        float t[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int b = b0 + RD_WARPS * q;
            t[q] = (active && b < rows) ? col[(size_t)b * stride] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (b0 + RD_WARPS * q < rows) acc = __fadd_rn(acc, t[q]);
    }
    return acc;
}

__global__ void __launch_bounds__(RD_WARPS * 32) k_reduce(ReduceArgs r) {
    __shared__ float sh[RD_WARPS][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const size_t nb = (r.P + 31) / 32;
    if (blockIdx.x == nb) {  // the loss
        const bool on = r.loss_partials && r.loss_out && lane == 0;
        sh[w][lane] = rows_sum(r.loss_partials, 1, r.blocks, w, on);
        __syncthreads();
        if (on && w == 0) {
            float l = 0.0f;
            for (int q = 0; q < RD_WARPS; ++q) l = __fadd_rn(l, sh[q][0]);
            *r.loss_out = l * r.loss_scale;
        }
        return;
    }
    const size_t p = (size_t)blockIdx.x * 32 + lane;
    sh[w][lane] = rows_sum(r.partials + p, r.P, r.blocks, w, p < r.P);
    __syncthreads();
    if (w != 0 || p >= r.P) return;
    float g = 0.0f;
    for (int q = 0; q < RD_WARPS; ++q) g = __fadd_rn(g, sh[q][lane]);
    if (r.out) r.out[p] = g;
    if (r.params) {
        const float m = r.b1 * r.m[p] + (1.0f - r.b1) * g;
        const float v = r.b2 * r.v[p] + (1.0f - r.b2) * g * g;
        r.m[p] = m;
        r.v[p] = v;
        const float mh = m / r.c1, vh = v / r.c2;
        float np = r.params[p] - r.lr * mh / (sqrtf(vh) + r.eps);
        if (r.mask && r.mask[p] * np < 0.0f) np = 0.0f;  // monotone projection
        r.params[p] = np;
    }
}
static unsigned reduce_grid(size_t P) { return (unsigned)((P + 31) / 32 + 1); }

cudaError_t launch_reduce_partials(const float *partials, int blocks, size_t P, float *out,
                                   const float *loss_partials, float *loss_out, float scale,
                                   cudaStream_t s) {
    ReduceArgs r{};
    r.partials = partials; r.blocks = blocks; r.P = P; r.out = out;
    r.loss_partials = loss_partials; r.loss_out = loss_out; r.loss_scale = scale;
    k_reduce<<<reduce_grid(P), RD_WARPS * 32, 0, s>>>(r);
    return nns_launched(cudaGetLastError());
}

cudaError_t launch_train_step(const PadArch &a, const TrainStepArgs &t, cudaStream_t s) {
    const uint64_t B = t.batch ? t.batch : t.S;
    const int blocks = train_grad_blocks(a, B);
    GradArgs g{};
    g.params = t.params; g.x = t.x; g.label = t.label; g.n = B; g.S = t.S;
    g.bseed = t.batch_seed; g.bofs = (uint64_t)t.step * B;
    g.mode = t.batch ? 2 : 1; g.loss = t.loss; g.delta = t.delta; g.inv_n = 1.0f / (float)B;
    g.partials = t.partials; g.loss_partials = t.loss_partials; g.gx = nullptr;
    cudaError_t e = grad_dispatch(a, g, blocks, s);
    if (e != cudaSuccess) return e;
    ReduceArgs r{};
    r.partials = t.partials; r.blocks = blocks; r.P = t.P; r.out = t.grad;
    r.loss_partials = t.loss_partials; r.loss_out = t.loss_out + t.step; r.loss_scale = 1.0f / (float)B;
    r.params = t.params; r.m = t.m; r.v = t.v; r.lr = t.lr; r.b1 = t.b1; r.b2 = t.b2; r.eps = t.eps;
    r.mask = t.mask;
    const double c1 = 1.0 - std::pow((double)t.b1, (double)(t.step + 1));
    const double c2 = 1.0 - std::pow((double)t.b2, (double)(t.step + 1));
    r.c1 = (float)c1; r.c2 = (float)c2;
    k_reduce<<<reduce_grid(t.P), RD_WARPS * 32, 0, s>>>(r);
    return nns_launched(cudaGetLastError());
}

cudaError_t launch_mlp_forward(const PadArch &a, const float *params, const float *x, uint64_t n,
                               float *y, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int grid = (int)std::min<uint64_t>((n + 255) / 256, 2048);
#define NNS_F(A, B)                                                                             \
    {                                                                                           \
        constexpr int P = (B == 0) ? (3 * A + 1) : (2 * A + B * A + 2 * B + 1);                 \
        k_mlp_forward<A, B><<<grid, 256, ((P + 3) / 4) * 16, s>>>(params, x, n, y);            \
        return nns_launched(cudaGetLastError());                                                              \
    }
    if (a.layers == 1) {
        switch (a.h1) {
        case 8: NNS_F(8, 0)
        case 16: NNS_F(16, 0)
        case 32: NNS_F(32, 0)
        case 64: NNS_F(64, 0)
        }
    } else {
        switch (a.h1) {
        case 8: NNS_F(8, 8)
        case 16: NNS_F(16, 16)
        case 32: NNS_F(32, 32)
        case 64: NNS_F(64, 64)
        }
    }
#undef NNS_F
    return cudaErrorInvalidValue;
}

cudaError_t launch_mlp_backward(const PadArch &a, const float *params, const float *x,
                                const float *gy, const float *label, uint64_t n, int mode,
                                int loss, float delta, float *partials, float *loss_partials,
                                float *gx, cudaStream_t s, int *blocks_out) {
    const int blocks = train_grad_blocks(a, n);
    if (blocks_out) *blocks_out = blocks;
    GradArgs g{};
    g.params = params; g.x = x; g.gy = gy; g.label = label; g.n = n; g.S = n;
    g.mode = mode; g.loss = loss; g.delta = delta; g.inv_n = n ? 1.0f / (float)n : 0.0f;
    g.partials = partials; g.loss_partials = loss_partials; g.gx = gx;
    return grad_dispatch(a, g, blocks, s);
}

}  // namespace nns
