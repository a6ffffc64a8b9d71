// k_train_tc.cu -- the gradient of one training step (Sec. "Training", Eq. (loss)) of the model with
// two hidden layers of width 64, its matrix products on the fifth-generation tensor cores
// (tcgen05.mma kind::f16: BF16 operands, FP32 accumulation in tensor memory).
//
// Binary32 operands enter the products as sums of BF16 parts: v = v0 + v1 (+ v2), each part the
// BF16 rounding of what the earlier parts leave, so two parts carry 16 significant bits and three
// carry the 24 of binary32. Part products are exact in FP32 and accumulate in tensor memory; the
// smallest are issued first so that they meet a small accumulator.
//
// A block holds two groups of four warps; a group takes chunks of 128 samples (one sample per
// thread and per tensor-memory lane) and, per chunk:
//   1. layer 1 on the CUDA cores, binary32 FMA and ReLU as in the forward pass; H1 = three parts;
//   2. Z = H1 W2^T: the six part products whose weight is at least 2^-24 (W2 in three parts,
//      staged once per block);
//   3. per sample: z = Z + b2, h2 = ReLU(z), y = b3 + W3 . h2, the loss derivative gy, and the rows
//      D2 = [z > 0] gy W3 and G = gy h2 (two parts each);
//   4. D1pre = D2 W2 (five part products); the sums over samples dW2 += D2^T H1 (hi and mid parts
//      of both stacked into one 128 x 128 product, four part products), db2 += D2^T 1 and
//      dW3 += G^T 1;
//   5. D1 = [W1 x + b1 > 0] D1pre (two parts); db1 += D1^T 1 and dW1 += D1^T x (x in two parts).
// Every row a thread writes (one sample's 64 units) is read by the products over units as a K-major
// operand and by the products over samples as an MN-major one, so nothing is transposed. The sums
// over samples stay in tensor memory across the group's chunks; at the end each group writes its
// own partial gradient row, summed in a fixed order by the reduction. Chunks go to groups
// round-robin, so the result does not depend on timing.
#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"
#include "internal.h"
#include "tc05.cuh"

namespace nns {

__device__ uint32_t g_train_err;  // ERR_TIMEOUT when a bounded wait of a training kernel expired

namespace {
using namespace tc05;

constexpr int GH = 64;                      // hidden width
constexpr int GM = 128;                     // samples per chunk = MMA rows = threads per group
constexpr int GNG = 2;                      // groups per block
constexpr int GTHREADS = GNG * GM;
constexpr int GP = 4 * GH + GH * GH + 1;    // parameters: W1 b1 W2 b2 W3 b3
constexpr uint32_t PART = GM * GH * 2;      // one BF16 part of a 128 x 64 matrix (16 KB)
constexpr uint32_t WPART = GH * GH * 2;     // one BF16 part of W2 (8 KB)
// Row-major BF16 layouts as 8 x 8 core matrices (16-byte rows): element (row r, column u) of a
// 128-row matrix at (u / 8) * CH_ACT + r * 16 + (u % 8) * 2, of W2 (row k, column j) at
// (j / 8) * CH_W + k * 16 + (j % 8) * 2. Read K-major over the columns: LBO = CH, SBO = 128;
// read MN-major (the columns as M or N, the rows as K): SBO = CH, LBO = 128. Parts of one matrix
// lie CH * 8 apart, so stacked parts continue the column-block sequence.
constexpr uint32_t CH_ACT = 2048;
constexpr uint32_t CH_W = 1024;
// group region: [H1 hi][H1 mid][R1: H1 lo, then D2 hi][R2: D2 mid][R3: G hi, then D1 hi]
//               [R4: G mid, then D1 mid][V: per-sample columns (valid, x hi, x mid, 0, ...)]
constexpr uint32_t O_H1 = 0, O_R1 = 2 * PART, O_R3 = 4 * PART, O_V = 6 * PART;
constexpr uint32_t GROUP_BYTES = O_V + 2 * CH_ACT;
constexpr uint32_t OFF_W = 0, OFF_GRP = 3 * WPART, OFF_PAR = OFF_GRP + GNG * GROUP_BYTES;
constexpr uint32_t NPAR = 4 * GH + 4;       // W1 | b1 | b2 | W3 | b3 in binary32
constexpr uint32_t SMEM_BYTES = OFF_PAR + NPAR * 4;
static_assert(SMEM_BYTES <= 232448, "one block per SM");
// tensor-memory columns of a group (two groups: 512 columns)
constexpr uint32_t C_Z = 0, C_W2 = 64, C_B2 = 192, C_W3 = 208, C_V1 = 224, GCOLS = 256;
constexpr int QW = 70;                      // row stride of the final per-lane sums (floats)
static_assert((uint32_t)GM * QW * 4 <= GROUP_BYTES, "final sums fit the group region");
constexpr int MAX_BLOCKS = 152;             // one block per SM of a 152-SM GPU

constexpr uint32_t I_ZK = idesc_bf16(GM, GH);               // A, B K-major
constexpr uint32_t I_D1 = idesc_bf16(GM, GH, false, true);  // B MN-major
constexpr uint32_t I_W2 = idesc_bf16(GM, 2 * GH, true, true);
constexpr uint32_t I_VEC = idesc_bf16(GM, 16, true, true);

__device__ __forceinline__ uint64_t kdesc(uint32_t addr, uint32_t ch) { return mdesc(addr, ch, 128); }
__device__ __forceinline__ uint64_t mndesc(uint32_t addr, uint32_t ch) { return mdesc(addr, 128, ch); }

// two binary32 values as BF16 (first in the low half), rounded to nearest
__device__ __forceinline__ uint32_t bf2_rn(float first, float second) {
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(second), "f"(first));
    return d;
}
// the rest of (a, b) after subtracting the BF16 pair p (exact: p is the rounding of a value that
// agrees with (a, b) to at least 8 bits)
__device__ __forceinline__ unsigned long long rest2(unsigned long long ab, uint32_t p) {
    return sub2_rn(ab, pk2(__uint_as_float(p << 16), __uint_as_float(p & 0xFFFF0000u)));
}
__device__ __forceinline__ void split2(float a, float b, uint32_t &p0, uint32_t &p1) {
    const unsigned long long ab = pk2(a, b);
    p0 = bf2_rn(a, b);
    float r0, r1;
    upk2(rest2(ab, p0), r0, r1);
    p1 = bf2_rn(r0, r1);
}
__device__ __forceinline__ void split3(float a, float b, uint32_t &p0, uint32_t &p1, uint32_t &p2) {
    p0 = bf2_rn(a, b);
    const unsigned long long r = rest2(pk2(a, b), p0);
    float r0, r1;
    upk2(r, r0, r1);
    p1 = bf2_rn(r0, r1);
    float s0, s1;
    upk2(rest2(r, p1), s0, s1);
    p2 = bf2_rn(s0, s1);
}

__device__ __forceinline__ void st16(unsigned char *p, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    *reinterpret_cast<uint4 *>(p) = make_uint4(a, b, c, d);
}
__device__ __forceinline__ void gsync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(GM) : "memory");
}
__device__ __forceinline__ bool gor(int id, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "n"(GM)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float *v) {
#pragma unroll
    for (int q = 0; q < 4; ++q) tmem_ld16(taddr + 16 * q, v + 16 * q);
    tmem_wait_ld();
}

__global__ void __launch_bounds__(GTHREADS, 1) k_grad_tc64(GradArgs g) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) unsigned long long bar[GNG];
    __shared__ uint32_t tmem_base;
    float *par = reinterpret_cast<float *>(sm + OFF_PAR);
    const float4 *pv = reinterpret_cast<const float4 *>(par);
    const int tid = threadIdx.x, warp = tid >> 5, grp = tid / GM, t = tid % GM;
    if (warp == 0) tmem_alloc<GNG * GCOLS>(smem_u32(&tmem_base));
    if (tid == 0) {
        for (int q = 0; q < GNG; ++q) mbar_init(smem_u32(&bar[q]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {   // W2 as three BF16 parts; the vectors in binary32; the zero columns 8..15 of V
        const float *P = g.params;
        for (int e = tid; e < GH * GH; e += GTHREADS) {
            const int k = e / GH, j = e % GH;
            const float w = P[2 * GH + e];
            const __nv_bfloat16 p0 = __float2bfloat16_rn(w);
            const float r = __fsub_rn(w, __bfloat162float(p0));
            const __nv_bfloat16 p1 = __float2bfloat16_rn(r);
            const __nv_bfloat16 p2 = __float2bfloat16_rn(__fsub_rn(r, __bfloat162float(p1)));
            unsigned char *o = sm + OFF_W + (j / 8) * CH_W + k * 16 + (j % 8) * 2;
            *reinterpret_cast<__nv_bfloat16 *>(o) = p0;
            *reinterpret_cast<__nv_bfloat16 *>(o + WPART) = p1;
            *reinterpret_cast<__nv_bfloat16 *>(o + 2 * WPART) = p2;
        }
        for (int e = tid; e < GH; e += GTHREADS) {
            par[e] = P[e];                              // W1
            par[GH + e] = P[GH + e];                    // b1
            par[2 * GH + e] = P[2 * GH + GH * GH + e];  // b2
            par[3 * GH + e] = P[3 * GH + GH * GH + e];  // W3
        }
        if (tid == 0) par[4 * GH] = P[4 * GH + GH * GH];  // b3
        for (int e = tid; e < GNG * GM; e += GTHREADS)
            st16(sm + OFF_GRP + (e / GM) * GROUP_BYTES + O_V + CH_ACT + (e % GM) * 16, 0u, 0u, 0u, 0u);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const uint32_t tb = tmem_base + (uint32_t)(grp * GCOLS);
    const uint32_t lane_addr = tb + ((uint32_t)((warp & 3) * 32) << 16);
    unsigned char *R = sm + OFF_GRP + grp * GROUP_BYTES;
    const uint32_t rb = smem_u32(R), wb = smem_u32(sm + OFF_W);
    const uint32_t mybar = smem_u32(&bar[grp]);
    const int bid = 1 + grp;
    const float b3 = par[4 * GH];
    const uint64_t nchunks = (g.n + GM - 1) / GM;
    const uint64_t ngroups = (uint64_t)gridDim.x * GNG;
    uint32_t phase = 0, err = 0, dead_parity = 0;
    bool dead = false, first = true;
    float pgy = 0.0f, plv = 0.0f;
    for (uint64_t c = (uint64_t)blockIdx.x * GNG + grp; c < nchunks; c += ngroups) {
        const uint64_t i = c * GM + t;
        const bool valid = i < g.n;
        uint64_t src = i;
        if (g.mode == 2 && valid) src = __umul64hi(rng_draw(g.bseed, g.bofs + i), g.S);
        const float x = valid ? g.x[src] : 0.0f;
        const float lab = (valid && g.mode != 0) ? g.label[src] : 0.0f;
        const float gyin = (valid && g.mode == 0) ? g.gy[i] : 0.0f;
        const unsigned long long xx = pk2(x, x);

        // 1. H1 = ReLU(W1 x + b1), three parts
#pragma unroll
        for (int c8 = 0; c8 < GH / 8; ++c8) {
            const float4 wa = pv[2 * c8], wq = pv[2 * c8 + 1];
            const float4 ba = pv[GH / 4 + 2 * c8], bq = pv[GH / 4 + 2 * c8 + 1];
            const float w8[8] = {wa.x, wa.y, wa.z, wa.w, wq.x, wq.y, wq.z, wq.w};
            const float b8[8] = {ba.x, ba.y, ba.z, ba.w, bq.x, bq.y, bq.z, bq.w};
            uint32_t p0[4], p1[4], p2[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float h0, h1;
                upk2(fma2_rn(pk2(w8[2 * q], w8[2 * q + 1]), xx, pk2(b8[2 * q], b8[2 * q + 1])), h0, h1);
                h0 = valid ? relu_f(h0) : 0.0f;
                h1 = valid ? relu_f(h1) : 0.0f;
                split3(h0, h1, p0[q], p1[q], p2[q]);
            }
            const uint32_t o = c8 * CH_ACT + t * 16;
            st16(R + O_H1 + o, p0[0], p0[1], p0[2], p0[3]);
            st16(R + O_H1 + PART + o, p1[0], p1[1], p1[2], p1[3]);
            st16(R + O_R1 + o, p2[0], p2[1], p2[2], p2[3]);
        }
        fence_async_smem();
        tc_fence_before();
        gsync(bid);
        tc_fence_after();

        // 2. Z = H1 W2^T (this commit also covers the previous chunk's column sums)
        if (t == 0 && !dead) {
            const uint32_t ha[3] = {rb + O_H1, rb + O_H1 + PART, rb + O_R1};
            const int pa[6] = {2, 0, 1, 1, 0, 0}, pb[6] = {0, 2, 1, 0, 1, 0};
#pragma unroll
            for (int pr = 0; pr < 6; ++pr)
#pragma unroll
                for (int ks = 0; ks < GH / 16; ++ks)
                    mma_bf16(tb + C_Z, kdesc(ha[pa[pr]] + ks * 2 * CH_ACT, CH_ACT),
                             kdesc(wb + pb[pr] * WPART + ks * 2 * CH_W, CH_W), I_ZK, (pr | ks) ? 1u : 0u);
            mma_commit(mybar);
            if (!mbar_wait(mybar, phase)) {
                dead = true;
                dead_parity = phase;
                err |= ERR_TIMEOUT;
            }
            phase ^= 1u;
            tc_fence_before();
        }
        dead = gor(bid, dead);
        tc_fence_after();

        // 3. output, loss derivative, D2 and G rows
        float z[GH];
        if (!dead) {
            tmem_ld64(lane_addr + C_Z, z);
        } else {
#pragma unroll
            for (int k = 0; k < GH; ++k) z[k] = 0.0f;
        }
        unsigned long long yy = pk2(b3, 0.0f);
#pragma unroll
        for (int k4 = 0; k4 < GH / 4; ++k4) {
            const float4 b2q = pv[GH / 2 + k4], w3q = pv[3 * GH / 4 + k4];
            float a0, a1, a2, a3;
            upk2(add2_rn(pk2(z[4 * k4], z[4 * k4 + 1]), pk2(b2q.x, b2q.y)), a0, a1);
            upk2(add2_rn(pk2(z[4 * k4 + 2], z[4 * k4 + 3]), pk2(b2q.z, b2q.w)), a2, a3);
            z[4 * k4] = relu_f(a0);
            z[4 * k4 + 1] = relu_f(a1);
            z[4 * k4 + 2] = relu_f(a2);
            z[4 * k4 + 3] = relu_f(a3);
            yy = fma2_rn(pk2(w3q.x, w3q.y), pk2(z[4 * k4], z[4 * k4 + 1]), yy);
            yy = fma2_rn(pk2(w3q.z, w3q.w), pk2(z[4 * k4 + 2], z[4 * k4 + 3]), yy);
        }
        float gy = 0.0f, lv = 0.0f;
        if (valid) {
            if (g.mode == 0) {
                gy = gyin;
            } else {
                float ye, yo;
                upk2(yy, ye, yo);
                const float r = __fsub_rn(__fadd_rn(ye, yo), lab);
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
        pgy = __fadd_rn(pgy, gy);
        plv = __fadd_rn(plv, lv);
        {
            const unsigned long long gg = pk2(gy, gy);
#pragma unroll
            for (int c8 = 0; c8 < GH / 8; ++c8) {
                uint32_t d0[4], d1[4], e0[4], e1[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int k = 8 * c8 + 2 * q;
                    const float w0 = par[3 * GH + k], w1 = par[3 * GH + k + 1];
                    float a, b;
                    upk2(mul2_rn(gg, pk2(w0, w1)), a, b);
                    split2(z[k] > 0.0f ? a : 0.0f, z[k + 1] > 0.0f ? b : 0.0f, d0[q], d1[q]);
                    upk2(mul2_rn(gg, pk2(z[k], z[k + 1])), a, b);
                    split2(a, b, e0[q], e1[q]);
                }
                const uint32_t o = c8 * CH_ACT + t * 16;
                st16(R + O_R1 + o, d0[0], d0[1], d0[2], d0[3]);
                st16(R + O_R1 + PART + o, d1[0], d1[1], d1[2], d1[3]);
                st16(R + O_R3 + o, e0[0], e0[1], e0[2], e0[3]);
                st16(R + O_R3 + PART + o, e1[0], e1[1], e1[2], e1[3]);
            }
            uint32_t xh, xm;
            split2(x, 0.0f, xh, xm);
            // columns: 0 = 1 (valid samples), 1 = x hi, 2 = x mid
            st16(R + O_V + t * 16, (valid ? 0x3F80u : 0u) | (xh << 16), xm & 0xFFFFu, 0u, 0u);
        }
        fence_async_smem();
        tc_fence_before();
        gsync(bid);
        tc_fence_after();

        // 4. D1pre = D2 W2; dW2 += D2^T H1; db2 += D2^T 1; dW3 += G^T 1
        if (t == 0 && !dead) {
            const uint32_t da[2] = {rb + O_R1, rb + O_R1 + PART};
            const int qa[5] = {1, 1, 0, 0, 0}, qb[5] = {1, 0, 2, 1, 0};
#pragma unroll
            for (int pr = 0; pr < 5; ++pr)
#pragma unroll
                for (int ks = 0; ks < GH / 16; ++ks)
                    mma_bf16(tb + C_Z, kdesc(da[qa[pr]] + ks * 2 * CH_ACT, CH_ACT),
                             mndesc(wb + qb[pr] * WPART + ks * 256, CH_W), I_D1, (pr | ks) ? 1u : 0u);
#pragma unroll
            for (int ks = 0; ks < GM / 16; ++ks) {
                const uint32_t acc = (!first || ks) ? 1u : 0u;
                const uint64_t d2 = mndesc(rb + O_R1 + ks * 256, CH_ACT);
                const uint64_t vv = mndesc(rb + O_V + ks * 256, CH_ACT);
                mma_bf16(tb + C_W2, d2, mndesc(rb + O_H1 + ks * 256, CH_ACT), I_W2, acc);
                mma_bf16(tb + C_B2, d2, vv, I_VEC, acc);
                mma_bf16(tb + C_W3, mndesc(rb + O_R3 + ks * 256, CH_ACT), vv, I_VEC, acc);
            }
            mma_commit(mybar);
            if (!mbar_wait(mybar, phase)) {
                dead = true;
                dead_parity = phase;
                err |= ERR_TIMEOUT;
            }
            phase ^= 1u;
            tc_fence_before();
        }
        dead = gor(bid, dead);
        tc_fence_after();

        // 5. D1 = [W1 x + b1 > 0] D1pre rows; the input gradient
        {
            float d[GH];
            if (!dead) {
                tmem_ld64(lane_addr + C_Z, d);
            } else {
#pragma unroll
                for (int k = 0; k < GH; ++k) d[k] = 0.0f;
            }
            float gx = 0.0f;
#pragma unroll
            for (int c8 = 0; c8 < GH / 8; ++c8) {
                const float4 wa = pv[2 * c8], wq = pv[2 * c8 + 1];
                const float4 ba = pv[GH / 4 + 2 * c8], bq = pv[GH / 4 + 2 * c8 + 1];
                const float w8[8] = {wa.x, wa.y, wa.z, wa.w, wq.x, wq.y, wq.z, wq.w};
                const float b8[8] = {ba.x, ba.y, ba.z, ba.w, bq.x, bq.y, bq.z, bq.w};
                uint32_t f0[4], f1[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = 8 * c8 + 2 * q;
                    float h0, h1;
                    upk2(fma2_rn(pk2(w8[2 * q], w8[2 * q + 1]), xx, pk2(b8[2 * q], b8[2 * q + 1])), h0, h1);
                    const float e0 = (valid && h0 > 0.0f) ? d[j] : 0.0f;
                    const float e1 = (valid && h1 > 0.0f) ? d[j + 1] : 0.0f;
                    gx = __fmaf_rn(e0, w8[2 * q], gx);
                    gx = __fmaf_rn(e1, w8[2 * q + 1], gx);
                    split2(e0, e1, f0[q], f1[q]);
                }
                const uint32_t o = c8 * CH_ACT + t * 16;
                st16(R + O_R3 + o, f0[0], f0[1], f0[2], f0[3]);
                st16(R + O_R3 + PART + o, f1[0], f1[1], f1[2], f1[3]);
            }
            if (g.gx && valid) g.gx[i] = gx;
        }
        fence_async_smem();
        tc_fence_before();
        gsync(bid);
        tc_fence_after();
        // db1 += D1^T 1, dW1 += D1^T x; completion is awaited with the next commit
        if (t == 0 && !dead) {
#pragma unroll
            for (int ks = 0; ks < GM / 16; ++ks)
                mma_bf16(tb + C_V1, mndesc(rb + O_R3 + ks * 256, CH_ACT), mndesc(rb + O_V + ks * 256, CH_ACT),
                         I_VEC, (!first || ks) ? 1u : 0u);
        }
        first = false;
    }
    if (t == 0 && !dead && !first) {
        mma_commit(mybar);
        if (!mbar_wait(mybar, phase)) {
            dead = true;
            dead_parity = phase;
            err |= ERR_TIMEOUT;
        }
        phase ^= 1u;
        tc_fence_before();
    }
    dead = gor(bid, dead);
    tc_fence_after();

    // per-lane sums of the part products: lane r < 64 holds the hi-part row r, lane 64 + r the mid
    float *Q = reinterpret_cast<float *>(R);
    float *q = Q + t * QW;
    if (!dead && !first) {
#pragma unroll
        for (int c16 = 0; c16 < GH / 16; ++c16) {
            float a[16], b[16];
            tmem_ld16(lane_addr + C_W2 + 16 * c16, a);
            tmem_ld16(lane_addr + C_W2 + GH + 16 * c16, b);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) q[16 * c16 + j] = __fadd_rn(a[j], b[j]);
        }
        float a[16], b[16], v[16];
        tmem_ld16(lane_addr + C_B2, a);
        tmem_ld16(lane_addr + C_W3, b);
        tmem_ld16(lane_addr + C_V1, v);
        tmem_wait_ld();
        q[GH] = a[0];
        q[GH + 1] = b[0];
        q[GH + 2] = v[0];
        q[GH + 3] = __fadd_rn(v[1], v[2]);
    } else {
        for (int j = 0; j < GH + 4; ++j) q[j] = 0.0f;
    }
    q[GH + 4] = pgy;
    q[GH + 5] = plv;
    tc_fence_before();
    gsync(bid);
    float *out = g.partials + ((size_t)blockIdx.x * GNG + grp) * GP;
    for (int e = t; e < GH * GH; e += GM) {
        const int k = e / GH, j = e % GH;
        out[2 * GH + e] = __fadd_rn(Q[k * QW + j], Q[(GH + k) * QW + j]);
    }
    if (t < GH) {
        out[2 * GH + GH * GH + t] = __fadd_rn(Q[t * QW + GH], Q[(GH + t) * QW + GH]);          // b2
        out[3 * GH + GH * GH + t] = __fadd_rn(Q[t * QW + GH + 1], Q[(GH + t) * QW + GH + 1]);  // W3
        out[GH + t] = __fadd_rn(Q[t * QW + GH + 2], Q[(GH + t) * QW + GH + 2]);                // b1
        out[t] = __fadd_rn(Q[t * QW + GH + 3], Q[(GH + t) * QW + GH + 3]);                     // W1
    } else if (t == GH) {
        float s = 0.0f;
        for (int r = 0; r < GM; ++r) s = __fadd_rn(s, Q[r * QW + GH + 4]);
        out[GP - 1] = s;  // b3
    } else if (t == GH + 1 && g.loss_partials) {
        float s = 0.0f;
        for (int r = 0; r < GM; ++r) s = __fadd_rn(s, Q[r * QW + GH + 5]);
        g.loss_partials[(size_t)blockIdx.x * GNG + grp] = s;
    }
    if (err) atomicOr(&g_train_err, err);
    // an MMA whose completion was not seen may still be running: wait for it (bounded) before the
    // tensor memory it writes is released
    if (dead && t == 0) mbar_wait(mybar, dead_parity);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_free<GNG * GCOLS>(tmem_base);
}

}  // namespace

int grad_tc64_blocks(uint64_t nsamples) {
    const uint64_t chunks = (nsamples + GM - 1) / GM;
    return (int)std::max<uint64_t>(1, std::min<uint64_t>((chunks + GNG - 1) / GNG, MAX_BLOCKS));
}

cudaError_t launch_grad_tc64(const GradArgs &g, cudaStream_t s) {
    const int blocks = grad_tc64_blocks(g.n);
    cudaError_t e = cudaFuncSetAttribute(k_grad_tc64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    k_grad_tc64<<<blocks, GTHREADS, SMEM_BYTES, s>>>(g);
    e = cudaGetLastError();
    if (e == cudaSuccess) note_launch(1);
    return e;
}

uint32_t *train_err_word() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_train_err) != cudaSuccess) return nullptr;
    return reinterpret_cast<uint32_t *>(p);
}

}  // namespace nns
