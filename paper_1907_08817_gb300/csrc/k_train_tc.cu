// k_train_tc.cu -- the gradient of one training step (Sec. "Training", Eq. (loss)) of the model with
// two hidden layers of width 64, its matrix products on the fifth-generation tensor cores
// (tcgen05.mma kind::f16: BF16 operands, FP32 accumulation in tensor memory).
//
// Binary32 operands enter the products as sums of BF16 parts: v = v0 + v1 (+ v2), each part the
// BF16 rounding of what the earlier parts leave, so two parts carry 16 significant bits and three
// carry the 24 of binary32. Part products are exact in FP32 and accumulate in tensor memory; the
// smallest are issued first so that they meet a small accumulator.
//
// A block holds two groups of eight warps; a group takes chunks of 128 samples (one sample per
// tensor-memory lane, two threads per sample, each with half of the 64 units) and, per chunk:
//   1. layer 1 on the CUDA cores, binary32 FMA and ReLU as in the forward pass; H1 = three parts;
//   2. Z = H1 W2^T: the six part products whose weight is at least 2^-24 (W2 in three parts,
//      staged once per block);
//   3. per sample: z = Z + b2, h2 = ReLU(z), y = b3 + W3 . h2 (the two halves' sums meet in tensor
//      memory), the loss derivative gy, and the rows D2 = [z > 0] gy W3 and G = gy h2 (two parts
//      each);
//   4. D1pre = D2 W2 (the three part products of weight >= 2^-8); the sums over samples
//      dW2 += D2^T H1 (hi and mid parts of both stacked into one 128 x 128 product, four part
//      products), db2 += D2^T 1 and dW3 += G^T 1;
//   5. D1 = [W1 x + b1 > 0] D1pre (two parts); db1 += D1^T 1 and dW1 += D1^T x (x in two parts).
// Every row a thread writes (one sample's units) is read by the products over units as a K-major
// operand and by the products over samples as an MN-major one, so nothing is transposed. The sums
// over samples stay in tensor memory across the group's chunks; at the end the block adds its two
// groups' sums (group 0 first) into one partial gradient row, summed over blocks in a fixed order by
// the reduction. Chunks go to groups round-robin, so the result does not depend on timing.
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
constexpr int GM = 128;                     // samples per chunk = MMA rows
constexpr int GU = GH / 2;                  // units per thread
constexpr int GT = 2 * GM;                  // threads per group
constexpr int GNG = 2;                      // groups per block
constexpr int GTHREADS = GNG * GT;
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
static_assert(SMEM_BYTES <= 232448 - 64, "one block per SM");
// tensor-memory columns of a group (two groups: 512 columns); C_X: the halves' partial sums
constexpr uint32_t C_Z = 0, C_W2 = 64, C_B2 = 192, C_W3 = 208, C_V1 = 224, C_X = 240, GCOLS = 256;
constexpr int QW = 70;                      // row stride of the final per-lane sums (floats)
static_assert((uint32_t)GM * QW * 4 <= GROUP_BYTES, "final sums fit the group region");
constexpr int MAX_BLOCKS = 152;             // one block per SM of a 152-SM GPU

constexpr uint32_t I_ZK = idesc_bf16(GM, GH);               // A, B K-major
constexpr uint32_t I_D1 = idesc_bf16(GM, GH, false, true);  // B MN-major
constexpr uint32_t I_W2 = idesc_bf16(GM, 2 * GH, true, true);
constexpr uint32_t I_VEC = idesc_bf16(GM, 16, true, true);

__device__ __forceinline__ uint64_t kdesc(uint32_t addr, uint32_t ch) { return mdesc(addr, ch, 128); }
__device__ __forceinline__ uint64_t mndesc(uint32_t addr, uint32_t ch) { return mdesc(addr, 128, ch); }
// the descriptor of the matrix `bytes` further on: the start-address field (address / 16, bits 0-13)
// of a base below 256 KB does not carry into the next field
__device__ __forceinline__ uint64_t at(uint64_t desc, uint32_t bytes) { return desc + (uint64_t)(bytes >> 4); }

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
    asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(GT) : "memory");
}
__device__ __forceinline__ bool gor(int id, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "n"(GT)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    tmem_ld16(taddr, v);
    tmem_ld16(taddr + 16, v + 16);
    tmem_wait_ld();
}
// a + b of two threads of a sample, through two tensor-memory columns (a group barrier)
__device__ __forceinline__ void halves_sum(uint32_t col, int hf, float mine, float &h0, float &h1, int bid) {
    tmem_st1(col + hf, mine);
    tmem_wait_st();
    tc_fence_before();
    gsync(bid);
    tc_fence_after();
    tmem_ld2(col, h0, h1);
    tmem_wait_ld();
}

// per-thread state of a group's MMA pipeline, kept from one gradient pass to the next.
// last_bar / last_par: the barrier and phase of the latest commit; once a wait gave up (dead),
// waiting for that phase covers every MMA still in flight
struct Pipe {
    uint32_t tmem, bar, bar2;   // the block's tensor memory; this group's two mbarriers
    uint32_t phase, phase2, err, last_bar, last_par;
    bool dead;
};

// One gradient pass of the block over the batch of g: the block's partial gradient row (out) and
// loss partial (loss_out, nullable). Every thread of the block calls it.
__device__ __forceinline__ void grad_pass(const GradArgs &g, unsigned char *sm, Pipe &pp, float *out,
                                          float *loss_out) {
    float *par = reinterpret_cast<float *>(sm + OFF_PAR);
    const float4 *pv = reinterpret_cast<const float4 *>(par);
    const int tid = threadIdx.x, grp = tid / GT, gt = tid % GT;
    // thread (sample s, half hf): warps 0-3 of the group take units 0-31, warps 4-7 units 32-63;
    // warp w reads tensor-memory lanes 32 (w % 4) ..
    const int wq = (gt >> 5) & 3, hf = gt >> 7, s = wq * 32 + (gt & 31), u0 = hf * GU;
    const uint64_t nchunks = (g.n + GM - 1) / GM;
    const uint64_t ngroups = (uint64_t)gridDim.x * GNG;
    // this thread's sample inputs, loaded one chunk ahead (the first while the
    // parameters are staged)
    auto load_inputs = [&](uint64_t c, float &x, float &lab, float &gyin) {
        const uint64_t i = c * GM + s;
        x = 0.0f; lab = 0.0f; gyin = 0.0f;
        if (c < nchunks && i < g.n) {
            uint64_t src = i;
            if (g.mode == 2) src = __umul64hi(rng_draw(g.bseed, g.bofs + i), g.S);
            x = g.x[src];
            if (g.mode != 0) lab = g.label[src];
            else gyin = g.gy[i];
        }
    };
    uint64_t c = (uint64_t)blockIdx.x * GNG + grp;
    float nx, nlab, ngy;
    load_inputs(c, nx, nlab, ngy);
    {   // W2 as three BF16 parts; the vectors in binary32; the zero columns 8..15 of V
        const float *P = g.params;
        for (int e = tid; e < GH * GH; e += GTHREADS) {
            const int k = e / GH, j = e % GH;
            const float w = __ldcg(P + 2 * GH + e);
            const __nv_bfloat16 p0 = __float2bfloat16_rn(w);
            const float r = __fsub_rn(w, __bfloat162float(p0));
            const __nv_bfloat16 p1 = __float2bfloat16_rn(r);
            const __nv_bfloat16 p2 = __float2bfloat16_rn(__fsub_rn(r, __bfloat162float(p1)));
            unsigned char *o = sm + OFF_W + (j / 8) * CH_W + k * 16 + (j % 8) * 2;
            *reinterpret_cast<__nv_bfloat16 *>(o) = p0;
            *reinterpret_cast<__nv_bfloat16 *>(o + WPART) = p1;
            *reinterpret_cast<__nv_bfloat16 *>(o + 2 * WPART) = p2;
        }
        // (read through L2: in a persistent launch other blocks update the parameters between passes)
        for (int e = tid; e < GH; e += GTHREADS) {
            par[e] = __ldcg(P + e);                              // W1
            par[GH + e] = __ldcg(P + GH + e);                    // b1
            par[2 * GH + e] = __ldcg(P + 2 * GH + GH * GH + e);  // b2
            par[3 * GH + e] = __ldcg(P + 3 * GH + GH * GH + e);  // W3
        }
        if (tid == 0) par[4 * GH] = __ldcg(P + 4 * GH + GH * GH);  // b3
        for (int e = tid; e < GNG * GM; e += GTHREADS)
            st16(sm + OFF_GRP + (e / GM) * GROUP_BYTES + O_V + CH_ACT + (e % GM) * 16, 0u, 0u, 0u, 0u);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const uint32_t tb = pp.tmem + (uint32_t)(grp * GCOLS);
    const uint32_t lane_base = tb + ((uint32_t)(wq * 32) << 16);
    unsigned char *R = sm + OFF_GRP + grp * GROUP_BYTES;
    const uint32_t rb = smem_u32(R), wb = smem_u32(sm + OFF_W);
    const uint32_t mybar = pp.bar, mybar2 = pp.bar2;
    const int bid = 1 + grp;
    // warp 0 of the group issues the MMAs (one elected lane) and waits for them
    const bool issuer = (gt >> 5) == 0;
    const float b3 = par[4 * GH];
    // descriptor bases: activations K-major (KA) and MN-major (MA), W2 K-major (KW) and MN-major (MW)
    const uint64_t KA = kdesc(rb, CH_ACT), MA = mndesc(rb, CH_ACT), KW = kdesc(wb, CH_W), MW = mndesc(wb, CH_W);
    uint32_t phase = pp.phase, phase2 = pp.phase2, err = pp.err, last_bar = pp.last_bar, last_par = pp.last_par;
    bool dead = pp.dead, first = true;
    float pgy = 0.0f, plv = 0.0f;
    for (; c < nchunks; c += ngroups) {
        const uint64_t i = c * GM + s;
        const bool valid = i < g.n;
        const float x = nx, lab = nlab, gyin = ngy;
        load_inputs(c + ngroups, nx, nlab, ngy);
        const unsigned long long xx = pk2(x, x);

        // 1. H1 = ReLU(W1 x + b1), three parts (this thread: units u0 .. u0 + 31)
#pragma unroll
        for (int c8 = 0; c8 < GU / 8; ++c8) {
            const int j0 = u0 + 8 * c8;
            const float4 wa = pv[j0 / 4], wq4 = pv[j0 / 4 + 1];
            const float4 ba = pv[GH / 4 + j0 / 4], bq = pv[GH / 4 + j0 / 4 + 1];
            const float w8[8] = {wa.x, wa.y, wa.z, wa.w, wq4.x, wq4.y, wq4.z, wq4.w};
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
            const uint32_t o = (j0 / 8) * CH_ACT + s * 16;
            st16(R + O_H1 + o, p0[0], p0[1], p0[2], p0[3]);
            st16(R + O_H1 + PART + o, p1[0], p1[1], p1[2], p1[3]);
            st16(R + O_R1 + o, p2[0], p2[1], p2[2], p2[3]);
        }
        fence_async_smem();
        tc_fence_before();
        gsync(bid);
        tc_fence_after();

        // 2. Z = H1 W2^T (this commit also covers the previous chunk's column sums)
        if (issuer && !dead) {
            constexpr uint32_t ha[3] = {O_H1, O_H1 + PART, O_R1};
            constexpr int pa[6] = {2, 0, 1, 1, 0, 0}, pb[6] = {0, 2, 1, 0, 1, 0};
#pragma unroll
            for (int pr = 0; pr < 6; ++pr)
#pragma unroll
                for (int ks = 0; ks < GH / 16; ++ks)
                    mma_bf16_warp(tb + C_Z, at(KA, ha[pa[pr]] + ks * 2 * CH_ACT), at(KW, pb[pr] * WPART + ks * 2 * CH_W),
                             I_ZK, (pr | ks) ? 1u : 0u);
            mma_commit_warp(mybar);
            last_bar = mybar;
            last_par = phase;
            if (__any_sync(0xFFFFFFFFu, !mbar_wait(mybar, phase))) {
                dead = true;
                err |= ERR_TIMEOUT;
            }
            phase ^= 1u;
            tc_fence_before();
        }
        dead = gor(bid, dead);
        tc_fence_after();

        // 3. output, loss derivative, D2 and G rows
        float z[GU];
        if (!dead) {
            tmem_ld32(lane_base + C_Z + u0, z);
        } else {
#pragma unroll
            for (int k = 0; k < GU; ++k) z[k] = 0.0f;
        }
        unsigned long long yy = pk2(0.0f, 0.0f);
#pragma unroll
        for (int k4 = 0; k4 < GU / 4; ++k4) {
            const float4 b2q = pv[GH / 2 + u0 / 4 + k4], w3q = pv[3 * GH / 4 + u0 / 4 + k4];
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
        float ye, yo, y0, y1;
        upk2(yy, ye, yo);
        halves_sum(lane_base + C_X, hf, __fadd_rn(ye, yo), y0, y1, bid);
        float gy = 0.0f, lv = 0.0f;
        if (valid) {
            if (g.mode == 0) {
                gy = gyin;
            } else {
                const float r = __fsub_rn(__fadd_rn(__fadd_rn(b3, y0), y1), lab);
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
        if (hf == 0) {
            pgy = __fadd_rn(pgy, gy);
            plv = __fadd_rn(plv, lv);
        }
        {
            const unsigned long long gg = pk2(gy, gy);
#pragma unroll
            for (int c8 = 0; c8 < GU / 8; ++c8) {
                uint32_t d0[4], d1[4], e0[4], e1[4];
#pragma unroll
                for (int q2 = 0; q2 < 2; ++q2) {
                    const int k = 8 * c8 + 4 * q2;
                    const float4 w3q = pv[3 * GH / 4 + (u0 + k) / 4];
                    float a, b, a2, b2v;
                    upk2(mul2_rn(gg, pk2(w3q.x, w3q.y)), a, b);
                    upk2(mul2_rn(gg, pk2(w3q.z, w3q.w)), a2, b2v);
                    split2(z[k] > 0.0f ? a : 0.0f, z[k + 1] > 0.0f ? b : 0.0f, d0[2 * q2], d1[2 * q2]);
                    split2(z[k + 2] > 0.0f ? a2 : 0.0f, z[k + 3] > 0.0f ? b2v : 0.0f, d0[2 * q2 + 1], d1[2 * q2 + 1]);
                    upk2(mul2_rn(gg, pk2(z[k], z[k + 1])), a, b);
                    split2(a, b, e0[2 * q2], e1[2 * q2]);
                    upk2(mul2_rn(gg, pk2(z[k + 2], z[k + 3])), a, b);
                    split2(a, b, e0[2 * q2 + 1], e1[2 * q2 + 1]);
                }
                const uint32_t o = ((u0 + 8 * c8) / 8) * CH_ACT + s * 16;
                st16(R + O_R1 + o, d0[0], d0[1], d0[2], d0[3]);
                st16(R + O_R1 + PART + o, d1[0], d1[1], d1[2], d1[3]);
                st16(R + O_R3 + o, e0[0], e0[1], e0[2], e0[3]);
                st16(R + O_R3 + PART + o, e1[0], e1[1], e1[2], e1[3]);
            }
            if (hf == 0) {
                uint32_t xh, xm;
                split2(x, 0.0f, xh, xm);
                // columns: 0 = 1 (valid samples), 1 = x hi, 2 = x mid
                st16(R + O_V + s * 16, (valid ? 0x3F80u : 0u) | (xh << 16), xm & 0xFFFFu, 0u, 0u);
            }
        }
        fence_async_smem();
        tc_fence_before();
        gsync(bid);
        tc_fence_after();

        // 4. dW3 += G^T 1 and D1pre = D2 W2, awaited (phase 5 needs D1pre and overwrites G); then
        //    dW2 += D2^T H1 and db2 += D2^T 1, which run during phase 5 (completion: bar2)
        if (issuer && !dead) {
#pragma unroll
            for (int ks = 0; ks < GM / 16; ++ks)
                mma_bf16_warp(tb + C_W3, at(MA, O_R3 + ks * 256), at(MA, O_V + ks * 256), I_VEC, (!first || ks) ? 1u : 0u);
            // the three part products of weight >= 2^-8 (the rest is below 2^-16 of D1pre)
            constexpr int qa[3] = {1, 0, 0}, qb[3] = {0, 1, 0};
#pragma unroll
            for (int pr = 0; pr < 3; ++pr)
#pragma unroll
                for (int ks = 0; ks < GH / 16; ++ks)
                    mma_bf16_warp(tb + C_Z, at(KA, O_R1 + qa[pr] * PART + ks * 2 * CH_ACT), at(MW, qb[pr] * WPART + ks * 256),
                             I_D1, (pr | ks) ? 1u : 0u);
            mma_commit_warp(mybar);
#pragma unroll
            for (int ks = 0; ks < GM / 16; ++ks) {
                const uint32_t acc = (!first || ks) ? 1u : 0u;
                const uint64_t d2 = at(MA, O_R1 + ks * 256);
                mma_bf16_warp(tb + C_W2, d2, at(MA, O_H1 + ks * 256), I_W2, acc);
                mma_bf16_warp(tb + C_B2, d2, at(MA, O_V + ks * 256), I_VEC, acc);
            }
            mma_commit_warp(mybar2);
            last_bar = mybar2;
            last_par = phase2;
            if (__any_sync(0xFFFFFFFFu, !mbar_wait(mybar, phase))) {
                dead = true;
                err |= ERR_TIMEOUT;
            }
            phase ^= 1u;
            tc_fence_before();
        }
        dead = gor(bid, dead);
        tc_fence_after();

        // 5. D1 = [W1 x + b1 > 0] D1pre rows; the input gradient
        {
            float d[GU];
            if (!dead) {
                tmem_ld32(lane_base + C_Z + u0, d);
            } else {
#pragma unroll
                for (int k = 0; k < GU; ++k) d[k] = 0.0f;
            }
            float gx = 0.0f;
#pragma unroll
            for (int c8 = 0; c8 < GU / 8; ++c8) {
                const int j0 = u0 + 8 * c8;
                const float4 wa = pv[j0 / 4], wq4 = pv[j0 / 4 + 1];
                const float4 ba = pv[GH / 4 + j0 / 4], bq = pv[GH / 4 + j0 / 4 + 1];
                const float w8[8] = {wa.x, wa.y, wa.z, wa.w, wq4.x, wq4.y, wq4.z, wq4.w};
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
                const uint32_t o = (j0 / 8) * CH_ACT + s * 16;
                st16(R + O_R3 + o, f0[0], f0[1], f0[2], f0[3]);
                st16(R + O_R3 + PART + o, f1[0], f1[1], f1[2], f1[3]);
            }
            if (g.gx) {  // (uniform) the halves' sums meet in tensor memory
                float g0, g1;
                halves_sum(lane_base + C_X + 2, hf, gx, g0, g1, bid);
                if (valid && hf == 0) g.gx[i] = __fadd_rn(g0, g1);
            }
        }
        fence_async_smem();
        // the next chunk's H1 rows overwrite what dW2 += D2^T H1 reads
        if (issuer && !dead) {
            if (__any_sync(0xFFFFFFFFu, !mbar_wait(mybar2, phase2))) {
                dead = true;
                err |= ERR_TIMEOUT;
            }
            phase2 ^= 1u;
        }
        tc_fence_before();
        dead = gor(bid, dead);
        tc_fence_after();
        // db1 += D1^T 1, dW1 += D1^T x; completion is awaited with the next commit
        if (issuer && !dead) {
#pragma unroll
            for (int ks = 0; ks < GM / 16; ++ks)
                mma_bf16_warp(tb + C_V1, at(MA, O_R3 + ks * 256), at(MA, O_V + ks * 256), I_VEC, (!first || ks) ? 1u : 0u);
        }
        first = false;
    }
    if (issuer && !dead && !first) {
        mma_commit_warp(mybar);
        last_bar = mybar;
        last_par = phase;
        if (__any_sync(0xFFFFFFFFu, !mbar_wait(mybar, phase))) {
            dead = true;
            err |= ERR_TIMEOUT;
        }
        phase ^= 1u;
        tc_fence_before();
    }
    dead = gor(bid, dead);
    tc_fence_after();

    // per-lane sums of the part products: lane r < 64 holds the hi-part row r, lane 64 + r the mid
    float *Q = reinterpret_cast<float *>(R);
    float *q = Q + s * QW;
    if (!dead && !first) {
#pragma unroll
        for (int c16 = 0; c16 < GU / 16; ++c16) {
            float a[16], b[16];
            tmem_ld16(lane_base + C_W2 + u0 + 16 * c16, a);
            tmem_ld16(lane_base + C_W2 + GH + u0 + 16 * c16, b);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) q[u0 + 16 * c16 + j] = __fadd_rn(a[j], b[j]);
        }
        if (hf == 0) {
            float a[16], b[16], v[16];
            tmem_ld16(lane_base + C_B2, a);
            tmem_ld16(lane_base + C_W3, b);
            tmem_ld16(lane_base + C_V1, v);
            tmem_wait_ld();
            q[GH] = a[0];
            q[GH + 1] = b[0];
            q[GH + 2] = v[0];
            q[GH + 3] = __fadd_rn(v[1], v[2]);
        }
    } else {
        for (int j = 0; j < GU; ++j) q[u0 + j] = 0.0f;
        if (hf == 0)
            for (int j = GH; j < GH + 4; ++j) q[j] = 0.0f;
    }
    if (hf == 0) {
        q[GH + 4] = pgy;
        q[GH + 5] = plv;
    }
    tc_fence_before();
    __syncthreads();
    // one partial row per block: group 0's sums, then group 1's
    const float *Q0 = reinterpret_cast<const float *>(sm + OFF_GRP);
    const float *Q1 = reinterpret_cast<const float *>(sm + OFF_GRP + GROUP_BYTES);
    auto both = [&](int r, int col) {
        return __fadd_rn(__fadd_rn(Q0[r * QW + col], Q0[(GH + r) * QW + col]),
                         __fadd_rn(Q1[r * QW + col], Q1[(GH + r) * QW + col]));
    };
    for (int e = tid; e < GH * GH; e += GTHREADS) out[2 * GH + e] = both(e / GH, e % GH);
    if (tid < GH) {
        out[2 * GH + GH * GH + tid] = both(tid, GH);      // b2
        out[3 * GH + GH * GH + tid] = both(tid, GH + 1);  // W3
        out[GH + tid] = both(tid, GH + 2);                // b1
        out[tid] = both(tid, GH + 3);                     // W1
    } else if (tid == GH) {
        float s0 = 0.0f, s1 = 0.0f;
        for (int r = 0; r < GM; ++r) {
            s0 = __fadd_rn(s0, Q0[r * QW + GH + 4]);
            s1 = __fadd_rn(s1, Q1[r * QW + GH + 4]);
        }
        out[GP - 1] = __fadd_rn(s0, s1);  // b3
    } else if (tid == GH + 1 && loss_out) {
        float s0 = 0.0f, s1 = 0.0f;
        for (int r = 0; r < GM; ++r) {
            s0 = __fadd_rn(s0, Q0[r * QW + GH + 5]);
            s1 = __fadd_rn(s1, Q1[r * QW + GH + 5]);
        }
        *loss_out = __fadd_rn(s0, s1);
    }
    pp.phase = phase;
    pp.phase2 = phase2;
    pp.err = err;
    pp.last_bar = last_bar;
    pp.last_par = last_par;
    pp.dead = dead;
    __syncthreads();  // the sums are read before the next pass writes the group regions
}

__device__ __forceinline__ void pipe_open(Pipe &pp, uint32_t *tmem_slot, unsigned long long *bars) {
    const int tid = threadIdx.x, grp = tid / GT;
    if ((tid >> 5) == 0) tmem_alloc<GNG * GCOLS>(smem_u32(tmem_slot));
    if (tid == 0) {
        for (int q = 0; q < 2 * GNG; ++q) mbar_init(smem_u32(&bars[q]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pp.tmem = *tmem_slot;
    pp.bar = smem_u32(&bars[grp]);
    pp.bar2 = smem_u32(&bars[GNG + grp]);
    pp.phase = pp.phase2 = pp.err = pp.last_par = 0;
    pp.last_bar = pp.bar;
    pp.dead = false;
}

__device__ __forceinline__ void pipe_close(Pipe &pp) {
    if (pp.err) atomicOr(&g_train_err, pp.err);
    // an MMA whose completion was not seen may still be running: wait for it (bounded) before the
    // tensor memory it writes is released
    if (pp.dead && (threadIdx.x % GT) < 32) mbar_wait(pp.last_bar, pp.last_par);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if ((threadIdx.x >> 5) == 0) tmem_free<GNG * GCOLS>(pp.tmem);
}

// one gradient of the batch: partial row and loss partial per block
__global__ void __launch_bounds__(GTHREADS, 1) k_grad_tc64(GradArgs g) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) unsigned long long bars[2 * GNG];
    __shared__ uint32_t tmem_slot;
    Pipe pp;
    pipe_open(pp, &tmem_slot, bars);
    grad_pass(g, sm, pp, g.partials + (size_t)blockIdx.x * GP,
              g.loss_partials ? g.loss_partials + blockIdx.x : nullptr);
    pipe_close(pp);
}

// ---- every Adam step of a training run in one cooperative launch
// Per step: the gradient pass (one partial row per block), a grid-wide meeting, the fixed-order sum
// of the rows and the Adam update of this block's parameter groups (32 parameters each, groups
// assigned round-robin; the owner of group 0 also sums the loss), another meeting, so the next pass
// reads the updated parameters.
struct TrainTcArgs {
    GradArgs g;                // n = batch; bofs of step t = t * n
    float *params;             // = g.params, updated in place
    float *m, *v;              // Adam moments
    const float *mask;         // nullable: sign a parameter must keep (monotone training)
    const float *c12;          // [2 * steps]: 1 - beta1^(t+1), then 1 - beta2^(t+1)
    float *loss_out;           // [steps]
    float loss_scale, lr, b1, b2, eps;
    int steps;
    unsigned int *count;       // arrivals at the grid meetings (zero before the launch)
};
constexpr int NGRP = (GP + 31) / 32;  // parameter groups

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// All blocks of the launch meet (they are co-resident: cooperative launch). The arrival count only
// grows: meeting k is complete when it reaches k * gridDim.x. The block's earlier global writes are
// released with the arrival (after the block barrier) and acquired by every block that sees the
// count complete. False when the wait gave up after the library's spin limit.
__device__ __forceinline__ bool grid_meet(unsigned int *count, unsigned int &target) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        target += gridDim.x;
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(count), "r"(1u) : "memory");
        const unsigned long long t0 = globaltimer_ns();
        uint32_t polls = 0;
        while (ld_acquire_u32(count) < target) {
            if (globaltimer_ns() - t0 > SPIN_LIMIT_NS || ++polls > SPIN_LIMIT_POLLS) {
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

constexpr int RW = GTHREADS / 32;  // warps of the reduction

// the fixed-order sum of the partial rows and Adam, for this block's parameter groups
__device__ __forceinline__ void reduce_adam(const TrainTcArgs &a, int step, float (*red)[33]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nb = gridDim.x;
    const float c1 = a.c12[step], c2 = a.c12[a.steps + step];
    for (int pg = blockIdx.x; pg < NGRP; pg += nb) {
        const int p = pg * 32 + lane;
        float acc = 0.0f;
        for (int r0 = w; r0 < nb; r0 += RW * 8) {
            float t[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int r = r0 + RW * q;
                t[q] = (p < GP && r < nb) ? __ldcg(a.g.partials + (size_t)r * GP + p) : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (r0 + RW * q < nb) acc = __fadd_rn(acc, t[q]);
        }
        red[w][lane] = acc;
        __syncthreads();
        if (w == 0 && p < GP) {
            float gsum = 0.0f;
            for (int q = 0; q < RW; ++q) gsum = __fadd_rn(gsum, red[q][lane]);
            const float m = a.b1 * a.m[p] + (1.0f - a.b1) * gsum;
            const float v = a.b2 * a.v[p] + (1.0f - a.b2) * gsum * gsum;
            a.m[p] = m;
            a.v[p] = v;
            const float mh = m / c1, vh = v / c2;
            float np = a.params[p] - a.lr * mh / (sqrtf(vh) + a.eps);
            if (a.mask && a.mask[p] * np < 0.0f) np = 0.0f;  // monotone projection
            a.params[p] = np;
        }
        if (pg == 0 && a.loss_out) {  // the loss
            __syncthreads();
            float l = 0.0f;
            if (lane == 0)
                for (int r = w; r < nb; r += RW) l = __fadd_rn(l, __ldcg(a.g.loss_partials + r));
            red[w][0] = l;
            __syncthreads();
            if (threadIdx.x == 0) {
                float sum = 0.0f;
                for (int q = 0; q < RW; ++q) sum = __fadd_rn(sum, red[q][0]);
                a.loss_out[step] = sum * a.loss_scale;
            }
        }
        __syncthreads();  // red is rewritten by the next group
    }
}

__global__ void __launch_bounds__(GTHREADS, 1) k_train_tc64(TrainTcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) unsigned long long bars[2 * GNG];
    __shared__ uint32_t tmem_slot;
    // the reduction's scratch: group 0's region, free between passes
    float(*red)[33] = reinterpret_cast<float(*)[33]>(sm + OFF_GRP);
    Pipe pp;
    pipe_open(pp, &tmem_slot, bars);
    unsigned int target = 0;
    for (int step = 0; step < a.steps; ++step) {
        GradArgs g = a.g;
        g.bofs = (uint64_t)step * g.n;
        grad_pass(g, sm, pp, g.partials + (size_t)blockIdx.x * GP, g.loss_partials + blockIdx.x);
        if (!grid_meet(a.count, target)) {
            pp.err |= ERR_TIMEOUT;
            break;
        }
        reduce_adam(a, step, red);
        if (!grid_meet(a.count, target)) {
            pp.err |= ERR_TIMEOUT;
            break;
        }
    }
    pipe_close(pp);
}

}  // namespace

int grad_tc64_blocks(uint64_t nsamples) {  // one partial row per block
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

cudaError_t launch_train_tc64(const TrainStepArgs &t, uint32_t steps, const float *c12, unsigned int *count,
                              cudaStream_t s) {
    if (steps == 0) return cudaSuccess;
    const uint64_t B = t.batch ? t.batch : t.S;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_train_tc64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_train_tc64, GTHREADS, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    // every block must be resident at once: the blocks meet twice per step
    const int blocks = std::min(grad_tc64_blocks(B), per_sm * sms);
    if (blocks < 1) return cudaErrorCooperativeLaunchTooLarge;
    TrainTcArgs a{};
    a.g.params = t.params; a.g.x = t.x; a.g.label = t.label; a.g.n = B; a.g.S = t.S;
    a.g.bseed = t.batch_seed; a.g.bofs = 0; a.g.mode = t.batch ? 2 : 1; a.g.loss = t.loss;
    a.g.delta = t.delta; a.g.inv_n = 1.0f / (float)B; a.g.partials = t.partials;
    a.g.loss_partials = t.loss_partials; a.g.gx = nullptr;
    a.params = t.params; a.m = t.m; a.v = t.v; a.mask = t.mask; a.c12 = c12; a.loss_out = t.loss_out;
    a.loss_scale = 1.0f / (float)B; a.lr = t.lr; a.b1 = t.b1; a.b2 = t.b2; a.eps = t.eps;
    a.steps = (int)steps; a.count = count;
    void *args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void *)k_train_tc64, dim3((unsigned)blocks), dim3(GTHREADS), args,
                                    SMEM_BYTES, s);
    if (e == cudaSuccess) note_launch(1);
    return e;
}

uint32_t *train_err_word() {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_train_err) != cudaSuccess) return nullptr;
    return reinterpret_cast<uint32_t *>(p);
}

}  // namespace nns
