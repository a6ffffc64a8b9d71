// common.cuh -- device-side building blocks shared by the NN-sort kernels (sm_103a).
//
// Bit-defined pieces (key order, translate, binary32 forward pass, position rounding) state the
// method's arithmetic as a fixed sequence of IEEE operations written with explicit _rn intrinsics
// so that the compiler cannot contract or reorder them.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "nnsort.h"

namespace nns {

constexpr int MAXR = NNSORT_MAX_ROUNDS;
constexpr int MAXH = NNSORT_MAX_HIDDEN;
constexpr uint32_t EMPTY32 = 0xFFFFFFFFu;
constexpr uint16_t EMPTY16 = 0xFFFFu;

// device error word bits
enum : uint32_t { ERR_NAN = 1u, ERR_TIMEOUT = 2u, ERR_SLOT = 4u, ERR_INTERNAL = 8u };

// normaliser of translate(A) (Sec. "Input Phase")
struct Norm {
    int32_t dtype, translate;
    uint64_t lo_bits;
    double lo_val, scale;
    float lo_f, scale_f;
};

// One array of a (batched) sort. Element space: the arrays concatenated; slot space: each array's
// positions [0, L) shifted by gs_base, a multiple of the bucket width W = 2^wlog.
struct Seg {
    void *keys;          // caller's device keys
    int32_t *payload;    // caller's device payload or null
    uint64_t n;          // elements
    uint64_t ebase;      // first element in the element space
    uint64_t L;          // positions floor(n m) + 1
    uint64_t gs_base;    // first global position
    uint32_t bbase, nb;  // first bucket, bucket count
    uint32_t tbase, ntiles;  // predict tiles
    float nm_hi, nm_lo;  // n*m as an unevaluated binary32 sum
    uint32_t eps;
    uint64_t tau;
    const float *params; // padded binary32 parameters of this array's model (null: injected)
    const uint32_t *slots;  // injected positions (null: model)
    Norm norm;
};

// per-array device statistics
struct SegStats {
    unsigned long long count_ge[MAXR + 1];  // elements whose round index is >= r (r >= 1)
    unsigned long long ooo[MAXR];           // out-of-order inserts of o_r
    unsigned long long repaired;             // elements in the seam repair ranges
    unsigned int t;                          // completed iterations
    unsigned int oversized;
    unsigned int ranges;                     // seam repair ranges
    unsigned int pad;
};

// (order image, tie-break) pair; the maximum of an empty set is {0, 0, 0}
struct OKey {
    unsigned long long k;
    unsigned int tb;
    unsigned int valid;
};

__device__ __forceinline__ bool okey_less(unsigned long long ka, unsigned int ta,
                                          unsigned long long kb, unsigned int tbb) {
    return ka < kb || (ka == kb && ta < tbb);
}

// ---------------------------------------------------------------------------------------------
// key order: IEEE floats -> unsigned integers in numeric order (-0.0 before +0.0)
__device__ __forceinline__ uint64_t ordbits(uint64_t w, int dtype) {
    if (dtype == NNSORT_F32) {
        const uint32_t b = (uint32_t)w;
        return (b & 0x80000000u) ? (uint64_t)(uint32_t)(~b) : (uint64_t)(b | 0x80000000u);
    }
    if (dtype == NNSORT_F64) return (w >> 63) ? ~w : (w | 0x8000000000000000ull);
    return w;
}

__device__ __forceinline__ bool key_is_nan(uint64_t w, int dtype) {
    if (dtype == NNSORT_F32) return ((uint32_t)w & 0x7FFFFFFFu) > 0x7F800000u;
    if (dtype == NNSORT_F64) return (w & 0x7FFFFFFFFFFFFFFFull) > 0x7FF0000000000000ull;
    return false;
}

template <typename W> __device__ __forceinline__ uint64_t word64(W w) { return (uint64_t)w; }

// translate(A): the model input in binary32 (bit-identical to the CPU reference)
__device__ __forceinline__ float translate_x(uint64_t w, const Norm &nm) {
    const int dt = nm.dtype;
    const bool ob = nm.translate == NNSORT_TRANSLATE_ORDBITS || dt == NNSORT_U32 || dt == NNSORT_U64;
    if (ob) {
        const uint64_t u = ordbits(w, dt);
        const float d = (u >= nm.lo_bits) ? __ull2float_rn(u - nm.lo_bits)
                                          : -__ull2float_rn(nm.lo_bits - u);
        return __fmul_rn(d, nm.scale_f);
    }
    if (dt == NNSORT_F32) {
        const float k = __uint_as_float((uint32_t)w);
        return __fmul_rn(__fsub_rn(k, nm.lo_f), nm.scale_f);
    }
    const double k = __longlong_as_double((long long)w);
    return __double2float_rn(__dmul_rn(__dsub_rn(k, nm.lo_val), nm.scale));
}

__device__ __forceinline__ float relu_f(float v) { return v > 0.0f ? v : 0.0f; }

// Two binary32 lanes per instruction (packed FP32 on sm_100 and later): each lane is rounded exactly
// as the scalar operation would be; the pair (lo, hi) travels as one 64-bit register.
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long fma2_rn(unsigned long long a, unsigned long long b,
                                                      unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ unsigned long long add2_rn(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long mul2_rn(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long sub2_rn(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// binary32 forward pass of the padded MLP (padding units have zero weights and biases, which
// leaves every partial sum of the real units unchanged). P points at the padded layout
// W1[H1] b1[H1] (W2[H2*H1] b2[H2])? W3[HL] b3.
template <int H1, int H2>
__device__ __forceinline__ float mlp_fwd_f32(const float *__restrict__ P, float x) {
    float h1[H1];
#pragma unroll
    for (int j = 0; j < H1; ++j) h1[j] = relu_f(__fmaf_rn(P[j], x, P[H1 + j]));
    if constexpr (H2 == 0) {
        const float *W3 = P + 2 * H1;
        float y = W3[H1];
#pragma unroll
        for (int k = 0; k < H1; ++k) y = __fmaf_rn(W3[k], h1[k], y);
        return y;
    } else {
        const float *W2 = P + 2 * H1;
        const float *b2 = W2 + H2 * H1;
        const float *W3 = b2 + H2;
        float y = W3[H2];
#pragma unroll 2
        for (int k = 0; k < H2; ++k) {
            const float4 *w4 = reinterpret_cast<const float4 *>(W2 + k * H1);
            float z = b2[k];
#pragma unroll
            for (int j = 0; j < H1 / 4; ++j) {
                const float4 w = w4[j];
                z = __fmaf_rn(w.x, h1[4 * j + 0], z);
                z = __fmaf_rn(w.y, h1[4 * j + 1], z);
                z = __fmaf_rn(w.z, h1[4 * j + 2], z);
                z = __fmaf_rn(w.w, h1[4 * j + 3], z);
            }
            y = __fmaf_rn(W3[k], relu_f(z), y);
        }
        return y;
    }
}

// position round(y * n * m) in binary32 with n*m = nm_hi + nm_lo (see the CPU reference):
// p = y nm_hi; e = fma(y, nm_hi, -p); e = fma(y, nm_lo, e); f = floor(p);
// slot = f + floor(((p - f) + e) + 0.5), clamped to [0, L-1]; y <= 0 or NaN -> 0; y capped at 1.
__device__ __forceinline__ uint32_t slot_of(float y, float nm_hi, float nm_lo, uint64_t L) {
    if (!(y > 0.0f)) return 0u;
    if (y > 1.0f) y = 1.0f;
    const float p = __fmul_rn(y, nm_hi);
    float e = __fmaf_rn(y, nm_hi, -p);
    e = __fmaf_rn(y, nm_lo, e);
    const float f = floorf(p);
    const float r = __fadd_rn(__fsub_rn(p, f), e);
    const float g = floorf(__fadd_rn(r, 0.5f));
    long long s = (long long)f + (long long)g;
    if (s < 0) s = 0;
    if ((unsigned long long)s > L - 1) s = (long long)(L - 1);
    return (uint32_t)s;
}

// ---------------------------------------------------------------------------------------------
// memory ordering helpers for decoupled look-back
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
// a 64-bit word read without ordering: enough when the word itself carries the flag and the value
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// every spin-wait in the library gives up after this long, or after this many polls (whichever
// comes first, so that a wait ends even if the timer were not to advance), and raises ERR_TIMEOUT
constexpr unsigned long long SPIN_LIMIT_NS = 4000000000ull;
constexpr uint32_t SPIN_LIMIT_POLLS = 1u << 26;

// SplitMix64 (Steele, Lea and Flood): draw i of the stream with seed `seed` (training samples and
// mini-batches)
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t rng_draw(uint64_t seed, uint64_t i) {
    return mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
}

// ---------------------------------------------------------------------------------------------
// block-wide exclusive sum of one u32 per thread (blockDim multiple of 32, <= 1024)
__device__ __forceinline__ uint32_t block_excl_sum(uint32_t v, uint32_t *scratch /*>= 33*/,
                                                   uint32_t *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = (lane < nw) ? scratch[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) scratch[lane] = s;
        if (lane == 31) scratch[32] = s;
    }
    __syncthreads();
    const uint32_t res = x - v + (wid > 0 ? scratch[wid - 1] : 0u);
    if (total) *total = scratch[32];
    __syncthreads();
    return res;
}

// block-wide inclusive/exclusive maximum of (key, tb) pairs; returns the exclusive prefix max
// (valid = 0 if none) and the block maximum through *tot.
struct KMax {
    unsigned long long k;
    unsigned int tb, valid;
};
__device__ __forceinline__ KMax kmax(const KMax &a, const KMax &b) {
    if (!a.valid) return b;
    if (!b.valid) return a;
    return okey_less(a.k, a.tb, b.k, b.tb) ? b : a;
}
__device__ __forceinline__ KMax shfl_up_kmax(const KMax &a, int o) {
    KMax r;
    r.k = __shfl_up_sync(0xFFFFFFFFu, a.k, o);
    r.tb = __shfl_up_sync(0xFFFFFFFFu, a.tb, o);
    r.valid = __shfl_up_sync(0xFFFFFFFFu, a.valid, o);
    return r;
}
__device__ __forceinline__ KMax block_excl_max(KMax v, KMax *scratch /*>= 33*/, KMax *tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    KMax x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const KMax y = shfl_up_kmax(x, o);
        if (lane >= o) x = kmax(y, x);
    }
    KMax ex = shfl_up_kmax(x, 1);
    if (lane == 0) ex.valid = 0;
    if (lane == 31) scratch[wid] = x;
    __syncthreads();
    if (wid == 0) {
        KMax s;
        if (lane < nw) s = scratch[lane]; else { s.k = 0; s.tb = 0; s.valid = 0; }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const KMax y = shfl_up_kmax(s, o);
            if (lane >= o) s = kmax(y, s);
        }
        if (lane < nw) scratch[lane] = s;
        if (lane == 31) scratch[32] = s;
    }
    __syncthreads();
    KMax res = ex;
    if (wid > 0) res = kmax(scratch[wid - 1], ex);
    if (tot) *tot = scratch[32];
    __syncthreads();
    return res;
}

}  // namespace nns
