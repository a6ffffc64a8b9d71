// pwl.cu -- the model f evaluated through its piecewise-linear form (NNSORT_PREC_PWL).
//
// With a one-dimensional input, a ReLU MLP is piecewise linear in x: each first-layer unit
// relu(W1_j x + b1_j) bends at x = -b1_j / W1_j; between two consecutive bends every second-layer
// pre-activation z_k(x) = sum_j W2_kj relu(W1_j x + b1_j) + b2_k is linear and adds at most one bend
// where it crosses zero; between all bends F(x) = s x + c. Compiling f (Fig. "Algorithm NN-sort",
// the map line; Sec. "Model" for the network) into these segments on the host, in binary64, gives
// F exactly up to rounding, i.e. the binary64 model.
//
// For a sort the bends are carried into the keys' order-image domain (a threshold per segment)
// and s, c are folded with the translate (Sec. "Input Phase") and the position scale n m, so that
// a key's position is one binary search over integer thresholds plus one multiply-add:
//   pos = clamp(floor(A_i d + C_i), 0, L - 1),  d = order image - lo (or value - lo for VALUE),
//   A_i = s_i scale n m,  C_i = c_i n m + 1/2,
// evaluated in pairs of binary32 (~48 significant bits, error-free products and sums); binary64 is
// used on the device only to normalise 64-bit floating-point keys.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace nns {
static inline cudaError_t nns_launched(cudaError_t e, int k = 1) {
    if (e == cudaSuccess) note_launch(k);
    return e;
}

// x-space segments of the binary64 model: segment i covers [brk[i], brk[i+1]) (brk[0] = -inf,
// the last segment is unbounded) with F = slope[i] x + icept[i]
void pwl_segments(int layers, int h1, int h2, const float *p, std::vector<double> &brk,
                  std::vector<double> &slope, std::vector<double> &icept) {
    brk.clear(); slope.clear(); icept.clear();
    const double inf = std::numeric_limits<double>::infinity();
    std::vector<double> W1(h1), b1(h1), W3, W2, b2;
    for (int j = 0; j < h1; ++j) { W1[j] = p[j]; b1[j] = p[h1 + j]; }
    double b3;
    if (layers == 1) {
        W3.assign(p + 2 * h1, p + 3 * h1);
        b3 = p[3 * h1];
    } else {
        W2.assign(p + 2 * h1, p + 2 * h1 + (size_t)h2 * h1);
        b2.assign(p + 2 * h1 + (size_t)h2 * h1, p + 2 * h1 + (size_t)h2 * h1 + h2);
        W3.assign(p + 2 * h1 + (size_t)h2 * h1 + h2, p + 2 * h1 + (size_t)h2 * h1 + 2 * h2);
        b3 = p[2 * h1 + (size_t)h2 * h1 + 2 * h2];
    }
    // first-layer bends
    std::vector<double> t1;
    for (int j = 0; j < h1; ++j)
        if (W1[j] != 0.0) t1.push_back(-b1[j] / W1[j]);
    std::sort(t1.begin(), t1.end());
    t1.erase(std::unique(t1.begin(), t1.end()), t1.end());
    // a point strictly inside [lo, hi)
    auto inside = [&](double lo, double hi) {
        if (lo == -inf && hi == inf) return 0.0;
        if (lo == -inf) return hi - std::max(1.0, std::fabs(hi));
        if (hi == inf) return lo + std::max(1.0, std::fabs(lo));
        return lo + 0.5 * (hi - lo);
    };
    auto push = [&](double lo, double s, double c) {
        if (!slope.empty() && slope.back() == s && icept.back() == c) return;  // same line: merge
        brk.push_back(lo); slope.push_back(s); icept.push_back(c);
    };
    std::vector<double> al(h2 > 0 ? h2 : 1), be(h2 > 0 ? h2 : 1), t2;
    std::vector<char> on(h1);
    for (size_t q = 0; q <= t1.size(); ++q) {
        const double lo = q == 0 ? -inf : t1[q - 1], hi = q == t1.size() ? inf : t1[q];
        const double xm = inside(lo, hi);
        for (int j = 0; j < h1; ++j) on[j] = (W1[j] * xm + b1[j]) > 0.0;
        if (layers == 1) {
            double s = 0.0, c = b3;
            for (int j = 0; j < h1; ++j)
                if (on[j]) { s += W3[j] * W1[j]; c += W3[j] * b1[j]; }
            push(lo, s, c);
            continue;
        }
        // second-layer pre-activations are linear here: z_k = al_k x + be_k
        t2.clear();
        for (int k = 0; k < h2; ++k) {
            double a = 0.0, b = b2[k];
            for (int j = 0; j < h1; ++j)
                if (on[j]) { a += W2[(size_t)k * h1 + j] * W1[j]; b += W2[(size_t)k * h1 + j] * b1[j]; }
            al[k] = a; be[k] = b;
            if (a != 0.0) {
                const double r = -b / a;
                if (r > lo && r < hi) t2.push_back(r);
            }
        }
        std::sort(t2.begin(), t2.end());
        t2.erase(std::unique(t2.begin(), t2.end()), t2.end());
        for (size_t u = 0; u <= t2.size(); ++u) {
            const double a0 = u == 0 ? lo : t2[u - 1], a1 = u == t2.size() ? hi : t2[u];
            const double xm2 = inside(a0, a1);
            double s = 0.0, c = b3;
            for (int k = 0; k < h2; ++k)
                if (al[k] * xm2 + be[k] > 0.0) { s += W3[k] * al[k]; c += W3[k] * be[k]; }
            push(a0, s, c);
        }
    }
    if (brk.empty()) push(-inf, 0.0, b3);
    brk[0] = -inf;
}

uint32_t pwl_max_segments(int layers, int h1, int h2) {
    return layers == 1 ? (uint32_t)h1 + 1u : 1u + (uint32_t)h1 + (uint32_t)(h1 + 1) * (uint32_t)h2;
}

static uint64_t host_ordbits_f32(float f) {
    uint32_t b;
    std::memcpy(&b, &f, 4);
    return (b & 0x80000000u) ? (uint64_t)(uint32_t)~b : (uint64_t)(b | 0x80000000u);
}
static uint64_t host_ordbits_f64(double v) {
    uint64_t b;
    std::memcpy(&b, &v, 8);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// the key-space table of one sort: thr[i] = smallest order image in segment i (thr[0] = 0)
void pwl_key_table(const nnsort_model_desc &d, const std::vector<double> &brk, const std::vector<double> &slope,
                   const std::vector<double> &icept, double nm, PwlEntry *out) {
    const size_t S = brk.size();
    const bool ob = d.translate == NNSORT_TRANSLATE_ORDBITS || d.dtype == NNSORT_U32 || d.dtype == NNSORT_U64;
    for (size_t i = 0; i < S; ++i) {
        uint64_t thr = 0;
        if (i > 0) {
            if (ob) {
                const long double v = (long double)d.lo_bits + ceill((long double)brk[i] / (long double)d.scale);
                thr = v <= 0.0L ? 0ull : (v >= 18446744073709551615.0L ? ~0ull : (uint64_t)v);
            } else {
                const double V = d.lo_val + brk[i] / d.scale;  // smallest key value in the segment
                if (d.dtype == NNSORT_F32) {
                    float f = (float)V;
                    if ((double)f < V) f = std::nextafter(f, std::numeric_limits<float>::infinity());
                    thr = host_ordbits_f32(f);
                } else {
                    thr = host_ordbits_f64(V);
                }
            }
        }
        out[i].thr = thr;
        const double A = slope[i] * d.scale * nm, Cv = icept[i] * nm + 0.5;
        out[i].Ah = (float)A;
        out[i].Al = (float)(A - (double)out[i].Ah);
        out[i].Ch = (float)Cv;
        out[i].Cl = (float)(Cv - (double)out[i].Ch);
    }
    for (size_t i = 1; i < S; ++i)  // rounding can only equalise neighbours, never reorder them
        if (out[i].thr < out[i - 1].thr) out[i].thr = out[i - 1].thr;
}

// ---------------------------------------------------------------------------------------------
// a + b exactly as hi + lo (Knuth's two-sum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// the key's translate offset d as a pair of binary32 (hi + lo): the order-image difference for
// ORDBITS and integer keys (integer arithmetic, exact to ~48 bits), the value difference for VALUE
// (binary32 pairs for f32 keys; binary64 only to normalise f64 keys)
__device__ __forceinline__ void pwl_offset(uint64_t w, uint64_t u, int dtype, bool ob, const Norm &nm,
                                           float lo_h, float lo_l, float &dh, float &dl) {
    if (ob) {
        const bool neg = u < nm.lo_bits;
        const uint64_t D = neg ? nm.lo_bits - u : u - nm.lo_bits;
        const float h = __ull2float_rn(D);
        const long long r = (long long)(D - (uint64_t)h);  // |r| <= half an ulp of h
        dh = neg ? -h : h;
        dl = neg ? -__ll2float_rn(r) : __ll2float_rn(r);
    } else if (dtype == NNSORT_F32) {
        float s1, e1;
        two_sum(__uint_as_float((uint32_t)w), -lo_h, s1, e1);
        e1 = __fsub_rn(e1, lo_l);
        two_sum(s1, e1, dh, dl);
    } else {
        const double v = __longlong_as_double((long long)w) - nm.lo_val;
        dh = __double2float_rn(v);
        dl = __double2float_rn(v - (double)dh);
    }
}

template <typename W>
__global__ void __launch_bounds__(PRED_THREADS) k_predict_pwl(PredictArgs a) {
    extern __shared__ __align__(16) unsigned char sraw[];
    const uint32_t S = a.pwl.S;
    float4 *cf = reinterpret_cast<float4 *>(sraw);  // Ah, Al, Ch, Cl (16-byte entries first)
    unsigned long long *thr = reinterpret_cast<unsigned long long *>(cf + S);
    const int tid = threadIdx.x;
    for (uint32_t i = tid; i < S; i += blockDim.x) {
        const PwlEntry e = a.pwl.tab[i];
        thr[i] = e.thr;
        cf[i] = make_float4(e.Ah, e.Al, e.Ch, e.Cl);
    }
    __syncthreads();
    uint32_t top = 1;  // largest power of two <= S
    while (top * 2 <= S) top *= 2;
    const Seg &sg = a.segs[0];
    const uint64_t n = sg.n;
    const Norm nm = sg.norm;
    const bool ob = nm.translate == NNSORT_TRANSLATE_ORDBITS || nm.dtype == NNSORT_U32 || nm.dtype == NNSORT_U64;
    const float lo_h = (float)nm.lo_val, lo_l = (float)(nm.lo_val - (double)lo_h);
    const long long Lm1 = (long long)(sg.L - 1);
    const W *keys = reinterpret_cast<const W *>(sg.keys);
    uint32_t err = 0;
    for (uint32_t tile = blockIdx.x; tile < a.total_tiles; tile += gridDim.x) {
        const uint64_t start = (uint64_t)tile * PRED_TILE;
        uint64_t wv[PRED_ITEMS];
#pragma unroll
        for (int k = 0; k < PRED_ITEMS; ++k) {
            const uint64_t i = start + (uint64_t)k * PRED_THREADS + tid;
            wv[k] = i < n ? word64(keys[i]) : 0ull;
        }
#pragma unroll
        for (int k = 0; k < PRED_ITEMS; ++k) {
            const uint64_t i = start + (uint64_t)k * PRED_THREADS + tid;
            if (i >= n) break;
            const uint64_t w = wv[k];
            if (key_is_nan(w, a.dtype)) err |= ERR_NAN;
            const uint64_t u = ordbits(w, a.dtype);
            uint32_t seg = 0;  // last segment whose threshold is <= u
            for (uint32_t step = top; step; step >>= 1)
                if (seg + step < S && thr[seg + step] <= u) seg += step;
            float dh, dl;
            pwl_offset(w, u, a.dtype, ob, nm, lo_h, lo_l, dh, dl);
            const float4 c = cf[seg];
            // y = A d + C in pairs of binary32: the product's rounding error by FMA, the cross
            // terms, then the sum with C by two-sum
            const float p = __fmul_rn(c.x, dh);
            float e = __fmaf_rn(c.x, dh, -p);
            e = __fmaf_rn(c.x, dl, e);
            e = __fmaf_rn(c.y, dh, e);
            float yh, ye;
            two_sum(p, c.z, yh, ye);
            const float yl = __fadd_rn(__fadd_rn(e, c.w), ye);
            // floor(yh + yl), clamped to [0, L - 1]; below -1 or beyond 2^33 the pair's low part
            // cannot move the result, and NaN (an infinite or NaN key) goes to position 0
            long long sl;
            if (!(yh >= -1.0f)) sl = 0;
            else if (yh >= 8589934592.0f) sl = Lm1;
            else {
                const float f = floorf(yh);
                sl = (long long)f + (long long)floorf(__fadd_rn(__fsub_rn(yh, f), yl));
            }
            if (sl < 0) sl = 0;
            if (sl > Lm1) sl = Lm1;
            const uint32_t slot = (uint32_t)sl;
            const uint32_t g = (uint32_t)(sg.gs_base + slot);
            if (a.gs) a.gs[i] = g;
            if (a.row_init) a.row_init[i] = (uint32_t)i;
            if (a.slots_out) a.slots_out[i] = slot;
            if (a.y_out) a.y_out[i] = __fdiv_rn(__fsub_rn(__fadd_rn(yh, yl), 0.5f), sg.nm_hi);
        }
    }
    if (err) atomicOr(a.err, err);
}

cudaError_t launch_predict_pwl(const PredictArgs &p, int sms, cudaStream_t s) {
    if (p.nseg != 1 || p.pwl.S == 0) return cudaErrorNotSupported;
    const size_t smem = (size_t)p.pwl.S * 24;  // float4 coefficients, then thresholds
    const int per_sm = std::max(1, std::min(8, (int)((size_t)(200 * 1024) / (smem + 2048 + 1024))));
    const int grid = (int)std::min<uint64_t>(p.total_tiles, (uint64_t)sms * per_sm);
    if (grid == 0) return cudaSuccess;
    auto k4 = k_predict_pwl<uint32_t>;
    auto k8 = k_predict_pwl<uint64_t>;
    cudaError_t e = cudaFuncSetAttribute(p.key_bytes == 4 ? k4 : k8,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (p.key_bytes == 4) k4<<<grid, PRED_THREADS, smem, s>>>(p);
    else k8<<<grid, PRED_THREADS, smem, s>>>(p);
    return nns_launched(cudaGetLastError());
}

}  // namespace nns
