// k_predict.cu -- the translate, map and rounding steps of Fig. "Algorithm NN-sort":
// w <- translate(A), w_pos <- w.map(f), pos <- round(w_pos * m), for every key, in binary32.
//
// One pass over the keys (128-bit friendly striped loads), the model's parameters staged once per
// block in shared memory, the position written as a global position gs = gs_base + pos.
#include "common.cuh"
#include "internal.h"

namespace nns {
static inline cudaError_t nns_launched(cudaError_t e, int k = 1) {
    if (e == cudaSuccess) note_launch(k);
    return e;
}
}  // namespace nns

namespace nns {

__device__ __forceinline__ int seg_of_tile(const Seg *segs, int nseg, uint32_t tile) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].tbase <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int H1, int H2, typename W>
__global__ void __launch_bounds__(PRED_THREADS) k_predict(PredictArgs a) {
    extern __shared__ __align__(16) float sp[];  // padded parameters
    __shared__ int sh_seg;
    const int tid = threadIdx.x;
    int loaded = -1;
    uint32_t err = 0;
    constexpr int P = (H2 == 0) ? (3 * H1 + 1) : (2 * H1 + H2 * H1 + 2 * H2 + 1);
    for (uint32_t tile = blockIdx.x; tile < a.total_tiles; tile += gridDim.x) {
        __syncthreads();
        if (tid == 0) sh_seg = seg_of_tile(a.segs, a.nseg, tile);
        __syncthreads();
        const int si = sh_seg;
        const Seg &sg = a.segs[si];
        const uint64_t n = sg.n;
        const bool model = sg.slots == nullptr;
        if (model && si != loaded) {
            for (int i = tid; i < P; i += blockDim.x) sp[i] = sg.params[i];
            loaded = si;
        }
        __syncthreads();
        const Norm nm = sg.norm;
        const uint64_t start = (uint64_t)(tile - sg.tbase) * PRED_TILE;
        const W *keys = reinterpret_cast<const W *>(sg.keys);
#pragma unroll 2
        for (int k = 0; k < PRED_ITEMS; ++k) {
            const uint64_t i = start + (uint64_t)k * PRED_THREADS + tid;
            if (i >= n) break;
            const uint64_t w = word64(keys[i]);
            uint32_t slot;
            float y = 0.0f;
            if (key_is_nan(w, a.dtype)) err |= ERR_NAN;
            if (model) {
                y = mlp_fwd_f32<H1, H2>(sp, translate_x(w, nm));
                slot = slot_of(y, sg.nm_hi, sg.nm_lo, sg.L);
            } else {
                slot = sg.slots[i];
                if ((uint64_t)slot >= sg.L) { err |= ERR_SLOT; slot = 0; }
            }
            const uint64_t e = sg.ebase + i;
            const uint32_t g = (uint32_t)(sg.gs_base + slot);
            if (a.gs) a.gs[e] = g;
            if (a.key_copy) reinterpret_cast<W *>(a.key_copy)[e] = (W)w;
            if (a.pay_copy && sg.payload) a.pay_copy[e] = (uint32_t)sg.payload[i];
            if (a.row_init) a.row_init[e] = (uint32_t)i;
            if (a.slots_out) a.slots_out[e] = slot;
            if (a.y_out) a.y_out[e] = y;
        }
    }
    if (err) atomicOr(a.err, err);
}

template <int H1, int H2>
static cudaError_t go(const PredictArgs &p, int sms, cudaStream_t s) {
    constexpr int P = (H2 == 0) ? (3 * H1 + 1) : (2 * H1 + H2 * H1 + 2 * H2 + 1);
    const size_t smem = ((P + 3) / 4) * 16;
    const int grid = (int)std::min<uint64_t>(p.total_tiles, (uint64_t)sms * 8);
    if (grid == 0) return cudaSuccess;
    if (p.key_bytes == 4)
        k_predict<H1, H2, uint32_t><<<grid, PRED_THREADS, smem, s>>>(p);
    else
        k_predict<H1, H2, uint64_t><<<grid, PRED_THREADS, smem, s>>>(p);
    return nns_launched(cudaGetLastError());
}

cudaError_t launch_predict_bf16(const PadArch &a, const PredictArgs &p, bool split, int sms, cudaStream_t s);

cudaError_t launch_predict(const PadArch &a, int precision, const PredictArgs &p, int sms,
                           cudaStream_t s) {
    if (precision == NNSORT_PREC_PWL) return launch_predict_pwl(p, sms, s);
    if ((precision == NNSORT_PREC_BF16 || precision == NNSORT_PREC_BF16X2) && a.layers == 2)
        return launch_predict_bf16(a, p, precision == NNSORT_PREC_BF16X2, sms, s);
    if (a.layers == 1) {
        switch (a.h1) {
        case 8: return go<8, 0>(p, sms, s);
        case 16: return go<16, 0>(p, sms, s);
        case 32: return go<32, 0>(p, sms, s);
        case 64: return go<64, 0>(p, sms, s);
        }
    } else {
        switch (a.h1) {
        case 8: return go<8, 8>(p, sms, s);
        case 16: return go<16, 16>(p, sms, s);
        case 32: return go<32, 32>(p, sms, s);
        case 64: return go<64, 64>(p, sms, s);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace nns
