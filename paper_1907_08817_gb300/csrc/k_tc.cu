// k_tc.cu -- BF16 tensor-core (tcgen05) forward pass for two-hidden-layer models.
#include "common.cuh"
#include "internal.h"

namespace nns {

cudaError_t launch_predict_bf16(const PadArch &, const PredictArgs &, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace nns
