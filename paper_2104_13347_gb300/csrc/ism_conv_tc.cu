// ism_conv_tc.cu -- K2: split-BF16 tensor-core convolution (in progress).
#include "ism_internal.h"

namespace ism {
int launch_conv_bf16x3(const ConvLaunch &, cudaStream_t) {
    return fail(ISM_ERR_INVALID_ARG, "ISM_BF16X3 is not built into this library yet");
}
}  // namespace ism
