// Internal interface between the solver and the learned predictor
// (otm_unet.cu).
#pragma once
#include <cuda_runtime.h>

#include "otm.h"

namespace otm {
// y (3 n^3 FP32, device) = net(x) with x the n^3 filtered density (FP32 or
// FP64 per x_double), ordered on st.
otm_status unet_predict(otm_unet* u, const void* x, bool x_double, float* y, cudaStream_t st);
// grid size the network was built for (0 for NULL)
int unet_grid(const otm_unet* u);
// kernels launched by all networks so far (for launch accounting)
long long unet_launches();
}  // namespace otm
