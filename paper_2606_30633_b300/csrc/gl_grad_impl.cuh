// Launch and shared-memory-limit helpers of k_grad, instantiated per
// lens-light count in gl_grad_l*.cu and dispatched in gl_grad.cu.
#pragma once

#include "gl_kernels.cuh"

namespace gl {

template <int NL, int NS, bool SURR>
cudaError_t grad_launch(const SysParams& sp, const float* theta, int B, float* logp, float* grad,
                     size_t dyn, cudaStream_t st) {
  k_grad<NL, NS, SURR><<<B, THREADS, dyn, st>>>(sp, theta, B, logp, grad);
  return cudaGetLastError();
}

template <int NL, int NS>
cudaError_t grad_smem(size_t bytes) {
  cudaError_t e =
      cudaFuncSetAttribute(k_grad<NL, NS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grad<NL, NS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

#define GL_GRAD_INST(EXT, NL)                                                              \
  EXT template cudaError_t grad_launch<NL, 1, false>(const SysParams&, const float*, int, float*,  \
                                                   float*, size_t, cudaStream_t);               \
  EXT template cudaError_t grad_launch<NL, 2, false>(const SysParams&, const float*, int, float*,  \
                                                   float*, size_t, cudaStream_t);               \
  EXT template cudaError_t grad_launch<NL, 3, false>(const SysParams&, const float*, int, float*,  \
                                                   float*, size_t, cudaStream_t);               \
  EXT template cudaError_t grad_launch<NL, 1, true>(const SysParams&, const float*, int, float*,   \
                                                  float*, size_t, cudaStream_t);                \
  EXT template cudaError_t grad_launch<NL, 2, true>(const SysParams&, const float*, int, float*,   \
                                                  float*, size_t, cudaStream_t);                \
  EXT template cudaError_t grad_launch<NL, 3, true>(const SysParams&, const float*, int, float*,   \
                                                  float*, size_t, cudaStream_t);                \
  EXT template cudaError_t grad_smem<NL, 1>(size_t);                                             \
  EXT template cudaError_t grad_smem<NL, 2>(size_t);                                             \
  EXT template cudaError_t grad_smem<NL, 3>(size_t);

}  // namespace gl
