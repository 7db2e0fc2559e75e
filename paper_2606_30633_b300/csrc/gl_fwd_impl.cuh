// Launch and shared-memory-limit helpers of k_forward, instantiated per
// lens-light count in gl_fwd_l*.cu and dispatched in gl_fwd.cu.
#pragma once

#include "gl_kernels.cuh"

namespace gl {

template <int NL, int NS, bool SURR>
cudaError_t fwd_launch(const SysParams& sp, const float* theta, int B, float* logp, float* img,
                     size_t dyn, cudaStream_t st) {
  k_forward<NL, NS, SURR><<<B, THREADS, dyn, st>>>(sp, theta, B, logp, img);
  return cudaGetLastError();
}

template <int NL, int NS>
cudaError_t fwd_smem(size_t bytes) {
  cudaError_t e =
      cudaFuncSetAttribute(k_forward<NL, NS, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_forward<NL, NS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

#define GL_FWD_INST(EXT, NL)                                                              \
  EXT template cudaError_t fwd_launch<NL, 1, false>(const SysParams&, const float*, int, float*,  \
                                                   float*, size_t, cudaStream_t);               \
  EXT template cudaError_t fwd_launch<NL, 2, false>(const SysParams&, const float*, int, float*,  \
                                                   float*, size_t, cudaStream_t);               \
  EXT template cudaError_t fwd_launch<NL, 3, false>(const SysParams&, const float*, int, float*,  \
                                                   float*, size_t, cudaStream_t);               \
  EXT template cudaError_t fwd_launch<NL, 1, true>(const SysParams&, const float*, int, float*,   \
                                                  float*, size_t, cudaStream_t);                \
  EXT template cudaError_t fwd_launch<NL, 2, true>(const SysParams&, const float*, int, float*,   \
                                                  float*, size_t, cudaStream_t);                \
  EXT template cudaError_t fwd_launch<NL, 3, true>(const SysParams&, const float*, int, float*,   \
                                                  float*, size_t, cudaStream_t);                \
  EXT template cudaError_t fwd_smem<NL, 1>(size_t);                                             \
  EXT template cudaError_t fwd_smem<NL, 2>(size_t);                                             \
  EXT template cudaError_t fwd_smem<NL, 3>(size_t);

}  // namespace gl
