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

template <int NL, int NS, bool SURR>
cudaError_t grad_multi_launch(const SysParams* systems, const void* items, int n_items,
                              int* counter, int grid, size_t dyn, cudaStream_t st) {
  k_grad_multi<NL, NS, SURR><<<grid, THREADS, dyn, st>>>(
      systems, static_cast<const MultiItem*>(items), n_items, counter);
  return cudaGetLastError();
}

template <int NL, int NS, bool S>
cudaError_t grad_smem(size_t bytes, size_t bytes_multi) {
  cudaError_t e =
      cudaFuncSetAttribute(k_grad<NL, NS, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grad_multi<NL, NS, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes_multi);
  return e;
}

#define GL_GRAD_INST_S(EXT, NL, S)                                                         \
  EXT template cudaError_t grad_launch<NL, 1, S>(const SysParams&, const float*, int, float*,  \
                                                 float*, size_t, cudaStream_t);                \
  EXT template cudaError_t grad_launch<NL, 2, S>(const SysParams&, const float*, int, float*,  \
                                                 float*, size_t, cudaStream_t);                \
  EXT template cudaError_t grad_launch<NL, 3, S>(const SysParams&, const float*, int, float*,  \
                                                 float*, size_t, cudaStream_t);                \
  EXT template cudaError_t grad_multi_launch<NL, 1, S>(const SysParams*, const void*, int,     \
                                                       int*, int, size_t, cudaStream_t);       \
  EXT template cudaError_t grad_multi_launch<NL, 2, S>(const SysParams*, const void*, int,     \
                                                       int*, int, size_t, cudaStream_t);       \
  EXT template cudaError_t grad_multi_launch<NL, 3, S>(const SysParams*, const void*, int,     \
                                                       int*, int, size_t, cudaStream_t);       \
  EXT template cudaError_t grad_smem<NL, 1, S>(size_t, size_t);                                        \
  EXT template cudaError_t grad_smem<NL, 2, S>(size_t, size_t);                                        \
  EXT template cudaError_t grad_smem<NL, 3, S>(size_t, size_t);

#define GL_GRAD_INST(EXT, NL)      \
  GL_GRAD_INST_S(EXT, NL, false)   \
  GL_GRAD_INST_S(EXT, NL, true)

}  // namespace gl
