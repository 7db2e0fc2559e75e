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

// The multi-system kernel of launch shape (threads, pairs): T threads per CTA,
// NPR pixel pairs per thread in phase 1.
template <int NL, int NS, bool SURR>
cudaError_t grad_multi_launch(int threads, int pairs, const SysParams* systems, const void* items,
                              int n_items, int* counter, int grid, size_t dyn, cudaStream_t st) {
  const MultiItem* it = static_cast<const MultiItem*>(items);
#define GL_SHAPE(T, N)                                                                  \
  if (threads == T && pairs == N) {                                                     \
    k_grad_multi<NL, NS, SURR, T, N><<<grid, T, dyn, st>>>(systems, it, n_items, counter); \
    return cudaGetLastError();                                                          \
  }
  GL_SHAPE(128, 2) GL_SHAPE(128, 3) GL_SHAPE(256, 2) GL_SHAPE(256, 3)
#undef GL_SHAPE
  return cudaErrorInvalidValue;
}

// Dynamic shared-memory limits: k_grad's, and each multi-system shape's (the
// per-block maximum less that kernel's static memory).
template <int NL, int NS, bool S>
cudaError_t grad_smem(size_t bytes, size_t block_max) {
  cudaError_t e =
      cudaFuncSetAttribute(k_grad<NL, NS, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
#define GL_SHAPE(T, N)                                                                     \
  if (e == cudaSuccess) {                                                                  \
    const size_t st = static_smem_bytes(true, T);                                          \
    e = cudaFuncSetAttribute(k_grad_multi<NL, NS, S, T, N>,                                \
                             cudaFuncAttributeMaxDynamicSharedMemorySize,                  \
                             (int)(block_max > st ? block_max - st : 0));                  \
  }
  GL_SHAPE(128, 2) GL_SHAPE(128, 3) GL_SHAPE(256, 2) GL_SHAPE(256, 3)
#undef GL_SHAPE
  return e;
}

#define GL_GRAD_INST_S(EXT, NL, S)                                                         \
  EXT template cudaError_t grad_launch<NL, 1, S>(const SysParams&, const float*, int, float*,  \
                                                 float*, size_t, cudaStream_t);                \
  EXT template cudaError_t grad_launch<NL, 2, S>(const SysParams&, const float*, int, float*,  \
                                                 float*, size_t, cudaStream_t);                \
  EXT template cudaError_t grad_launch<NL, 3, S>(const SysParams&, const float*, int, float*,  \
                                                 float*, size_t, cudaStream_t);                \
  EXT template cudaError_t grad_multi_launch<NL, 1, S>(int, int, const SysParams*, const void*, \
                                                       int, int*, int, size_t, cudaStream_t);  \
  EXT template cudaError_t grad_multi_launch<NL, 2, S>(int, int, const SysParams*, const void*, \
                                                       int, int*, int, size_t, cudaStream_t);  \
  EXT template cudaError_t grad_multi_launch<NL, 3, S>(int, int, const SysParams*, const void*, \
                                                       int, int*, int, size_t, cudaStream_t);  \
  EXT template cudaError_t grad_smem<NL, 1, S>(size_t, size_t);                                        \
  EXT template cudaError_t grad_smem<NL, 2, S>(size_t, size_t);                                        \
  EXT template cudaError_t grad_smem<NL, 3, S>(size_t, size_t);

#define GL_GRAD_INST(EXT, NL)      \
  GL_GRAD_INST_S(EXT, NL, false)   \
  GL_GRAD_INST_S(EXT, NL, true)

}  // namespace gl
