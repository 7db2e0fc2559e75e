// Instantiates the fused forward + adjoint kernels for every supported
// component count and dispatches on the system's counts.
#include "gl_kernels.cuh"

namespace gl {

template <int NL, int NS>
static cudaError_t launch_grad_t(const SysParams& sp, const float* theta, int B, float* logp,
                                 float* grad, size_t dyn, cudaStream_t st) {
  k_grad<NL, NS><<<B, THREADS, dyn, st>>>(sp, theta, B, logp, grad);
  return cudaGetLastError();
}

cudaError_t launch_grad(const SysParams& sp, const float* theta, int B, float* logp, float* grad,
                        size_t dyn, cudaStream_t st) {
#define GL_CASE(a, b) \
  if (sp.nL == a && sp.nS == b) return launch_grad_t<a, b>(sp, theta, B, logp, grad, dyn, st);
  GL_CASE(0, 1) GL_CASE(0, 2) GL_CASE(0, 3)
  GL_CASE(1, 1) GL_CASE(1, 2) GL_CASE(1, 3)
  GL_CASE(2, 1) GL_CASE(2, 2) GL_CASE(2, 3)
#undef GL_CASE
  return cudaErrorInvalidValue;
}

cudaError_t set_smem_limits_grad(size_t bytes) {
  cudaError_t e = cudaSuccess;
#define GL_SET(a, b)                                                                       \
  if (e == cudaSuccess)                                                                     \
    e = cudaFuncSetAttribute(k_grad<a, b>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)bytes);
  GL_SET(0, 1) GL_SET(0, 2) GL_SET(0, 3)
  GL_SET(1, 1) GL_SET(1, 2) GL_SET(1, 3)
  GL_SET(2, 1) GL_SET(2, 2) GL_SET(2, 3)
#undef GL_SET
  return e;
}

}  // namespace gl
