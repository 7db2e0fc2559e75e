// Instantiates the forward kernels (log p, model image) for every supported
// component count and dispatches on the system's counts.
#include "gl_kernels.cuh"

namespace gl {

template <int NL, int NS>
static cudaError_t launch_fwd_t(const SysParams& sp, const float* theta, int B, float* logp,
                                float* img, size_t dyn, cudaStream_t st) {
  k_forward<NL, NS><<<B, THREADS, dyn, st>>>(sp, theta, B, logp, img);
  return cudaGetLastError();
}

cudaError_t launch_forward(const SysParams& sp, const float* theta, int B, float* logp,
                           float* img, size_t dyn, cudaStream_t st) {
#define GL_CASE(a, b) \
  if (sp.nL == a && sp.nS == b) return launch_fwd_t<a, b>(sp, theta, B, logp, img, dyn, st);
  GL_CASE(0, 1) GL_CASE(0, 2) GL_CASE(0, 3)
  GL_CASE(1, 1) GL_CASE(1, 2) GL_CASE(1, 3)
  GL_CASE(2, 1) GL_CASE(2, 2) GL_CASE(2, 3)
#undef GL_CASE
  return cudaErrorInvalidValue;
}

cudaError_t set_smem_limits_fwd(size_t bytes) {
  cudaError_t e = cudaSuccess;
#define GL_SET(a, b)                                                                          \
  if (e == cudaSuccess)                                                                        \
    e = cudaFuncSetAttribute(k_forward<a, b>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)bytes);
  GL_SET(0, 1) GL_SET(0, 2) GL_SET(0, 3)
  GL_SET(1, 1) GL_SET(1, 2) GL_SET(1, 3)
  GL_SET(2, 1) GL_SET(2, 2) GL_SET(2, 3)
#undef GL_SET
  return e;
}

}  // namespace gl
