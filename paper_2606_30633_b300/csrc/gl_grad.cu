// Dispatch of k_grad on the system's component counts and deflection kind
// (instantiations live in gl_grad_l*.cu).
#include "gl_fused.cuh"
#include "gl_grad_impl.cuh"

namespace gl {

GL_GRAD_INST(extern, 0)
GL_GRAD_INST(extern, 1)
GL_GRAD_INST(extern, 2)
GL_FUSED_INST(extern, 0)
GL_FUSED_INST(extern, 1)
GL_FUSED_INST(extern, 2)

cudaError_t launch_grad_fused(const SysParams& sp, const float* theta, int B, float* logp,
                              float* grad, size_t dyn, bool* fits, cudaStream_t st) {
#define GL_CASE(a, b) \
  if (sp.nL == a && sp.nS == b) return grad_fused_launch<a, b>(sp, theta, B, logp, grad, dyn, fits, st);
  GL_CASE(0, 1) GL_CASE(0, 2) GL_CASE(0, 3)
  GL_CASE(1, 1) GL_CASE(1, 2) GL_CASE(1, 3)
  GL_CASE(2, 1) GL_CASE(2, 2) GL_CASE(2, 3)
#undef GL_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_grad(const SysParams& sp, const float* theta, int B, float* logp, float* grad,
                        size_t dyn, cudaStream_t st) {
#define GL_CASE(a, b)                                                         \
  if (sp.nL == a && sp.nS == b)                                               \
    return sp.table ? grad_launch<a, b, true>(sp, theta, B, logp, grad, dyn, st) \
                    : grad_launch<a, b, false>(sp, theta, B, logp, grad, dyn, st);
  GL_CASE(0, 1) GL_CASE(0, 2) GL_CASE(0, 3)
  GL_CASE(1, 1) GL_CASE(1, 2) GL_CASE(1, 3)
  GL_CASE(2, 1) GL_CASE(2, 2) GL_CASE(2, 3)
#undef GL_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_grad_multi(int nL, int nS, bool surr, int threads, int pairs,
                              const SysParams* systems, const void* items, int n_items,
                              int* counter, int grid, size_t dyn, cudaStream_t st) {
#define GL_CASE(a, b)                                                                        \
  if (nL == a && nS == b)                                                                    \
    return surr ? grad_multi_launch<a, b, true>(threads, pairs, systems, items, n_items,     \
                                                counter, grid, dyn, st)                      \
                : grad_multi_launch<a, b, false>(threads, pairs, systems, items, n_items,    \
                                                 counter, grid, dyn, st);
  GL_CASE(0, 1) GL_CASE(0, 2) GL_CASE(0, 3)
  GL_CASE(1, 1) GL_CASE(1, 2) GL_CASE(1, 3)
  GL_CASE(2, 1) GL_CASE(2, 2) GL_CASE(2, 3)
#undef GL_CASE
  return cudaErrorInvalidValue;
}

cudaError_t set_smem_limits_grad(size_t block_max) {
  // dynamic limit = the per-block maximum less each kernel's static memory
  const size_t st = static_smem_bytes(false);
  const size_t bytes = block_max > st ? block_max - st : 0;
  cudaError_t e = cudaSuccess;
#define GL_SET(a, b) \
  if (e == cudaSuccess) e = grad_smem<a, b, false>(bytes, block_max); \
  if (e == cudaSuccess) e = grad_smem<a, b, true>(bytes, block_max);  \
  if (e == cudaSuccess) e = grad_fused_smem<a, b>(block_max);
  GL_SET(0, 1) GL_SET(0, 2) GL_SET(0, 3)
  GL_SET(1, 1) GL_SET(1, 2) GL_SET(1, 3)
  GL_SET(2, 1) GL_SET(2, 2) GL_SET(2, 3)
#undef GL_SET
  return e;
}

}  // namespace gl
