// Dispatch of k_forward on the system's component counts and deflection kind
// (instantiations live in gl_fwd_l*.cu).
#include "gl_fwd_impl.cuh"

namespace gl {

GL_FWD_INST(extern, 0)
GL_FWD_INST(extern, 1)
GL_FWD_INST(extern, 2)

cudaError_t launch_forward(const SysParams& sp, const float* theta, int B, float* logp, float* img,
                        size_t dyn, cudaStream_t st) {
#define GL_CASE(a, b)                                                         \
  if (sp.nL == a && sp.nS == b)                                               \
    return sp.table ? fwd_launch<a, b, true>(sp, theta, B, logp, img, dyn, st) \
                    : fwd_launch<a, b, false>(sp, theta, B, logp, img, dyn, st);
  GL_CASE(0, 1) GL_CASE(0, 2) GL_CASE(0, 3)
  GL_CASE(1, 1) GL_CASE(1, 2) GL_CASE(1, 3)
  GL_CASE(2, 1) GL_CASE(2, 2) GL_CASE(2, 3)
#undef GL_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_component_images(const SysParams& sp, const float* theta, int B, float* img,
                                    size_t dyn, cudaStream_t st) {
  if (sp.table)
    k_component_images<true><<<B, THREADS, dyn, st>>>(sp, theta, B, img);
  else
    k_component_images<false><<<B, THREADS, dyn, st>>>(sp, theta, B, img);
  return cudaGetLastError();
}

size_t static_smem_bytes(bool multi, int threads) {
  // SmemStatic + the table (+ k_grad_multi's work index and parameter
  // block), with alignment slack
  const size_t smem_static = threads == 128 ? sizeof(SmemStatic<4>) : sizeof(SmemStatic<NWARPS>);
  return smem_static + TABLE_ROW * sizeof(float4) + 256 + (multi ? sizeof(SysParams) + 16 : 0);
}

cudaError_t set_smem_limits_fwd(size_t block_max) {
  const size_t st = static_smem_bytes(false);
  const size_t bytes = block_max > st ? block_max - st : 0;
  cudaError_t e = cudaSuccess;
#define GL_SET(a, b) \
  if (e == cudaSuccess) e = fwd_smem<a, b>(bytes);
  GL_SET(0, 1) GL_SET(0, 2) GL_SET(0, 3)
  GL_SET(1, 1) GL_SET(1, 2) GL_SET(1, 3)
  GL_SET(2, 1) GL_SET(2, 2) GL_SET(2, 3)
#undef GL_SET
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_component_images<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_component_images<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
  return e;
}

}  // namespace gl
