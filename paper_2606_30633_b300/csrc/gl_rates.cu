// gl_unit_rates: per-SM, per-clock throughput of the pipes the lens kernels
// are bound by, measured on the running GPU. The roofline of the fused
// forward + adjoint is max(F / (n_SM r_FP32 f), M / (n_SM r_MUFU f)) with F
// FP32 operations and M MUFU operations per evaluation; this entry point
// measures r_FP32 (scalar FFMA and paired FFMA2, an FMA counted as one
// operation per lane) and r_MUFU (ex2 / lg2 approximations).
//
// One CTA of 1024 threads per SM (its dynamic shared memory keeps a second
// CTA off the SM), eight independent dependency chains per thread, timed in
// SM clocks with clock64 between two block barriers; the rate is the CTA's
// operations over its own cycle count, averaged over the SMs. Values stay
// bounded (contractions for the FMAs, lg2 followed by ex2 for the MUFU), so
// the results are written out only to keep the loops live.
#include <cuda_runtime.h>

#include <string>

#include "../../include/gl.h"
#include "gl_model.cuh"

namespace gl {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int RT = 1024;                   // threads per CTA
constexpr int RATE_SMEM = 160 * 1024;      // > half an SM's shared memory: one CTA per SM
constexpr int CHAINS = 8;

__device__ __forceinline__ float mufu_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// KIND 0: FFMA; 1: FFMA2 (two lanes per instruction); 2: MUFU lg2 + ex2.
template <int KIND>
__global__ void __launch_bounds__(RT, 1) k_rate(int iters, float* __restrict__ sink,
                                                long long* __restrict__ cycles) {
  extern __shared__ float pad[];
  const float s = 1.f + 1e-3f * (threadIdx.x & 31);
  if (threadIdx.x == 0) pad[0] = s;  // touch the reservation
  float x[CHAINS];
  float2 p[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) {
    x[c] = 0.5f + 0.01f * c * s;
    p[c] = make_float2(x[c], x[c] + 0.003f);
  }
  const float a = 0.9999f, b = 1e-4f;
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      if (KIND == 0) x[c] = fmaf(x[c], a, b);
      if (KIND == 1) p[c] = gl::fma2(p[c], a2, b2);
      if (KIND == 2) x[c] = mufu_ex2(mufu_lg2(x[c]));
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) acc += KIND == 1 ? p[c].x + p[c].y : x[c];
  sink[(size_t)blockIdx.x * RT + threadIdx.x] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

template <int KIND>
cudaError_t rate(int n_sm, int iters, float* sink, long long* cyc, long long* host, double ops,
                 double* out) {
  cudaError_t e = cudaFuncSetAttribute(k_rate<KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       RATE_SMEM);
  if (e != cudaSuccess) return e;
  k_rate<KIND><<<n_sm, RT, RATE_SMEM>>>(iters, sink, cyc);  // warm-up
  k_rate<KIND><<<n_sm, RT, RATE_SMEM>>>(iters, sink, cyc);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaMemcpy(host, cyc, n_sm * sizeof(long long), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return e;
  double sum = 0.0;
  for (int k = 0; k < n_sm; ++k) sum += ops / (double)(host[k] > 0 ? host[k] : 1);
  *out = sum / n_sm;
  return cudaSuccess;
}

}  // namespace

extern "C" gl_status gl_unit_rates(double* fp32, double* fp32x2, double* mufu) {
  if (!fp32 || !fp32x2 || !mufu) {
    gl::set_last_error("NULL output");
    return GL_EINVAL;
  }
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  float* sink = nullptr;
  long long* cyc = nullptr;
  long long* host = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&sink, (size_t)n_sm * RT * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&cyc, (size_t)n_sm * sizeof(long long));
  if (e == cudaSuccess) host = new long long[n_sm];
  // iteration counts give about 2e6 cycles per kind at the nominal rates
  const int it_fma = 32768, it_mufu = 2048;
  const double per_thread = (double)RT * CHAINS;
  if (e == cudaSuccess) e = rate<0>(n_sm, it_fma, sink, cyc, host, per_thread * it_fma, fp32);
  if (e == cudaSuccess)
    e = rate<1>(n_sm, it_fma / 2, sink, cyc, host, 2.0 * per_thread * (it_fma / 2), fp32x2);
  if (e == cudaSuccess)
    e = rate<2>(n_sm, it_mufu, sink, cyc, host, 2.0 * per_thread * it_mufu, mufu);
  delete[] host;
  cudaFree(sink);
  cudaFree(cyc);
  if (e != cudaSuccess) {
    gl::set_last_error(std::string("unit rates: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? GL_ENOMEM : GL_ECUDA;
  }
  return GL_OK;
}
