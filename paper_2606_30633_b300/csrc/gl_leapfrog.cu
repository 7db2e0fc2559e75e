// HMC leapfrog blocks (the integrator inside every HMC trajectory of the
// pipeline's sampling stage, Sec. 3): n_steps leapfrog steps for B chains,
// captured once into a CUDA graph and replayed.
//
// One step with diagonal inverse mass M^-1 and step size eps:
//   p     <- p + eps/2 grad log p(theta)          (k_kick_drift, first half)
//   theta <- theta + eps M^-1 p                   (k_kick_drift, second half)
//   (log p, grad) at the new theta                (the fused gradient kernel)
//   p     <- p + eps/2 grad log p(theta)          (k_kick)
// A chain whose log p is not finite (outside the support, or NaN) is frozen:
// neither kernel touches its theta or p again, and its log p stays -inf/NaN
// so that the caller can see and reject the divergent trajectory.
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "../../include/gl.h"
#include "gl_internal.cuh"

namespace gl {

__global__ void k_kick_drift(float* __restrict__ theta, float* __restrict__ p,
                             const float* __restrict__ grad, const float* __restrict__ logp,
                             const float* __restrict__ inv_mass, float half_eps, float eps, int B,
                             int P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * P) return;
  const int b = i / P, k = i - b * P;
  if (!isfinite(logp[b])) return;
  const float pk = fmaf(half_eps, grad[i], p[i]);
  p[i] = pk;
  theta[i] = fmaf(eps * inv_mass[k], pk, theta[i]);
}

__global__ void k_kick(float* __restrict__ p, const float* __restrict__ grad,
                       const float* __restrict__ logp, float half_eps, int B, int P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * P) return;
  const int b = i / P;
  if (!isfinite(logp[b])) return;
  p[i] = fmaf(half_eps, grad[i], p[i]);
}

cudaError_t launch_leapfrog_block(const SysParams& sp, size_t dyn, float* theta, float* p,
                                  float* logp, float* grad, const float* inv_mass, float eps,
                                  int n_steps, int B, cudaStream_t st) {
  const int n = B * sp.P;
  const int threads = 256;
  const int blocks = (n + threads - 1) / threads;
  for (int s = 0; s < n_steps; ++s) {
    k_kick_drift<<<blocks, threads, 0, st>>>(theta, p, grad, logp, inv_mass, 0.5f * eps, eps, B,
                                             sp.P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_grad(sp, theta, B, logp, grad, dyn, st);
    if (e != cudaSuccess) return e;
    k_kick<<<blocks, threads, 0, st>>>(p, grad, logp, 0.5f * eps, B, sp.P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace gl
