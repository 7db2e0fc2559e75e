// The fused learned-deflection kernel: forward + adjoint of one row per CTA,
// with the row's angular table built by the surrogate network inside the same
// CTA (tcgen05 MMAs, TMEM accumulators) instead of by a separate launch that
// writes the tables to global memory. The network's operands use the CTA's
// dynamic shared memory before the image buffers do (the two are never live
// together); the table stays in static shared memory for the lens phases.
// Tables are bit-identical to the stand-alone build's (the same net_row).
#pragma once

#include "gl_kernels.cuh"
#include "gl_tc.cuh"

namespace gl {

template <int NL, int NS>
__global__ void __launch_bounds__(THREADS, 2)
k_grad_fused(const __grid_constant__ SysParams sp, const float* __restrict__ theta, int B,
             float* __restrict__ logp, float* __restrict__ grad) {
  constexpr int P = 8 + 7 * (NL + NS);
  // the tensor-core operands want an aligned base (its own name: the other
  // kernels' dynamic array is declared with 16-byte alignment)
  extern __shared__ __align__(1024) unsigned char fsm[];
  float* dsm = reinterpret_cast<float*>(fsm);
  __shared__ SmemStatic<NWARPS> st;
  __shared__ float4 tab[TABLE_ROW];
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t bar;
  const int b = blockIdx.x;
  if (b >= B) return;
  const int t = threadIdx.x, w = t >> 5;
  const float* th = theta + (size_t)b * P;
  SampleC& sc = st.sc;
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // 256 columns: at most two CTAs per SM (registers), 512 columns in all
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&tmem_base)),
                 "r"(tc::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (t < 32) stage_warp(sp, th, sc, st.fin, true);
  for (int k = t; k < NWARPS * MAX_P; k += THREADS) (&st.adj.redP[0][0])[k] = 0.f;
  tc::to_async();
  const uint32_t tb = tmem_base;
  if (sc.status == 0 && sc.use_table) {
    unsigned char* net = fsm;
    tc::load_weights<THREADS>(net, sp.net_wimg,
                              static_cast<const __nv_bfloat16*>(sp.net_wb));
    // (q, gamma) as the stand-alone table build computes them
    const float e1 = th[2], e2 = th[3];
    const float cc = sqrtf(e1 * e1 + e2 * e2);
    const float q = (1.f - cc) / (1.f + cc), gamma = th[1];
    float4(*node)[2] = reinterpret_cast<float4(*)[2]>(net + tc::TB_A);
    uint32_t phase = 0;
    float vp, dv;
    table_node(t & 127, vp, dv);
    const bool ok = net_row<THREADS>(static_cast<const __nv_bfloat16*>(sp.net_wb), sp.net_params,
                                     q, gamma, vp, dv, net, node, tb, &bar, phase,
                                     sp.net_forced != 0);
    if (ok) {
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      write_intervals(node, tab);
    } else {
      // a wait ran out with one commit outstanding: wait for it once more
      // (also bounded) before the tensor memory is freed and the shared memory
      // reused; flag the failure; a NaN table makes the row's results NaN
      tc::wait_phase(&bar, phase);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (t == 0) atomicExch(sp.net_timeout, 1);
      const float nan = __int_as_float(0x7fc00000);
      for (int k = t; k < TABLE_ROW; k += THREADS) tab[k] = make_float4(nan, nan, nan, nan);
    }
    __syncthreads();
  }
  grad_row<NL, NS, true, false, THREADS, 3, true>(sp, th, logp + b, grad + (size_t)b * P, nullptr,
                                                  b, dsm, st, tab);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb),
                 "r"(tc::TMEM_COLS));
}

// Two CTAs of the fused kernel fit per SM when two CTAs' registers and shared
// memory (static, rounded up to the dynamic array's 1024-byte alignment, plus
// dynamic, plus the per-block reserve) fit the SM's. (The occupancy query of
// the runtime reports one CTA for this kernel although the SM runs two: ncu
// shows both limits at two CTAs and 14.4 warps active.)
template <int NL, int NS>
cudaError_t grad_fused_launch(const SysParams& sp, const float* theta, int B, float* logp,
                              float* grad, size_t dyn, bool* fits, cudaStream_t st) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_grad_fused<NL, NS>);
  int dev = 0, smem_sm = 0, resv = 0, regs_sm = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  if (e != cudaSuccess) return e;
  const size_t per_cta = ((fa.sharedSizeBytes + 1023) & ~(size_t)1023) + dyn + (size_t)resv;
  *fits = 2 * per_cta <= (size_t)smem_sm && 2 * fa.numRegs * THREADS <= regs_sm;
  if (!*fits) return cudaSuccess;
  k_grad_fused<NL, NS><<<B, THREADS, dyn, st>>>(sp, theta, B, logp, grad);
  return cudaGetLastError();
}

template <int NL, int NS>
cudaError_t grad_fused_smem(size_t block_max) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, k_grad_fused<NL, NS>);
  if (e != cudaSuccess) return e;
  // the dynamic array starts 1024-byte aligned after the static memory
  const size_t st = (a.sharedSizeBytes + 1023) & ~(size_t)1023;
  return cudaFuncSetAttribute(k_grad_fused<NL, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(block_max > st ? block_max - st : 0));
}

#define GL_FUSED_INST(EXT, NL)                                                                    \
  EXT template cudaError_t grad_fused_launch<NL, 1>(const SysParams&, const float*, int, float*, \
                                                    float*, size_t, bool*, cudaStream_t);        \
  EXT template cudaError_t grad_fused_launch<NL, 2>(const SysParams&, const float*, int, float*, \
                                                    float*, size_t, bool*, cudaStream_t);        \
  EXT template cudaError_t grad_fused_launch<NL, 3>(const SysParams&, const float*, int, float*, \
                                                    float*, size_t, bool*, cudaStream_t);        \
  EXT template cudaError_t grad_fused_smem<NL, 1>(size_t);                                       \
  EXT template cudaError_t grad_fused_smem<NL, 2>(size_t);                                       \
  EXT template cudaError_t grad_fused_smem<NL, 3>(size_t);

}  // namespace gl
