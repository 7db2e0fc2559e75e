// The gl_system object (internal to libgl).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/gl.h"
#include "gl_internal.cuh"

namespace gl {
struct InferState;  // the inference layer's per-system state (gl_infer.cu)
}

struct gl_system {
  int device = 0;
  gl::SysParams sp;
  float* d_data = nullptr;
  float* d_w = nullptr;
  gl::PriorDev* d_prior = nullptr;
  float* d_emax = nullptr;
  // buffer plans (dynamic shared memory bytes and placement) per kernel kind
  size_t fwd_smem = 0, grad_smem = 0;
  int fwd_A = 1, grad_A = 1, grad_B = 1;
  size_t fwd_slot = 0, grad_slot = 0;  // global scratch floats per CTA
  float* scratch = nullptr;
  size_t scratch_floats = 0;
  // host-buffer entry point staging
  float *h_stage = nullptr, *d_stage = nullptr;
  size_t stage_floats = 0;
  const gl_surrogate* sur = nullptr;
  bool no_fused = false;  // the fused surrogate kernel does not fit two CTAs per SM here
  float4* d_table = nullptr;  // surrogate tables, [rows][TABLE_ROW]
  size_t table_rows = 0;
  // leapfrog block: one instantiated CUDA graph, re-captured when its
  // arguments (or the scratch it points into) change
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t lf_exec = nullptr;
  struct LfKey {
    float *theta, *p, *logp, *grad, *scratch;
    const float* inv_mass;
    float eps;
    int n_steps, B;
  } lf_key;
  gl::InferState* inf = nullptr;
};

namespace gl {
// Plans the buffer placement of a system for a shared-memory budget: dynamic
// shared memory bytes, placement flags and global floats per row (gl_api.cu).
void plan_buffers(size_t buf_floats, int nbufs, size_t smem_budget, size_t* dyn, int* a_smem,
                  int* b_smem, size_t* slot);
void set_last_error(const std::string& msg);
// Frees the inference layer's state of a system (gl_infer.cu).
void infer_release(gl_system* s);
// GL_ETIMEOUT (and clears it) if a table build of s that the host has seen
// complete ran out of its bounded tensor-core wait, else GL_OK. The table
// launch copies its flag to pinned host memory in stream order, so a timeout
// is reported by the first surrogate call after the failed build completed
// (like CUDA's own asynchronous errors).
gl_status surrogate_take_timeout(const gl_surrogate* s);  // gl_surrogate.cu
}  // namespace gl
