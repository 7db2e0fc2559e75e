// gl_logp_grad_noalloc: the fused log p + gradient kernel with its global
// scratch taken from a fixed array in the library instead of cudaMalloc.
//
// Who needs it: callers that are not allowed to allocate device memory after
// start-up, e.g. code running under a framework that owns a fixed device
// memory budget and forbids allocations behind its back, or a real-time
// sampling loop that cannot afford the implicit device synchronisation of
// cudaMalloc/cudaFree. The ordinary gl_logp_grad grows the system's scratch
// with cudaMalloc the first time a batch needs more; this entry point never
// allocates (no cudaMalloc, cudaFree or allocating library routine).
//
// The scratch is one file-scope __device__ array of GL_NOALLOC_SCRATCH_FLOATS
// floats (64 MiB) that every GPU which loads the library holds until the
// process exits. Images small enough for shared memory need none of it; for
// larger images every row of the batch needs a slot, and a batch whose slots
// do not fit is rejected with GL_EINVAL.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/gl.h"
#include "gl_internal.cuh"

namespace gl {
int system_grad_plan(const gl_system* sys, SysParams* sp, size_t* dyn_smem, size_t* slot_floats);
void set_last_error(const std::string& msg);
}

namespace {

static __device__ __align__(256) float g_noalloc_scratch[GL_NOALLOC_SCRATCH_FLOATS];

constexpr int kMaxDevices = 128;
std::mutex g_mu;
float* g_scratch_dev[kMaxDevices];  // device address of g_noalloc_scratch per device
gl_status fail(gl_status st, const std::string& msg) {
  gl::set_last_error("gl_logp_grad_noalloc: " + msg);
  return st;
}

// Host code may not use g_noalloc_scratch directly (on the host it is only a
// stand-in symbol); its device address is looked up once per device, with
// that device current, and kept for the life of the process (a device reset
// would leave it stale: the entry point is not for use after cudaDeviceReset).
cudaError_t scratch_address(int dev, float** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" gl_status gl_logp_grad_noalloc(gl_system* sys, const float* theta, int B, float* logp,
                                          float* grad, void* stream) {
  gl::Range nvtx_range("gl_logp_grad_noalloc");
  if (!sys) return fail(GL_EINVAL, "system is NULL");
  if (B < 0) return fail(GL_EINVAL, "B < 0");
  if (B > 0 && (!theta || !logp || !grad)) return fail(GL_EINVAL, "NULL theta, logp or grad");
  if (B == 0) return GL_OK;
  gl::SysParams sp;
  size_t dyn = 0, slot = 0;
  const int dev = gl::system_grad_plan(sys, &sp, &dyn, &slot);
  if (dev < 0 || dev >= kMaxDevices) return fail(GL_EINVAL, "unsupported device index");
  if (slot && (size_t)B * slot > (size_t)GL_NOALLOC_SCRATCH_FLOATS) {
    const size_t max_rows = (size_t)GL_NOALLOC_SCRATCH_FLOATS / slot;
    return fail(GL_EINVAL, "batch of " + std::to_string(B) + " rows needs " +
                               std::to_string((size_t)B * slot * sizeof(float)) +
                               " bytes of scratch, above the fixed " +
                               std::to_string((size_t)GL_NOALLOC_SCRATCH_FLOATS * sizeof(float)) +
                               "; split it into batches of at most " + std::to_string(max_rows) +
                               " rows");
  }
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return fail(GL_ECUDA, cudaGetErrorString(e));
  if (cur != dev) {
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) return fail(GL_ECUDA, cudaGetErrorString(e));
  }
  // the caller's current device is restored on every return below
  struct Restore {
    int dev, cur;
    ~Restore() {
      if (cur >= 0 && cur != dev) cudaSetDevice(cur);
    }
  } restore{dev, cur};
  if (slot) {
    float* base = nullptr;
    e = scratch_address(dev, &base);
    if (e != cudaSuccess) return fail(GL_ECUDA, std::string("scratch address: ") + cudaGetErrorString(e));
    sp.scratch = base;
  }
  e = gl::launch_grad(sp, theta, B, logp, grad, dyn, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(GL_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return GL_OK;
}
