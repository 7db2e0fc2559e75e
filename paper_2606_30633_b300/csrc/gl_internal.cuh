// Internal types of libgl shared by the C-ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

struct gl_surrogate;

namespace gl {

// NVTX range over one library call: named spans on an Nsight Systems
// timeline; a no-op unless a tool is attached (NVTX3 is header-only).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

constexpr int MAX_K = 21;      // largest PSF side
constexpr int MAX_S = 8;       // largest supersampling factor
constexpr int MAX_LIGHT = 2;   // lens-light components
constexpr int MAX_SRC = 3;     // source components
constexpr int MAX_COMP = MAX_LIGHT + MAX_SRC;
constexpr int MAX_P = 8 + 7 * MAX_COMP;
constexpr int N_MAX = 128;     // EPL series terms for |e| < 0.8 at FP32 tolerance
constexpr float TABLE_MIN_E = 1e-2f;  // rows with a smaller |e| use the series, not tables
constexpr int THREADS = 256;   // threads per CTA of the fused kernels
constexpr int NWARPS = THREADS / 32;
constexpr int ROWS_STRIP = 10;  // output rows per thread in the unrolled convolution
constexpr int TABLE_M = 128;   // surrogate angular table intervals over [0, pi)
constexpr int TABLE_ROW = 4 * TABLE_M;  // float4 per row's table (4 per interval)

// One prior entry as the kernels see it; cnst is the log normalisation
// constant, computed once at system creation.
struct PriorDev {
  int kind;
  float a, b, lo, hi;
  double cnst;
};

// Kernel parameter block of one system (passed by value: the PSF taps live in
// the constant bank, so the unrolled convolution reads them as FFMA operands).
struct SysParams {
  int ny, nx, s, P, nL, nS;
  int ky, kx, cy, cx;      // PSF size and centre
  int Hp, Wp;              // padded buffer size (rows, row pitch in floats)
  int bufA_smem, bufB_smem;  // buffer placement: 1 = dynamic shared memory
  size_t slot_floats;      // global scratch floats per CTA
  float D;                 // pixel scale (arcsec)
  float scale;             // D^2 / s^2
  float xg0, yg0;          // -(nx-1)/2, -(ny-1)/2
  float off[MAX_S];        // sub-pixel offsets (l + 1/2)/s - 1/2 (pixel units)
  const float* data;       // [ny*nx]
  const float* w;          // sigma^-2 [ny*nx]
  const PriorDev* prior;   // [P]
  const float* emax;       // [1 + nL + nS]
  float* scratch;          // global scratch base (CTA b uses slot b)
  const float4* table;     // surrogate tables [B][TABLE_ROW] (null: exact series)
  float sq_lo, sq_hi, sg_lo, sg_hi;  // surrogate domain in q and gamma
  // the network, for the fused kernel that builds each row's table itself
  // (null: tables come from `table` or the row uses the series)
  const unsigned char* net_wimg;  // packed weight operands of layers 1-4
  const void* net_wb;             // BF16 operands (__nv_bfloat16)
  const float* net_params;        // FP32 parameters (biases)
  int* net_timeout;               // set when a bounded tensor-core wait ran out
  int net_forced;                 // test hook: act as if the first wait ran out
  float kconv[MAX_K * MAX_K];  // flipped PSF: m = correlate(b_pad, kconv)
  float kcorr[MAX_K * MAX_K];  // PSF: adjoint = correlate(g_pad, kcorr)
};

// One work item (row) of an uneven multi-system batch.
struct MultiItem {
  int sys;              // index into the system table
  const float* theta;   // the row
  float* logp;
  float* grad;
  const float4* table;  // the row's surrogate/exact table (or null)
};

// Launch entry points (defined in the kernel translation units).
// img != nullptr: write the model image instead of reducing chi^2.
// sp.table != nullptr selects the surrogate instantiations.
cudaError_t launch_forward(const SysParams& sp, const float* theta, int B, float* logp,
                           float* img, size_t dyn_smem, cudaStream_t st);
// Images of single light components (k_component_images): one row per image.
cudaError_t launch_component_images(const SysParams& sp, const float* theta, int B, float* img,
                                    size_t dyn, cudaStream_t st);
cudaError_t launch_grad(const SysParams& sp, const float* theta, int B, float* logp, float* grad,
                        size_t dyn_smem, cudaStream_t st);
cudaError_t launch_leapfrog_block(const SysParams& sp, size_t dyn, float* theta, float* p,
                                  float* logp, float* grad, const float* inv_mass, float eps,
                                  int n_steps, int B, cudaStream_t st);
// Forward + adjoint with the surrogate's tables built by the network inside
// each row's CTA (sp.net_* set); false in *fits when two CTAs of it do not fit
// per SM with dyn_smem bytes, in which case nothing is launched.
cudaError_t launch_grad_fused(const SysParams& sp, const float* theta, int B, float* logp,
                              float* grad, size_t dyn_smem, bool* fits, cudaStream_t st);
// Persistent forward + adjoint over multi-system work items (MultiItem array),
// launch shape (threads per CTA 128 or 256, phase-1 pixel pairs 2 or 3).
cudaError_t launch_grad_multi(int nL, int nS, bool surr, int threads, int pairs,
                              const SysParams* systems, const void* items, int n_items,
                              int* counter, int grid, size_t dyn, cudaStream_t st);
// Per-row tables [B][TABLE_ROW] for the rows of theta (gl_surrogate.cu): from
// the network s (defl GL_DEFL_SURROGATE) or from the exact series in FP64
// (GL_DEFL_TABLE) or FP32 (GL_DEFL_TABLE32); s is ignored for the latter two.
cudaError_t launch_table(int defl, const gl_surrogate* s, const float* theta, int P, int B,
                         float4* table, cudaStream_t st);
// The (q, gamma) domain the tables of a deflection kind cover: the network's
// training domain for GL_DEFL_SURROGATE, |e| <= 0.5 for the exact tables.
void table_domain(int defl, const gl_surrogate* s, float* q_lo, float* q_hi, float* g_lo,
                  float* g_hi);
// The surrogate's device operands for the fused kernel (sp->net_*), the
// dynamic shared memory its network needs, and its timeout flag's reset
// before and stream-ordered copy to the host after a launch that may set it
// (gl_surrogate.cu).
void surrogate_net(const gl_surrogate* s, SysParams* sp);
size_t net_smem_bytes();
cudaError_t surrogate_flag_begin(const gl_surrogate* s, cudaStream_t st);
cudaError_t surrogate_flag_end(const gl_surrogate* s, cudaStream_t st);
// A valid deflection kind (gl_deflection), and whether it is the network.
inline bool defl_valid(int defl) { return defl >= 0 && defl <= 4; }
inline bool defl_network(int defl) { return defl == 1 || defl == 4; }

// Largest static shared memory of the forward and gradient kernels (bytes,
// with the surrogate table), or of the multi-system kernel of CTAs of
// `threads` threads.
size_t static_smem_bytes(bool multi = false, int threads = THREADS);
// Sets the kernels' dynamic shared-memory limit from the device's per-block
// maximum (each kernel's own static memory deducted).
cudaError_t set_smem_limits_fwd(size_t block_max);
cudaError_t set_smem_limits_grad(size_t block_max);

}  // namespace gl
