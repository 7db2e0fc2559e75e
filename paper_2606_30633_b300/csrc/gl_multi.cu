// Uneven multi-system batches: many lens systems of different image sizes,
// supersampling and component counts, each with its own rows and its own
// launch shape (threads per CTA, phase-1 pixel pairs per thread), evaluated
// by one persistent launch per group of systems that share component counts
// and shape. Work items (rows) are ordered heaviest first so the dynamic
// queue ends with short items (longest processing time first); every CTA
// keeps one global-scratch slot for the image buffers that do not fit in
// shared memory under the chosen policy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gl.h"
#include "gl_internal.cuh"
#include "gl_system.h"

namespace {

gl_status fail(gl_status st, const std::string& msg) {
  gl::set_last_error("multi: " + msg);
  return st;
}

#define MU_CUDA(call, what)                                                             \
  do {                                                                                  \
    cudaError_t _e = (call);                                                            \
    if (_e != cudaSuccess)                                                              \
      return fail(_e == cudaErrorMemoryAllocation ? GL_ENOMEM : GL_ECUDA,              \
                  std::string(what) + ": " + cudaGetErrorString(_e));                   \
  } while (0)

struct Group {
  int nL, nS, threads, pairs;
  std::vector<int> sys;  // systems of this group, heaviest first
  int n_items = 0;
  gl::MultiItem* d_items = nullptr;
  int grid = 0;          // persistent CTAs
  size_t dyn = 0;        // dynamic shared memory per CTA
  size_t slot = 0;       // global-scratch floats per CTA
  size_t scratch_off = 0;  // the group's scratch area (floats into the plan's)
  cudaStream_t stream = nullptr;  // the group's launch stream (concurrent groups)
  cudaEvent_t done = nullptr;
};

// CTAs per SM of a launch shape at 128 registers a thread.
int ctas_per_sm(int threads) { return 65536 / (threads * 128); }

}  // namespace

struct gl_multi {
  int device = 0;
  int policy = 1;
  std::vector<gl_system*> systems;
  std::vector<int> counts;
  std::vector<size_t> row_offset;  // first item (table row) of each system
  std::vector<Group> groups;
  gl::SysParams* d_sys = nullptr;
  std::vector<gl::SysParams> h_sys;
  int* d_counters = nullptr;
  float* scratch = nullptr;
  float4* d_table = nullptr;
  size_t total_rows = 0;
  int last_mode = -1;
  std::vector<const void*> last_ptrs;
  gl::MultiItem* h_items = nullptr;  // pinned staging of the item lists
  cudaEvent_t fork = nullptr;        // the caller's stream, ready for the group launches
};

extern "C" {

gl_status gl_multi_create_ex(gl_system* const* systems, int n_sys, const int* rows_per_sys,
                             int smem_policy, const int* threads_per_cta,
                             const int* pixel_pairs, gl_multi** out) {
  if (!out) return fail(GL_EINVAL, "out is NULL");
  *out = nullptr;
  if (!systems || !rows_per_sys || n_sys < 1) return fail(GL_EINVAL, "need >= 1 system");
  if (smem_policy < 0 || smem_policy > 2) return fail(GL_EINVAL, "smem_policy must be 0, 1 or 2");
  for (int k = 0; k < n_sys; ++k) {
    if (!systems[k]) return fail(GL_EINVAL, "NULL system");
    if (rows_per_sys[k] < 0) return fail(GL_EINVAL, "negative row count");
    if (threads_per_cta && threads_per_cta[k] != 128 && threads_per_cta[k] != 256)
      return fail(GL_EINVAL, "threads_per_cta must be 128 or 256");
    if (pixel_pairs && pixel_pairs[k] != 2 && pixel_pairs[k] != 3)
      return fail(GL_EINVAL, "pixel_pairs must be 2 or 3");
  }
  gl_multi* m = new gl_multi();
  auto bail = [&](gl_status st) {
    gl_multi_destroy(m);
    return st;
  };
  cudaGetDevice(&m->device);
  m->policy = smem_policy;
  m->systems.assign(systems, systems + n_sys);
  m->counts.assign(rows_per_sys, rows_per_sys + n_sys);
  int sms = 0, smem_sm = 0, smem_blk = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, m->device);
  cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device);
  // per launch shape: CTAs per SM under the policy and the dynamic shared
  // memory budget of one CTA (static memory with the table + system reserve
  // deducted)
  auto shape_plan = [&](int threads, int* ctas, size_t* budget) {
    const size_t reserve = gl::static_smem_bytes(true, threads) + 1024;
    const int full = ctas_per_sm(threads);
    *ctas = smem_policy == 2 ? 1 : full;
    const size_t share = smem_policy == 2 ? (size_t)smem_blk : (size_t)smem_sm / full;
    *budget = smem_policy == 0 ? 0 : (share > reserve ? share - reserve : 0);
  };
  if ((size_t)smem_blk <= gl::static_smem_bytes(true, 256) + 1024)
    return bail(fail(GL_ECUDA, "device shared memory too small"));
  // per-system plans under their shape's budget
  m->h_sys.resize(n_sys);
  m->row_offset.resize(n_sys);
  std::vector<size_t> sys_dyn(n_sys), sys_slot(n_sys);
  std::vector<int> sys_threads(n_sys), sys_pairs(n_sys);
  for (int k = 0; k < n_sys; ++k) {
    gl_system* s = systems[k];
    if (s->device != m->device) return bail(fail(GL_EINVAL, "systems must share the current device"));
    sys_threads[k] = threads_per_cta ? threads_per_cta[k] : 256;
    sys_pairs[k] = pixel_pairs ? pixel_pairs[k] : 2;
    int ctas = 0;
    size_t budget = 0;
    shape_plan(sys_threads[k], &ctas, &budget);
    gl::SysParams sp = s->sp;
    const size_t nbuf = ((size_t)sp.Hp * sp.Wp + 3) & ~(size_t)3;
    size_t d = 0, sl = 0;
    int a = 0, b = 0;
    gl::plan_buffers(nbuf, 2, budget, &d, &a, &b, &sl);
    sp.bufA_smem = a;
    sp.bufB_smem = b;
    sys_dyn[k] = d;
    sys_slot[k] = sl;
    m->h_sys[k] = sp;
    m->row_offset[k] = m->total_rows;
    m->total_rows += rows_per_sys[k];
  }
  // groups by component counts and launch shape, systems heaviest first
  std::vector<int> order(n_sys);
  for (int k = 0; k < n_sys; ++k) order[k] = k;
  auto cost = [&](int k) {
    const gl::SysParams& sp = m->h_sys[k];
    return (double)sp.ny * sp.nx * sp.s * sp.s * (4.0 + sp.nL + sp.nS);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  for (int k : order) {
    const gl::SysParams& sp = m->h_sys[k];
    auto it = std::find_if(m->groups.begin(), m->groups.end(), [&](const Group& g) {
      return g.nL == sp.nL && g.nS == sp.nS && g.threads == sys_threads[k] &&
             g.pairs == sys_pairs[k];
    });
    if (it == m->groups.end()) {
      Group g{sp.nL, sp.nS, sys_threads[k], sys_pairs[k], {}, 0, nullptr};
      int ctas = 0;
      size_t budget = 0;
      shape_plan(g.threads, &ctas, &budget);
      g.grid = sms * ctas;
      m->groups.push_back(g);
      it = m->groups.end() - 1;
    }
    it->sys.push_back(k);
    it->n_items += rows_per_sys[k];
    it->dyn = std::max(it->dyn, sys_dyn[k]);
    it->slot = std::max(it->slot, sys_slot[k]);
  }
  // a scratch area per group: the groups' persistent launches run
  // concurrently (each on its own stream), so that one group's tail overlaps
  // the next group's start
  size_t scratch_floats = 0;
  for (auto& g : m->groups) {
    g.scratch_off = scratch_floats;
    scratch_floats += (size_t)g.grid * g.slot;
    for (int k : g.sys) m->h_sys[k].slot_floats = g.slot;
  }
  if (cudaMalloc(&m->d_sys, n_sys * sizeof(gl::SysParams)) != cudaSuccess ||
      cudaMalloc(&m->d_counters, m->groups.size() * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&m->h_items, std::max<size_t>(m->total_rows, 1) * sizeof(gl::MultiItem)) != cudaSuccess)
    return bail(fail(GL_ENOMEM, "multi allocation"));
  for (auto& g : m->groups)
    if (cudaMalloc(&g.d_items, std::max(g.n_items, 1) * sizeof(gl::MultiItem)) != cudaSuccess)
      return bail(fail(GL_ENOMEM, "multi item allocation"));
  if (scratch_floats && cudaMalloc(&m->scratch, scratch_floats * sizeof(float)) != cudaSuccess)
    return bail(fail(GL_ENOMEM, "multi scratch allocation"));
  for (auto& g : m->groups)
    for (int k : g.sys) m->h_sys[k].scratch = m->scratch ? m->scratch + g.scratch_off : nullptr;
  if (cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(GL_ECUDA, "multi event"));
  for (auto& g : m->groups)
    if (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess)
      return bail(fail(GL_ECUDA, "multi stream"));
  if (gl::set_smem_limits_grad((size_t)smem_blk) != cudaSuccess)
    return bail(fail(GL_ECUDA, "kernel shared-memory limit"));
  *out = m;
  return GL_OK;
}

gl_status gl_multi_create(gl_system* const* systems, int n_sys, const int* rows_per_sys,
                          int smem_policy, gl_multi** out) {
  return gl_multi_create_ex(systems, n_sys, rows_per_sys, smem_policy, nullptr, nullptr, out);
}

gl_status gl_multi_logp_grad(gl_multi* m, const float* const* theta, float* const* logp,
                             float* const* grad, gl_deflection defl, void* stream) {
  gl::Range nvtx_range("gl_multi_logp_grad");
  if (!m) return fail(GL_EINVAL, "multi is NULL");
  if (!theta || !logp || !grad) return fail(GL_EINVAL, "NULL pointer arrays");
  if (!gl::defl_valid(defl)) return fail(GL_EINVAL, "unknown deflection kind");
  const int n_sys = (int)m->systems.size();
  for (int k = 0; k < n_sys; ++k) {
    if (m->counts[k] > 0 && (!theta[k] || !logp[k] || !grad[k]))
      return fail(GL_EINVAL, "NULL theta, logp or grad for a system with rows");
    if (gl::defl_network(defl) && !m->systems[k]->sur)
      return fail(GL_ENOSURROGATE, "a system has no surrogate attached");
  }
  if (gl::defl_network(defl))
    for (int k = 0; k < n_sys; ++k) {
      const gl_status r = gl::surrogate_take_timeout(m->systems[k]->sur);
      if (r != GL_OK) return r;
    }
  cudaStream_t st = (cudaStream_t)stream;
  int cur = -1;
  MU_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
  if (cur != m->device) MU_CUDA(cudaSetDevice(m->device), "cudaSetDevice");
  const bool surr = defl != GL_DEFL_SERIES;
  if (surr) {
    if (!m->d_table)
      MU_CUDA(cudaMalloc(&m->d_table, std::max<size_t>(m->total_rows, 1) * gl::TABLE_ROW *
                                          sizeof(float4)),
              "table allocation");
    for (int k = 0; k < n_sys; ++k) {
      if (!m->counts[k]) continue;
      MU_CUDA(gl::launch_table(defl, m->systems[k]->sur, theta[k], m->h_sys[k].P, m->counts[k],
                               m->d_table + m->row_offset[k] * gl::TABLE_ROW, st),
              "table launch");
    }
  }
  // system parameters for this deflection kind
  if (m->last_mode != (int)defl) {
    for (int k = 0; k < n_sys; ++k) {
      gl::SysParams& sp = m->h_sys[k];
      if (surr) {
        sp.table = m->d_table;
        gl::table_domain(defl, m->systems[k]->sur, &sp.sq_lo, &sp.sq_hi, &sp.sg_lo, &sp.sg_hi);
      } else {
        sp.table = nullptr;
      }
    }
    MU_CUDA(cudaMemcpyAsync(m->d_sys, m->h_sys.data(), n_sys * sizeof(gl::SysParams),
                            cudaMemcpyHostToDevice, st),
            "system table upload");
    m->last_mode = (int)defl;
  }
  // work items (rebuilt when the caller's pointers change)
  std::vector<const void*> ptrs;
  for (int k = 0; k < n_sys; ++k) {
    ptrs.push_back(theta[k]);
    ptrs.push_back(logp[k]);
    ptrs.push_back(grad[k]);
  }
  ptrs.push_back(surr ? (const void*)m->d_table : nullptr);
  if (ptrs != m->last_ptrs) {
    MU_CUDA(cudaStreamSynchronize(st), "synchronize before item upload");
    size_t off = 0;
    for (auto& g : m->groups) {
      gl::MultiItem* it = m->h_items + off;
      int n = 0;
      for (int k : g.sys) {
        const int P = m->h_sys[k].P;
        for (int r = 0; r < m->counts[k]; ++r, ++n) {
          it[n].sys = k;
          it[n].theta = theta[k] + (size_t)r * P;
          it[n].logp = logp[k] + r;
          it[n].grad = grad[k] + (size_t)r * P;
          it[n].table = surr ? m->d_table + (m->row_offset[k] + r) * gl::TABLE_ROW : nullptr;
        }
      }
      MU_CUDA(cudaMemcpyAsync(g.d_items, it, n * sizeof(gl::MultiItem), cudaMemcpyHostToDevice, st),
              "item upload");
      off += n;
    }
    m->last_ptrs = ptrs;
  }
  MU_CUDA(cudaMemsetAsync(m->d_counters, 0, m->groups.size() * sizeof(int), st), "counter reset");
  // fork: every group's launch waits for the work above on the caller's
  // stream; join: the caller's stream waits for every group
  MU_CUDA(cudaEventRecord(m->fork, st), "fork record");
  for (size_t gi = 0; gi < m->groups.size(); ++gi) {
    const Group& g = m->groups[gi];
    if (!g.n_items) continue;
    MU_CUDA(cudaStreamWaitEvent(g.stream, m->fork, 0), "fork wait");
    MU_CUDA(gl::launch_grad_multi(g.nL, g.nS, surr, g.threads, g.pairs, m->d_sys, g.d_items,
                                  g.n_items, m->d_counters + gi, std::min(g.grid, g.n_items),
                                  g.dyn, g.stream),
            "multi launch");
    MU_CUDA(cudaEventRecord(g.done, g.stream), "join record");
    MU_CUDA(cudaStreamWaitEvent(st, g.done, 0), "join wait");
  }
  return GL_OK;
}

gl_status gl_multi_destroy(gl_multi* m) {
  if (!m) return GL_OK;
  cudaDeviceSynchronize();
  for (auto& g : m->groups) {
    cudaFree(g.d_items);
    if (g.done) cudaEventDestroy(g.done);
    if (g.stream) cudaStreamDestroy(g.stream);
  }
  if (m->fork) cudaEventDestroy(m->fork);
  cudaFree(m->d_sys);
  cudaFree(m->d_counters);
  cudaFree(m->scratch);
  cudaFree(m->d_table);
  cudaFreeHost(m->h_items);
  delete m;
  return GL_OK;
}

}  // extern "C"
