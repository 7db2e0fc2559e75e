// Uneven multi-system batches: many lens systems of different image sizes,
// supersampling and component counts, each with its own rows, evaluated by
// one persistent launch per component-count group. Work items (rows) are
// ordered heaviest first so the dynamic queue ends with short items (longest
// processing time first); every CTA keeps one global-scratch slot for the
// image buffers that do not fit in shared memory under the chosen policy.
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
  int nL, nS;
  std::vector<int> sys;  // systems of this group, heaviest first
  int n_items = 0;
  gl::MultiItem* d_items = nullptr;
};

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
  size_t slot_floats = 0;
  size_t dyn = 0;
  int grid = 0;
  float4* d_table = nullptr;
  size_t total_rows = 0;
  int last_mode = -1;
  std::vector<const void*> last_ptrs;
  gl::MultiItem* h_items = nullptr;  // pinned staging of the item lists
};

extern "C" {

gl_status gl_multi_create(gl_system* const* systems, int n_sys, const int* rows_per_sys,
                          int smem_policy, gl_multi** out) {
  if (!out) return fail(GL_EINVAL, "out is NULL");
  *out = nullptr;
  if (!systems || !rows_per_sys || n_sys < 1) return fail(GL_EINVAL, "need >= 1 system");
  if (smem_policy < 0 || smem_policy > 2) return fail(GL_EINVAL, "smem_policy must be 0, 1 or 2");
  for (int k = 0; k < n_sys; ++k) {
    if (!systems[k]) return fail(GL_EINVAL, "NULL system");
    if (rows_per_sys[k] < 0) return fail(GL_EINVAL, "negative row count");
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
  const size_t stat = gl::static_smem_bytes(true);
  const size_t reserve = stat + 1024;  // static shared memory (with the table) + system reserve
  if ((size_t)smem_blk <= reserve) return bail(fail(GL_ECUDA, "device shared memory too small"));
  size_t budget = 0;
  int ctas = 2;
  if (smem_policy == 1) budget = (size_t)smem_sm / 2 > reserve ? (size_t)smem_sm / 2 - reserve : 0;
  if (smem_policy == 2) {
    budget = (size_t)smem_blk > reserve ? (size_t)smem_blk - reserve : 0;
    ctas = 1;
  }
  m->grid = sms * ctas;
  // per-system plans under the common budget
  m->h_sys.resize(n_sys);
  m->row_offset.resize(n_sys);
  size_t dyn = 0, slot = 0;
  for (int k = 0; k < n_sys; ++k) {
    gl_system* s = systems[k];
    if (s->device != m->device) return bail(fail(GL_EINVAL, "systems must share the current device"));
    gl::SysParams sp = s->sp;
    const size_t nbuf = ((size_t)sp.Hp * sp.Wp + 3) & ~(size_t)3;
    size_t d = 0, sl = 0;
    int a = 0, b = 0;
    gl::plan_buffers(nbuf, 2, budget, &d, &a, &b, &sl);
    sp.bufA_smem = a;
    sp.bufB_smem = b;
    dyn = std::max(dyn, d);
    slot = std::max(slot, sl);
    m->h_sys[k] = sp;
    m->row_offset[k] = m->total_rows;
    m->total_rows += rows_per_sys[k];
  }
  m->dyn = dyn;
  m->slot_floats = slot;
  for (auto& sp : m->h_sys) sp.slot_floats = slot;
  // groups by component counts, systems heaviest first
  std::vector<int> order(n_sys);
  for (int k = 0; k < n_sys; ++k) order[k] = k;
  auto cost = [&](int k) {
    const gl::SysParams& sp = m->h_sys[k];
    return (double)sp.ny * sp.nx * sp.s * sp.s * (4.0 + sp.nL + sp.nS);
  };
  std::sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  for (int k : order) {
    const gl::SysParams& sp = m->h_sys[k];
    auto it = std::find_if(m->groups.begin(), m->groups.end(),
                           [&](const Group& g) { return g.nL == sp.nL && g.nS == sp.nS; });
    if (it == m->groups.end()) {
      m->groups.push_back(Group{sp.nL, sp.nS, {}, 0, nullptr});
      it = m->groups.end() - 1;
    }
    it->sys.push_back(k);
    it->n_items += rows_per_sys[k];
  }
  if (cudaMalloc(&m->d_sys, n_sys * sizeof(gl::SysParams)) != cudaSuccess ||
      cudaMalloc(&m->d_counters, m->groups.size() * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&m->h_items, std::max<size_t>(m->total_rows, 1) * sizeof(gl::MultiItem)) != cudaSuccess)
    return bail(fail(GL_ENOMEM, "multi allocation"));
  for (auto& g : m->groups)
    if (cudaMalloc(&g.d_items, std::max(g.n_items, 1) * sizeof(gl::MultiItem)) != cudaSuccess)
      return bail(fail(GL_ENOMEM, "multi item allocation"));
  if (slot && cudaMalloc(&m->scratch, (size_t)m->grid * slot * sizeof(float)) != cudaSuccess)
    return bail(fail(GL_ENOMEM, "multi scratch allocation"));
  for (auto& sp : m->h_sys) sp.scratch = m->scratch;
  if (gl::set_smem_limits_grad((size_t)smem_blk) != cudaSuccess)
    return bail(fail(GL_ECUDA, "kernel shared-memory limit"));
  *out = m;
  return GL_OK;
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
    if (defl == GL_DEFL_SURROGATE && !m->systems[k]->sur)
      return fail(GL_ENOSURROGATE, "a system has no surrogate attached");
  }
  if (defl == GL_DEFL_SURROGATE)
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
  for (size_t gi = 0; gi < m->groups.size(); ++gi) {
    const Group& g = m->groups[gi];
    if (!g.n_items) continue;
    MU_CUDA(gl::launch_grad_multi(g.nL, g.nS, surr, m->d_sys, g.d_items, g.n_items,
                                  m->d_counters + gi, std::min(m->grid, g.n_items), m->dyn, st),
            "multi launch");
  }
  return GL_OK;
}

gl_status gl_multi_destroy(gl_multi* m) {
  if (!m) return GL_OK;
  cudaDeviceSynchronize();
  for (auto& g : m->groups) cudaFree(g.d_items);
  cudaFree(m->d_sys);
  cudaFree(m->d_counters);
  cudaFree(m->scratch);
  cudaFree(m->d_table);
  cudaFreeHost(m->h_items);
  delete m;
  return GL_OK;
}

}  // extern "C"
