// C ABI of libgl: system objects, argument validation, buffer planning and
// launches. All model arithmetic runs in the kernels; the host only checks
// arguments, copies inputs and normalises the PSF once at creation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gl.h"
#include "gl_internal.cuh"
#include "gl_system.h"

using gl::PriorDev;
using gl::SysParams;



namespace {

thread_local std::string g_last_error;

gl_status fail(gl_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

gl_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? GL_ENOMEM : GL_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define GL_CUDA(call, what)                        \
  do {                                             \
    cudaError_t _e = (call);                       \
    if (_e != cudaSuccess) return cuda_fail(_e, what); \
  } while (0)

__global__ void k_prior_setup(PriorDev* pr, int P) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P) return;
  const double a = pr[k].a, b = pr[k].b, lo = pr[k].lo, hi = pr[k].hi;
  const double ls2p = 0.91893853320467274178;  // log(2 pi)/2
  double c = 0.0;
  switch (pr[k].kind) {
    case 1: c = -log(hi - lo); break;
    case 2: c = -(log(b) + ls2p); break;
    case 3: {
      const double mass = 0.5 * erfc(-(hi - a) / b * 0.70710678118654752440) -
                          0.5 * erfc(-(lo - a) / b * 0.70710678118654752440);
      c = -(log(b) + ls2p) - log(mass);
      break;
    }
    case 4: c = -(log(b) + ls2p); break;
    default: break;
  }
  pr[k].cnst = c;
}

__global__ void k_weights(const float* sigma, float* w, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double s = sigma[k];
  w[k] = isinf(s) ? 0.f : (float)(1.0 / (s * s));
}

size_t align4(size_t n) { return (n + 3) & ~(size_t)3; }

}  // namespace

namespace gl {
// Chooses buffer placement for a kernel needing nbufs padded images: all in
// shared memory when they fit the budget, else the first one when it fits,
// else global scratch.
void plan_buffers(size_t buf_floats, int nbufs, size_t smem_budget, size_t* dyn, int* a_smem, int* b_smem,
          size_t* slot) {
  const size_t bb = buf_floats * sizeof(float);
  *a_smem = 0;
  *b_smem = 0;
  *dyn = 0;
  *slot = 0;
  if (nbufs * bb <= smem_budget) {
    *a_smem = 1;
    *b_smem = nbufs > 1;
    *dyn = nbufs * bb;
  } else if (nbufs > 1 && bb <= smem_budget) {
    *a_smem = 1;
    *dyn = bb;
    *slot = buf_floats;
  } else {
    *slot = nbufs * buf_floats;
  }
}
}  // namespace gl

namespace {

// True when [p, p + bytes) starts and ends in page-locked host memory, which
// the copy engines read and write directly. An unregistered pointer is not an
// error for the query (its type is cudaMemoryTypeUnregistered); any error it
// does return is cleared.
bool page_locked(const void* p, size_t bytes) {
  const char* c = static_cast<const char*>(p);
  for (const char* q : {c, c + bytes - 1}) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (a.type != cudaMemoryTypeHost) return false;
  }
  return true;
}

gl_status ensure_scratch(gl_system* s, size_t floats) {
  if (floats <= s->scratch_floats) return GL_OK;
  if (s->scratch) cudaFree(s->scratch);
  s->scratch = nullptr;
  s->scratch_floats = 0;
  GL_CUDA(cudaMalloc(&s->scratch, floats * sizeof(float)), "scratch allocation");
  s->scratch_floats = floats;
  return GL_OK;
}

// Builds the surrogate tables for B rows and points sp at them.
gl_status prepare_surrogate(gl_system* s, const float* theta, int B, SysParams& sp,
                            gl_deflection defl, cudaStream_t st) {
  if (gl::defl_network(defl)) {
    gl_status r = gl::surrogate_take_timeout(s->sur);
    if (r != GL_OK) return r;
  }
  if ((size_t)B > s->table_rows) {
    cudaFree(s->d_table);
    s->d_table = nullptr;
    s->table_rows = 0;
    GL_CUDA(cudaMalloc(&s->d_table, (size_t)B * gl::TABLE_ROW * sizeof(float4)),
            "surrogate table allocation");
    s->table_rows = B;
  }
  GL_CUDA(gl::launch_table(defl, s->sur, theta, s->sp.P, B, s->d_table, st), "table launch");
  sp.table = s->d_table;
  gl::table_domain(defl, s->sur, &sp.sq_lo, &sp.sq_hi, &sp.sg_lo, &sp.sg_hi);
  return GL_OK;
}

gl_status check_call(gl_system* sys, const void* theta, int B, const void* out,
                     gl_deflection defl) {
  if (!sys) return fail(GL_EINVAL, "system is NULL");
  if (B < 0) return fail(GL_EINVAL, "B < 0");
  if (B > 0 && (!theta || !out)) return fail(GL_EINVAL, "NULL theta or output");
  if (!gl::defl_valid(defl)) return fail(GL_EINVAL, "unknown deflection kind");
  if (gl::defl_network(defl) && !sys->sur)
    return fail(GL_ENOSURROGATE, "no surrogate attached to this system");
  return GL_OK;
}

gl_status set_device(gl_system* sys) {
  int cur = -1;
  GL_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
  if (cur != sys->device) GL_CUDA(cudaSetDevice(sys->device), "cudaSetDevice");
  return GL_OK;
}

}  // namespace

extern "C" {

const char* gl_last_error(void) { return g_last_error.c_str(); }

gl_status gl_system_set_surrogate(gl_system* sys, const gl_surrogate* sur) {
  if (!sys) return fail(GL_EINVAL, "system is NULL");
  sys->sur = sur;
  return GL_OK;
}

int gl_system_num_params(const gl_system* sys) { return sys ? sys->sp.P : -1; }

gl_status gl_system_create(const gl_system_desc* d, gl_system** out) {
  if (!out) return fail(GL_EINVAL, "out is NULL");
  *out = nullptr;
  if (!d) return fail(GL_EINVAL, "desc is NULL");
  if (d->ny < 1 || d->nx < 1 || d->ny > 2048 || d->nx > 2048)
    return fail(GL_EINVAL, "image size must be 1..2048 per side");
  if (!(d->pixel_scale > 0.f) || !std::isfinite(d->pixel_scale))
    return fail(GL_EINVAL, "pixel_scale must be positive and finite");
  if (d->supersample < 1 || d->supersample > gl::MAX_S)
    return fail(GL_EINVAL, "supersample must be 1..8");
  if (d->psf_ny < 1 || d->psf_nx < 1 || d->psf_ny > gl::MAX_K || d->psf_nx > gl::MAX_K ||
      d->psf_ny % 2 == 0 || d->psf_nx % 2 == 0)
    return fail(GL_EINVAL, "PSF sides must be odd, 1..21");
  if (d->n_lens_light < 0 || d->n_lens_light > gl::MAX_LIGHT)
    return fail(GL_EINVAL, "n_lens_light must be 0..2");
  if (d->n_source < 1 || d->n_source > gl::MAX_SRC) return fail(GL_EINVAL, "n_source must be 1..3");
  if (!d->data || !d->sigma || !d->psf || !d->prior)
    return fail(GL_EINVAL, "data, sigma, psf and prior are required");
  const int P = 8 + 7 * (d->n_lens_light + d->n_source);
  const int nc = 1 + d->n_lens_light + d->n_source;
  const size_t npix = (size_t)d->ny * d->nx;
  const size_t nk = (size_t)d->psf_ny * d->psf_nx;

  std::vector<float> data(npix), sigma(npix), psf(nk);
  if (d->inputs_on_device) {
    GL_CUDA(cudaMemcpy(data.data(), d->data, npix * 4, cudaMemcpyDeviceToHost), "copy data");
    GL_CUDA(cudaMemcpy(sigma.data(), d->sigma, npix * 4, cudaMemcpyDeviceToHost), "copy sigma");
    GL_CUDA(cudaMemcpy(psf.data(), d->psf, nk * 4, cudaMemcpyDeviceToHost), "copy psf");
  } else {
    std::memcpy(data.data(), d->data, npix * 4);
    std::memcpy(sigma.data(), d->sigma, npix * 4);
    std::memcpy(psf.data(), d->psf, nk * 4);
  }
  for (size_t k = 0; k < npix; ++k) {
    if (!std::isfinite(data[k])) return fail(GL_EINVAL, "data holds a non-finite value");
    if (!(sigma[k] > 0.f)) return fail(GL_EINVAL, "sigma must be > 0 (+inf masks a pixel)");
  }
  double psum = 0.0;
  for (size_t k = 0; k < nk; ++k) {
    if (!std::isfinite(psf[k])) return fail(GL_EINVAL, "PSF holds a non-finite value");
    psum += psf[k];
  }
  if (!(psum > 0.0)) return fail(GL_EINVAL, "PSF sum must be positive");
  std::vector<PriorDev> prior(P);
  for (int k = 0; k < P; ++k) {
    const gl_prior& p = d->prior[k];
    PriorDev& q = prior[k];
    q.kind = p.kind;
    q.a = p.a;
    q.b = p.b;
    q.lo = p.lo;
    q.hi = p.hi;
    q.cnst = 0.0;
    char msg[96];
    std::snprintf(msg, sizeof msg, "invalid prior for parameter %d", k);
    switch (p.kind) {
      case GL_PRIOR_FLAT:
        if (!(p.lo <= p.hi)) return fail(GL_EINVAL, msg);
        break;
      case GL_PRIOR_UNIFORM:
        if (!(std::isfinite(p.lo) && std::isfinite(p.hi) && p.lo < p.hi)) return fail(GL_EINVAL, msg);
        break;
      case GL_PRIOR_NORMAL:
      case GL_PRIOR_LOGNORMAL:
        if (!(std::isfinite(p.a) && p.b > 0.f && std::isfinite(p.b))) return fail(GL_EINVAL, msg);
        break;
      case GL_PRIOR_TRUNCNORM:
        if (!(std::isfinite(p.a) && p.b > 0.f && std::isfinite(p.b) && p.lo < p.hi))
          return fail(GL_EINVAL, msg);
        break;
      default:
        return fail(GL_EINVAL, msg);
    }
  }
  std::vector<float> emax(nc, 0.f);
  if (d->emax) {
    for (int c = 0; c < nc; ++c) {
      if (!(d->emax[c] >= 0.f) || !std::isfinite(d->emax[c]))
        return fail(GL_EINVAL, "emax entries must be finite and >= 0");
      emax[c] = d->emax[c];
    }
  }

  gl_system* s = new gl_system();
  auto bail = [&](gl_status st) {
    gl_system_destroy(s);
    return st;
  };
  if (cudaGetDevice(&s->device) != cudaSuccess) return bail(fail(GL_ECUDA, "no CUDA device"));
  SysParams& sp = s->sp;
  std::memset(&sp, 0, sizeof sp);
  sp.ny = d->ny;
  sp.nx = d->nx;
  sp.s = d->supersample;
  sp.P = P;
  sp.nL = d->n_lens_light;
  sp.nS = d->n_source;
  sp.ky = d->psf_ny;
  sp.kx = d->psf_nx;
  sp.cy = (sp.ky - 1) / 2;
  sp.cx = (sp.kx - 1) / 2;
  sp.Hp = ((sp.ny + gl::ROWS_STRIP - 1) / gl::ROWS_STRIP) * gl::ROWS_STRIP + sp.ky - 1;
  sp.Wp = sp.nx + sp.kx - 1;
  sp.D = d->pixel_scale;
  sp.scale = (float)((double)d->pixel_scale * d->pixel_scale / ((double)sp.s * sp.s));
  sp.xg0 = -0.5f * (float)(sp.nx - 1);
  sp.yg0 = -0.5f * (float)(sp.ny - 1);
  for (int l = 0; l < sp.s; ++l) sp.off[l] = (float)((l + 0.5) / sp.s - 0.5);
  for (int u = 0; u < sp.ky; ++u)
    for (int v = 0; v < sp.kx; ++v) {
      const float k = (float)(psf[(size_t)u * sp.kx + v] / psum);
      sp.kcorr[u * sp.kx + v] = k;
      sp.kconv[(sp.ky - 1 - u) * sp.kx + (sp.kx - 1 - v)] = k;
    }

  if (cudaMalloc(&s->d_data, npix * 4) != cudaSuccess || cudaMalloc(&s->d_w, npix * 4) != cudaSuccess ||
      cudaMalloc(&s->d_prior, P * sizeof(PriorDev)) != cudaSuccess ||
      cudaMalloc(&s->d_emax, nc * sizeof(float)) != cudaSuccess)
    return bail(fail(GL_ENOMEM, "device allocation failed"));
  float* d_sigma = nullptr;
  if (cudaMalloc(&d_sigma, npix * 4) != cudaSuccess) return bail(fail(GL_ENOMEM, "device allocation failed"));
  cudaError_t e = cudaMemcpy(s->d_data, data.data(), npix * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d_sigma, sigma.data(), npix * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(s->d_prior, prior.data(), P * sizeof(PriorDev), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_emax, emax.data(), nc * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_weights<<<(unsigned)((npix + 255) / 256), 256>>>(d_sigma, s->d_w, (int)npix);
    k_prior_setup<<<1, 64>>>(s->d_prior, P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(d_sigma);
  if (e != cudaSuccess) return bail(cuda_fail(e, "system upload"));
  sp.data = s->d_data;
  sp.w = s->d_w;
  sp.prior = s->d_prior;
  sp.emax = s->d_emax;

  // buffer plans: a CTA keeps two resident per SM when it can
  int dev = s->device, smem_sm = 0, smem_blk = 0;
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t static_smem = gl::static_smem_bytes() + 1024;  // static + per-CTA reservation
  size_t budget = (size_t)smem_sm / 2 > static_smem ? (size_t)smem_sm / 2 - static_smem : 0;
  if (budget + static_smem > (size_t)smem_blk)
    budget = (size_t)smem_blk > static_smem ? smem_blk - static_smem : 0;
  const size_t nbuf = align4((size_t)sp.Hp * sp.Wp);
  int bdummy = 0;
  gl::plan_buffers(nbuf, 1, budget, &s->fwd_smem, &s->fwd_A, &bdummy, &s->fwd_slot);
  gl::plan_buffers(nbuf, 2, budget, &s->grad_smem, &s->grad_A, &s->grad_B, &s->grad_slot);
  // the attribute is per kernel and process-wide: always the device maximum
  // (less the kernel's static memory), so that no system or plan lowers
  // another's limit (it does not change occupancy, which follows each
  // launch's own size)
  e = gl::set_smem_limits_fwd((size_t)smem_blk);
  if (e == cudaSuccess) e = gl::set_smem_limits_grad((size_t)smem_blk);
  if (e != cudaSuccess) return bail(cuda_fail(e, "kernel shared-memory limit"));
  g_last_error.clear();
  *out = s;
  return GL_OK;
}

gl_status gl_system_destroy(gl_system* s) {
  if (!s) return GL_OK;
  cudaDeviceSynchronize();
  gl::infer_release(s);
  if (s->lf_exec) cudaGraphExecDestroy(s->lf_exec);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  cudaFree(s->d_data);
  cudaFree(s->d_w);
  cudaFree(s->d_prior);
  cudaFree(s->d_emax);
  cudaFree(s->scratch);
  cudaFree(s->d_table);
  cudaFree(s->d_stage);
  cudaFreeHost(s->h_stage);
  delete s;
  return GL_OK;
}

static gl_status run_forward(gl_system* sys, const float* theta, int B, float* logp, float* img,
                             gl_deflection defl, cudaStream_t st) {
  SysParams sp = sys->sp;
  if (defl != GL_DEFL_SERIES) {
    gl_status r = prepare_surrogate(sys, theta, B, sp, defl, st);
    if (r != GL_OK) return r;
  }
  sp.bufA_smem = sys->fwd_A;
  sp.bufB_smem = 0;
  sp.slot_floats = sys->fwd_slot;
  if (sys->fwd_slot) {
    gl_status r = ensure_scratch(sys, (size_t)B * sys->fwd_slot);
    if (r != GL_OK) return r;
    sp.scratch = sys->scratch;
  }
  GL_CUDA(gl::launch_forward(sp, theta, B, logp, img, sys->fwd_smem, st), "forward launch");
  return GL_OK;
}

gl_status gl_logp(gl_system* sys, const float* theta, int B, float* logp, gl_deflection defl,
                  void* stream) {
  gl::Range nvtx_range("gl_logp");
  gl_status r = check_call(sys, theta, B, logp, defl);
  if (r != GL_OK) return r;
  if (B == 0) return GL_OK;
  if ((r = set_device(sys)) != GL_OK) return r;
  return run_forward(sys, theta, B, logp, nullptr, defl, (cudaStream_t)stream);
}

gl_status gl_model_image(gl_system* sys, const float* theta, int B, float* img,
                         gl_deflection defl, void* stream) {
  gl::Range nvtx_range("gl_model_image");
  gl_status r = check_call(sys, theta, B, img, defl);
  if (r != GL_OK) return r;
  if (B == 0) return GL_OK;
  if ((r = set_device(sys)) != GL_OK) return r;
  return run_forward(sys, theta, B, nullptr, img, defl, (cudaStream_t)stream);
}

gl_status gl_logp_grad(gl_system* sys, const float* theta, int B, float* logp, float* grad,
                       gl_deflection defl, void* stream) {
  gl::Range nvtx_range("gl_logp_grad");
  gl_status r = check_call(sys, theta, B, logp, defl);
  if (r != GL_OK) return r;
  if (B > 0 && !grad) return fail(GL_EINVAL, "grad is NULL");
  if (B == 0) return GL_OK;
  if ((r = set_device(sys)) != GL_OK) return r;
  const cudaStream_t st = (cudaStream_t)stream;
  SysParams sp = sys->sp;
  sp.bufA_smem = sys->grad_A;
  sp.bufB_smem = sys->grad_B;
  sp.slot_floats = sys->grad_slot;
  if (sys->grad_slot) {
    r = ensure_scratch(sys, (size_t)B * sys->grad_slot);
    if (r != GL_OK) return r;
    sp.scratch = sys->scratch;
  }
  if (defl == GL_DEFL_SURROGATE_FUSED && !sys->no_fused) {
    // the surrogate evaluated inside each row's CTA (no table launch, no
    // tables in global memory), where two CTAs of it still fit per SM
    if ((r = gl::surrogate_take_timeout(sys->sur)) != GL_OK) return r;
    SysParams spf = sp;
    gl::surrogate_net(sys->sur, &spf);
    spf.table = nullptr;
    gl::table_domain(defl, sys->sur, &spf.sq_lo, &spf.sq_hi, &spf.sg_lo, &spf.sg_hi);
    const size_t dyn = std::max(sys->grad_smem, gl::net_smem_bytes());
    GL_CUDA(gl::surrogate_flag_begin(sys->sur, st), "timeout flag reset");
    bool fits = false;
    GL_CUDA(gl::launch_grad_fused(spf, theta, B, logp, grad, dyn, &fits, st), "fused launch");
    if (fits) {
      GL_CUDA(gl::surrogate_flag_end(sys->sur, st), "timeout flag copy");
      return GL_OK;
    }
    sys->no_fused = true;
  }
  if (defl != GL_DEFL_SERIES) {
    r = prepare_surrogate(sys, theta, B, sp, defl, st);
    if (r != GL_OK) return r;
  }
  GL_CUDA(gl::launch_grad(sp, theta, B, logp, grad, sys->grad_smem, st), "gradient launch");
  return GL_OK;
}

gl_status gl_leapfrog(gl_system* sys, float* theta, float* p, float* logp, float* grad,
                      const float* inv_mass, float eps, int n_steps, int B, void* stream) {
  gl::Range nvtx_range("gl_leapfrog");
  if (!sys) return fail(GL_EINVAL, "system is NULL");
  if (B < 0 || n_steps < 0) return fail(GL_EINVAL, "B and n_steps must be >= 0");
  if (!std::isfinite(eps)) return fail(GL_EINVAL, "eps must be finite");
  if (B == 0 || n_steps == 0) return GL_OK;
  if (!theta || !p || !logp || !grad || !inv_mass)
    return fail(GL_EINVAL, "NULL theta, p, logp, grad or inv_mass");
  gl_status r = set_device(sys);
  if (r != GL_OK) return r;
  SysParams sp = sys->sp;
  sp.bufA_smem = sys->grad_A;
  sp.bufB_smem = sys->grad_B;
  sp.slot_floats = sys->grad_slot;
  if (sys->grad_slot) {
    r = ensure_scratch(sys, (size_t)B * sys->grad_slot);
    if (r != GL_OK) return r;
    sp.scratch = sys->scratch;
  }
  gl_system::LfKey key;
  std::memset(&key, 0, sizeof key);  // padding takes part in the comparison
  key.theta = theta;
  key.p = p;
  key.logp = logp;
  key.grad = grad;
  key.scratch = sp.scratch;
  key.inv_mass = inv_mass;
  key.eps = eps;
  key.n_steps = n_steps;
  key.B = B;
  const bool same = sys->lf_exec && std::memcmp(&key, &sys->lf_key, sizeof key) == 0;
  if (!same) {
    if (sys->lf_exec) {
      GL_CUDA(cudaGraphExecDestroy(sys->lf_exec), "graph destroy");
      sys->lf_exec = nullptr;
    }
    if (!sys->cap_stream)
      GL_CUDA(cudaStreamCreateWithFlags(&sys->cap_stream, cudaStreamNonBlocking), "stream");
    GL_CUDA(cudaStreamBeginCapture(sys->cap_stream, cudaStreamCaptureModeThreadLocal),
            "begin capture");
    cudaError_t e = gl::launch_leapfrog_block(sp, sys->grad_smem, theta, p, logp, grad, inv_mass,
                                              eps, n_steps, B, sys->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(sys->cap_stream, &g);
    if (e != cudaSuccess) return cuda_fail(e, "leapfrog capture");
    if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
    e = cudaGraphInstantiate(&sys->lf_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      sys->lf_exec = nullptr;
      return cuda_fail(e, "graph instantiate");
    }
    std::memcpy(&sys->lf_key, &key, sizeof key);
  }
  GL_CUDA(cudaGraphLaunch(sys->lf_exec, (cudaStream_t)stream), "graph launch");
  return GL_OK;
}

gl_status gl_logp_grad_host(gl_system* sys, const float* theta_host, int B, float* logp_host,
                            float* grad_host, gl_deflection defl, void* stream) {
  gl::Range nvtx_range("gl_logp_grad_host");
  gl_status r = check_call(sys, theta_host, B, logp_host, defl);
  if (r != GL_OK) return r;
  if (B == 0) return GL_OK;
  if ((r = set_device(sys)) != GL_OK) return r;
  const int P = sys->sp.P;
  const size_t need = (size_t)B * (2 * P + 1);
  if (need > sys->stage_floats) {
    cudaFree(sys->d_stage);
    cudaFreeHost(sys->h_stage);
    sys->d_stage = nullptr;
    sys->h_stage = nullptr;
    sys->stage_floats = 0;
    GL_CUDA(cudaMalloc(&sys->d_stage, need * 4), "staging allocation");
    GL_CUDA(cudaMallocHost(&sys->h_stage, need * 4), "pinned staging allocation");
    sys->stage_floats = need;
  }
  cudaStream_t st = (cudaStream_t)stream;
  float* d_theta = sys->d_stage;
  float* d_grad = d_theta + (size_t)B * P;
  float* d_logp = d_grad + (size_t)B * P;
  // page-locked caller buffers are copied directly, others through the staging
  const bool direct = page_locked(theta_host, (size_t)B * P * 4) &&
                      page_locked(logp_host, (size_t)B * 4) &&
                      (!grad_host || page_locked(grad_host, (size_t)B * P * 4));
  float* h_theta = direct ? const_cast<float*>(theta_host) : sys->h_stage;
  float* h_grad = direct ? grad_host : h_theta + (size_t)B * P;
  float* h_logp = direct ? logp_host : h_grad + (size_t)B * P;
  if (!direct) std::memcpy(h_theta, theta_host, (size_t)B * P * 4);
  GL_CUDA(cudaMemcpyAsync(d_theta, h_theta, (size_t)B * P * 4, cudaMemcpyHostToDevice, st), "H2D");
  if (grad_host)
    r = gl_logp_grad(sys, d_theta, B, d_logp, d_grad, defl, stream);
  else
    r = gl_logp(sys, d_theta, B, d_logp, defl, stream);
  if (r != GL_OK) return r;
  GL_CUDA(cudaMemcpyAsync(h_logp, d_logp, (size_t)B * 4, cudaMemcpyDeviceToHost, st), "D2H");
  if (grad_host)
    GL_CUDA(cudaMemcpyAsync(h_grad, d_grad, (size_t)B * P * 4, cudaMemcpyDeviceToHost, st), "D2H");
  GL_CUDA(cudaStreamSynchronize(st), "stream synchronize");
  if (!direct) {
    std::memcpy(logp_host, h_logp, (size_t)B * 4);
    if (grad_host) std::memcpy(grad_host, h_grad, (size_t)B * P * 4);
  }
  return GL_OK;
}

}  // extern "C"

namespace gl {
// Sets the message gl_last_error() returns on this host thread.
void set_last_error(const std::string& msg) { g_last_error = msg; }

// Evaluations of B rows for the inference drivers (gl_infer.cu): eval_prepare
// makes the device ready (current device, global scratch, the table buffer
// for a surrogate or table deflection) and fills the kernel parameters of the
// gradient kernel (with_grad) or the log-p-only kernel, allocating nothing
// after it returns; eval_launch then launches one evaluation (the row tables
// first, when there are any) and can be captured into a CUDA graph. The
// parameters stay valid until the system's next call.
gl_status eval_prepare(gl_system* s, int B, gl_deflection defl, bool with_grad, SysParams* sp,
                       size_t* dyn) {
  gl_status r = check_call(s, s, B, s, defl);
  if (r != GL_OK) return r;
  if ((r = set_device(s)) != GL_OK) return r;
  *sp = s->sp;
  sp->bufA_smem = with_grad ? s->grad_A : s->fwd_A;
  sp->bufB_smem = with_grad ? s->grad_B : 0;
  sp->slot_floats = with_grad ? s->grad_slot : s->fwd_slot;
  sp->table = nullptr;
  if (sp->slot_floats) {
    r = ensure_scratch(s, (size_t)B * sp->slot_floats);
    if (r != GL_OK) return r;
    sp->scratch = s->scratch;
  }
  if (gl::defl_network(defl) && (r = gl::surrogate_take_timeout(s->sur)) != GL_OK) return r;
  if (defl != GL_DEFL_SERIES) {
    if ((size_t)B > s->table_rows) {
      cudaFree(s->d_table);
      s->d_table = nullptr;
      s->table_rows = 0;
      GL_CUDA(cudaMalloc(&s->d_table, (size_t)B * gl::TABLE_ROW * sizeof(float4)),
              "surrogate table allocation");
      s->table_rows = B;
    }
    sp->table = s->d_table;
    gl::table_domain(defl, s->sur, &sp->sq_lo, &sp->sq_hi, &sp->sg_lo, &sp->sg_hi);
  }
  *dyn = with_grad ? s->grad_smem : s->fwd_smem;
  return GL_OK;
}

cudaError_t eval_launch(const gl_system* s, const SysParams& sp, size_t dyn, const float* theta,
                        int B, float* logp, float* grad, gl_deflection defl, cudaStream_t st) {
  if (sp.table) {
    cudaError_t e =
        gl::launch_table(defl, s->sur, theta, sp.P, B, const_cast<float4*>(sp.table), st);
    if (e != cudaSuccess) return e;
  }
  if (grad) return gl::launch_grad(sp, theta, B, logp, grad, dyn, st);
  return gl::launch_forward(sp, theta, B, logp, nullptr, dyn, st);
}

// Read-only view of a system's gradient-kernel plan for other translation
// units of the library: kernel parameters with buffer placement, dynamic
// shared memory and global scratch floats per row. Returns the device index.
int system_grad_plan(const gl_system* sys, SysParams* sp, size_t* dyn_smem, size_t* slot_floats) {
  *sp = sys->sp;
  sp->bufA_smem = sys->grad_A;
  sp->bufB_smem = sys->grad_B;
  sp->slot_floats = sys->grad_slot;
  sp->scratch = nullptr;
  *dyn_smem = sys->grad_smem;
  *slot_floats = sys->grad_slot;
  return sys->device;
}
}  // namespace gl
