// Inference layer around the fused log-posterior (Sec. 3): the bijection to
// an unconstrained space with log|J|, log p~(u) and its gradient, multi-start
// MAP with Adam, HMC transitions with Metropolis-Hastings acceptance and
// step-size / mass adaptation, and SVI with the score-function ELBO gradient
// and AdaBelief. Row-wise work runs one warp per row (lanes over the
// parameters); every loop of steps or transitions is one CUDA graph per step
// with its control state in device memory, so nothing waits on the host.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "../../include/gl.h"
#include "gl_internal.cuh"
#include "gl_system.h"

namespace gl {
gl_status eval_prepare(gl_system* s, int B, gl_deflection defl, bool with_grad, SysParams* sp,
                       size_t* dyn);
cudaError_t eval_launch(const gl_system* s, const SysParams& sp, size_t dyn, const float* theta,
                        int B, float* logp, float* grad, gl_deflection defl, cudaStream_t st);
}  // namespace gl

namespace {

using gl::SysParams;

gl_status fail(gl_status s, const std::string& msg) {
  gl::set_last_error(msg);
  return s;
}

gl_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? GL_ENOMEM : GL_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define GI_CUDA(call, what)                              \
  do {                                                   \
    cudaError_t _e = (call);                             \
    if (_e != cudaSuccess) return cuda_fail(_e, what);   \
  } while (0)

constexpr int RPB = 8;  // rows per 256-thread block (one warp each)
constexpr double LOG_2PI = 1.8378770664093454836;

// ----------------------------------------------------------- bijection ----
enum { BJ_ID = 0, BJ_INTERVAL, BJ_EXP, BJ_LOWER, BJ_UPPER, BJ_DISC, BJ_DISC2 };

struct BijDev {
  int mode;
  float lo, hi, rmax;  // interval bounds; disc radius (on the e1 entry)
};

// One map per prior support; a disc map on an ellipticity pair whose priors
// are both unbounded while |e| < emax restricts it (one thread).
__global__ void k_bij_setup(const gl::PriorDev* pr, const float* emax, int P, int nc,
                            BijDev* bj) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int k = 0; k < P; ++k) {
    const int kind = pr[k].kind;
    const float lo = pr[k].lo, hi = pr[k].hi;
    // normal: unbounded; log-normal: (0, inf); uniform, truncated normal and
    // flat: by which of their bounds are finite
    const bool bounded = kind == 0 || kind == 1 || kind == 3;
    int m = BJ_ID;
    if (kind == 4)
      m = BJ_EXP;
    else if (bounded && isfinite(lo) && isfinite(hi))
      m = BJ_INTERVAL;
    else if (bounded && isfinite(lo))
      m = BJ_LOWER;
    else if (bounded && isfinite(hi))
      m = BJ_UPPER;
    bj[k] = BijDev{m, lo, hi, 0.f};
  }
  for (int c = 0; c < nc; ++c) {
    const int i = c == 0 ? 2 : 8 + 7 * (c - 1) + 2;
    const float em = emax ? emax[c] : 0.f;
    if (em > 0.f && bj[i].mode == BJ_ID && bj[i + 1].mode == BJ_ID) {
      bj[i].mode = BJ_DISC;
      bj[i].rmax = em;
      bj[i + 1].mode = BJ_DISC2;
    }
  }
}

struct Scal {
  double th, dth, logj, dlogj;  // theta, d theta/du, log|d theta/du|, its derivative
};

__device__ Scal bij_scalar(const BijDev& d, double x) {
  switch (d.mode) {
    case BJ_INTERVAL: {
      const double w = (double)d.hi - (double)d.lo;
      const double ax = fabs(x), e = exp(-ax), q = 1.0 / (1.0 + e);
      const double s = x >= 0.0 ? q : e * q;  // sigmoid(x)
      double th = (double)d.lo + w * s;
      th = fmin(fmax(th, (double)d.lo), (double)d.hi);
      return Scal{th, w * e * q * q, log(w) - ax - 2.0 * log1p(e), 1.0 - 2.0 * s};
    }
    case BJ_EXP: {
      const double ex = exp(x);
      return Scal{ex, ex, x, 1.0};
    }
    case BJ_LOWER: {
      const double ex = exp(x);
      return Scal{(double)d.lo + ex, ex, x, 1.0};
    }
    case BJ_UPPER: {
      const double ex = exp(x);
      return Scal{(double)d.hi - ex, -ex, x, 1.0};
    }
    default:
      return Scal{x, 1.0, 0.0, 0.0};
  }
}

__device__ double bij_scalar_inverse(const BijDev& d, double th) {
  switch (d.mode) {
    case BJ_INTERVAL: {
      const double s = (th - (double)d.lo) / ((double)d.hi - (double)d.lo);
      return log(s) - log1p(-s);
    }
    case BJ_EXP: return log(th);
    case BJ_LOWER: return log(th - (double)d.lo);
    case BJ_UPPER: return log((double)d.hi - th);
    default: return th;
  }
}

// The radial disc map e = v R tanh(rho)/rho, rho = |v|: e, the symmetric
// Jacobian (j11, j12, j22), log|J| = 2 log R - 2 log cosh rho + log(tanh rho/rho)
// and its gradient (g1, g2). Series below rho = 1e-3.
struct Disc {
  double e1, e2, j11, j12, j22, logj, g1, g2;
};

__device__ Disc bij_disc(double R, double v1, double v2) {
  const double rho = hypot(v1, v2);
  double tor, gpo, ko;  // tanh(rho)/rho, (d/drho of it)/rho, (d log|J|/drho)/rho
  if (rho < 1e-3) {
    const double r2 = rho * rho;
    tor = 1.0 - r2 / 3.0;
    gpo = -2.0 / 3.0 + 8.0 * r2 / 15.0;
    ko = -8.0 / 3.0 + 44.0 * r2 / 45.0;
  } else {
    const double t = tanh(rho), c = cosh(rho);
    tor = t / rho;
    gpo = (rho / (c * c) - t) / (rho * rho * rho);
    ko = (-2.0 * t + 2.0 / sinh(2.0 * rho) - 1.0 / rho) / rho;
  }
  Disc d;
  const double g = R * tor;
  d.e1 = g * v1;
  d.e2 = g * v2;
  d.j11 = g + R * gpo * v1 * v1;
  d.j12 = R * gpo * v1 * v2;
  d.j22 = g + R * gpo * v2 * v2;
  d.logj = 2.0 * log(R) - 2.0 * log(cosh(rho)) + log(tor);
  d.g1 = ko * v1;
  d.g2 = ko * v2;
  return d;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// theta(u) of one row (all lanes of the warp); returns log|J| on every lane.
__device__ double row_to_theta(const BijDev* __restrict__ bj, int P, const float* __restrict__ u,
                               float* __restrict__ th) {
  const int lane = threadIdx.x & 31;
  double lj = 0.0;
  for (int k = lane; k < P; k += 32) {
    const BijDev d = bj[k];
    if (d.mode == BJ_DISC2) continue;
    if (d.mode == BJ_DISC) {
      const Disc q = bij_disc((double)d.rmax, (double)u[k], (double)u[k + 1]);
      th[k] = (float)q.e1;
      th[k + 1] = (float)q.e2;
      lj += q.logj;
    } else {
      const Scal q = bij_scalar(d, (double)u[k]);
      th[k] = (float)q.th;
      lj += q.logj;
    }
  }
  return warp_sum(lj);
}

// log|J| and the pulled-back gradient gu = J^T g + grad log|J| of one row;
// gu may alias shared memory. Returns log|J| on every lane.
__device__ double row_pullback(const BijDev* __restrict__ bj, int P, const float* __restrict__ u,
                               const float* __restrict__ g, float* gu) {
  const int lane = threadIdx.x & 31;
  double lj = 0.0;
  for (int k = lane; k < P; k += 32) {
    const BijDev d = bj[k];
    if (d.mode == BJ_DISC2) continue;
    if (d.mode == BJ_DISC) {
      const Disc q = bij_disc((double)d.rmax, (double)u[k], (double)u[k + 1]);
      const double g1 = g[k], g2 = g[k + 1];
      gu[k] = (float)(q.j11 * g1 + q.j12 * g2 + q.g1);
      gu[k + 1] = (float)(q.j12 * g1 + q.j22 * g2 + q.g2);
      lj += q.logj;
    } else {
      const Scal q = bij_scalar(d, (double)u[k]);
      gu[k] = (float)(q.dth * (double)g[k] + q.dlogj);
      lj += q.logj;
    }
  }
  return warp_sum(lj);
}

// theta(u) of one row like row_to_theta, and the Jacobian terms a later
// pull-back at the same u needs, in jc[3 k .. 3 k + 2] (FP64, as computed):
// a scalar map keeps (d theta/du, d log|J|/du); a disc pair keeps (j11, j12,
// g1) in its first slot and (j22, g2) in its second. Returns log|J|.
__device__ double row_to_theta_cache(const BijDev* __restrict__ bj, int P,
                                     const float* __restrict__ u, float* __restrict__ th,
                                     double* __restrict__ jc) {
  const int lane = threadIdx.x & 31;
  double lj = 0.0;
  for (int k = lane; k < P; k += 32) {
    const BijDev d = bj[k];
    if (d.mode == BJ_DISC2) continue;
    if (d.mode == BJ_DISC) {
      const Disc q = bij_disc((double)d.rmax, (double)u[k], (double)u[k + 1]);
      th[k] = (float)q.e1;
      th[k + 1] = (float)q.e2;
      jc[3 * k] = q.j11;
      jc[3 * k + 1] = q.j12;
      jc[3 * k + 2] = q.g1;
      jc[3 * k + 3] = q.j22;
      jc[3 * k + 4] = q.g2;
      lj += q.logj;
    } else {
      const Scal q = bij_scalar(d, (double)u[k]);
      th[k] = (float)q.th;
      jc[3 * k] = q.dth;
      jc[3 * k + 1] = q.dlogj;
      lj += q.logj;
    }
  }
  return warp_sum(lj);
}

// The pull-back gu = J^T g + grad log|J| of one row from the terms that
// row_to_theta_cache stored at the same u (the same arithmetic as
// row_pullback without evaluating the maps again).
__device__ void row_pullback_cached(const BijDev* __restrict__ bj, int P,
                                    const double* __restrict__ jc, const float* __restrict__ g,
                                    float* gu) {
  const int lane = threadIdx.x & 31;
  for (int k = lane; k < P; k += 32) {
    const BijDev d = bj[k];
    if (d.mode == BJ_DISC2) continue;
    if (d.mode == BJ_DISC) {
      const double g1 = g[k], g2 = g[k + 1];
      gu[k] = (float)(jc[3 * k] * g1 + jc[3 * k + 1] * g2 + jc[3 * k + 2]);
      gu[k + 1] = (float)(jc[3 * k + 1] * g1 + jc[3 * k + 3] * g2 + jc[3 * k + 4]);
    } else {
      gu[k] = (float)(jc[3 * k] * (double)g[k] + jc[3 * k + 1]);
    }
  }
}

__global__ void k_to_theta(const BijDev* __restrict__ bj, int P, const float* __restrict__ u,
                           int B, float* __restrict__ th, float* __restrict__ logj) {
  const int row = blockIdx.x * RPB + (threadIdx.x >> 5);
  if (row >= B) return;
  const double lj = row_to_theta(bj, P, u + (size_t)row * P, th + (size_t)row * P);
  if (logj && (threadIdx.x & 31) == 0) logj[row] = (float)lj;
}

// theta(u) with the Jacobian terms for a later pull-back at the same u
// (jc [B][3 P], ljc [B]; row_to_theta_cache).
__global__ void k_to_theta_cache(const BijDev* __restrict__ bj, int P, const float* __restrict__ u,
                                 int B, float* __restrict__ th, double* __restrict__ jc,
                                 double* __restrict__ ljc) {
  const int row = blockIdx.x * RPB + (threadIdx.x >> 5);
  if (row >= B) return;
  const size_t o = (size_t)row * P;
  const double lj = row_to_theta_cache(bj, P, u + o, th + o, jc + 3 * o);
  if ((threadIdx.x & 31) == 0) ljc[row] = lj;
}

__global__ void k_to_u(const BijDev* __restrict__ bj, int P, const float* __restrict__ th, int B,
                       float* __restrict__ u) {
  const int row = blockIdx.x * RPB + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= B) return;
  const float* t = th + (size_t)row * P;
  float* o = u + (size_t)row * P;
  for (int k = lane; k < P; k += 32) {
    const BijDev d = bj[k];
    if (d.mode == BJ_DISC2) continue;
    if (d.mode == BJ_DISC) {
      const double e1 = t[k], e2 = t[k + 1], R = d.rmax;
      const double r = hypot(e1, e2);
      const double f = r > 0.0 ? atanh(r / R) / r : 1.0 / R;
      o[k] = (float)(f * e1);
      o[k + 1] = (float)(f * e2);
    } else {
      o[k] = (float)bij_scalar_inverse(d, (double)t[k]);
    }
  }
}

// log p~ = log p + log|J| and its gradient; a row with a non-finite log p
// keeps it, with the theta-space gradient (0 or NaN) passed through.
__global__ void k_pullback(const BijDev* __restrict__ bj, int P, const float* __restrict__ u,
                           int B, const float* __restrict__ lp_th, const float* __restrict__ g_th,
                           float* __restrict__ lp_u, float* __restrict__ g_u) {
  const int row = blockIdx.x * RPB + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= B) return;
  const float lp = lp_th[row];
  const size_t o = (size_t)row * P;
  if (!isfinite(lp)) {
    for (int k = lane; k < P; k += 32) g_u[o + k] = g_th[o + k];
    if (lane == 0) lp_u[row] = lp;
    return;
  }
  const double lj = row_pullback(bj, P, u + o, g_th + o, g_u + o);
  if (lane == 0) lp_u[row] = (float)((double)lp + lj);
}

// ----------------------------------------------------- random numbers ----
// SplitMix64 output for state seed + ctr * gamma (Steele, Lea & Flood 2014).
__device__ __forceinline__ uint64_t splitmix(uint64_t seed, uint64_t ctr) {
  uint64_t z = seed + (ctr + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Uniform in (0, 1) on the grid (k + 1/2) 2^-24 (exact in FP32).
__device__ __forceinline__ float uniform24(uint64_t seed, uint64_t ctr) {
  return ((float)(splitmix(seed, ctr) >> 40) + 0.5f) * (1.f / 16777216.f);
}

// Box-Muller on uniforms ctr (radius) and ctr + 1 (angle).
__device__ __forceinline__ float normal_bm(uint64_t seed, uint64_t ctr) {
  const float u1 = uniform24(seed, ctr), u2 = uniform24(seed, ctr + 1);
  return sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

// ------------------------------------------------------------------ MAP ----
struct MapCtl {
  int t0;
  float lr, b1, b2, eps;
};

// Pull-back of the step's gradient, one Adam update (ascending log p~) and
// theta of the new point for the next evaluation; logp receives log p~ at
// the point evaluated. A row with a non-finite log p does not move.
__global__ void k_map_update(const BijDev* __restrict__ bj, int P, int B, float* __restrict__ u,
                             float* __restrict__ m, float* __restrict__ v,
                             const float* __restrict__ lp_th, const float* __restrict__ g_th,
                             float* __restrict__ logp, const MapCtl* __restrict__ ctl, int step,
                             float* __restrict__ th_next, double* __restrict__ jc,
                             double* __restrict__ ljc) {
  __shared__ float gsh[RPB][gl::MAX_P];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * RPB + w;
  if (row >= B) return;
  const size_t o = (size_t)row * P;
  const float lp = lp_th[row];
  if (isfinite(lp)) {
    // theta was evaluated at the current u, where its Jacobian terms were cached
    row_pullback_cached(bj, P, jc + 3 * o, g_th + o, gsh[w]);
    const double lj = ljc[row];
    __syncwarp();
    if (lane == 0) logp[row] = (float)((double)lp + lj);
    const MapCtl c = *ctl;
    const double t = (double)(c.t0 + step + 1);
    const float bc1 = (float)(1.0 - pow((double)c.b1, t)), bc2 = (float)(1.0 - pow((double)c.b2, t));
    for (int k = lane; k < P; k += 32) {
      const float gd = -gsh[w][k];
      const float mk = c.b1 * m[o + k] + (1.f - c.b1) * gd;
      const float vk = c.b2 * v[o + k] + (1.f - c.b2) * gd * gd;
      m[o + k] = mk;
      v[o + k] = vk;
      u[o + k] -= c.lr * (mk / bc1) / (sqrtf(vk / bc2) + c.eps);
    }
    __syncwarp();
  } else if (lane == 0) {
    logp[row] = lp;
  }
  const double ljn = row_to_theta_cache(bj, P, u + o, th_next + o, jc + 3 * o);
  if (lane == 0) ljc[row] = ljn;
}

// ------------------------------------------------------------------ HMC ----
struct HmcDev {
  float eps;
  int flags;
  unsigned long long step;  // transitions so far (the generator's counter)
  int local;                // transitions in the current run (draw index)
  float* draws;
  float* accept;
  // dual averaging (Hoffman & Gelman 2014, Sec. 3.2)
  double mu, hbar, log_eps, log_eps_bar, target;
  int m;
  // moments of u for the mass adaptation (Sec. 3.3)
  double count;
  double sum[gl::MAX_P], sum2[gl::MAX_P];
};

struct HmcBufs {
  float *u, *lp, *g;      // current state in u-space
  float *u0, *lp0, *g0;   // state at the trajectory's start
  float *p, *H0, *prob;
  float *th, *lp_th, *g_th;
  float* inv_mass;
  double* jc;   // [B][3 P] Jacobian terms of theta(u) at the current u (row_to_theta_cache)
  double* ljc;  // [B] log|J| at the current u
};

// Momenta, the trajectory's start, H0, then the first half kick and drift and
// theta for the first evaluation. A chain with a non-finite log p stays put.
__global__ void k_hmc_begin(const BijDev* __restrict__ bj, int P, int B,
                            const HmcDev* __restrict__ ctl, uint64_t seed, HmcBufs b) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * RPB + w;
  if (row >= B) return;
  const size_t o = (size_t)row * P;
  const float eps = ctl->eps;
  const uint64_t base = (ctl->step * (uint64_t)B + (uint64_t)row) * (uint64_t)(2 * P + 2);
  const float lp = b.lp[row];
  const bool live = isfinite(lp);
  double kin = 0.0;
  for (int k = lane; k < P; k += 32) {
    const float im = b.inv_mass[k];
    float pk = normal_bm(seed, base + 2 * k) * rsqrtf(im);
    kin += (double)im * (double)pk * (double)pk;
    const float uk = b.u[o + k], gk = b.g[o + k];
    b.u0[o + k] = uk;
    b.g0[o + k] = gk;
    float un = uk;
    if (live) {
      pk = fmaf(0.5f * eps, gk, pk);
      un = fmaf(eps * im, pk, uk);
    }
    b.p[o + k] = pk;
    b.u[o + k] = un;
  }
  kin = warp_sum(kin);
  __syncwarp();
  if (lane == 0) {
    b.lp0[row] = lp;
    b.H0[row] = (float)(-(double)lp + 0.5 * kin);
  }
  const double lj = row_to_theta_cache(bj, P, b.u + o, b.th + o, b.jc + 3 * o);
  if (lane == 0) b.ljc[row] = lj;
}

// After an evaluation: pull-back, then a full kick and drift (a half kick on
// the last step). A chain whose log p turned non-finite stops moving.
__global__ void k_hmc_mid(const BijDev* __restrict__ bj, int P, int B,
                          const HmcDev* __restrict__ ctl, HmcBufs b, int last) {
  __shared__ float gsh[RPB][gl::MAX_P];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * RPB + w;
  if (row >= B) return;
  const size_t o = (size_t)row * P;
  const float eps = ctl->eps;
  const float lpt = b.lp_th[row];
  bool live = isfinite(lpt);
  double lj = 0.0;
  if (live) {
    // theta was evaluated at the current u, where the terms were cached
    row_pullback_cached(bj, P, b.jc + 3 * o, b.g_th + o, gsh[w]);
    lj = b.ljc[row];
    __syncwarp();
  }
  for (int k = lane; k < P; k += 32) {
    const float gk = live ? gsh[w][k] : b.g_th[o + k];
    b.g[o + k] = gk;
    if (live) {
      float pk = b.p[o + k];
      pk = fmaf(last ? 0.5f * eps : eps, gk, pk);
      b.p[o + k] = pk;
      if (!last) b.u[o + k] = fmaf(eps * b.inv_mass[k], pk, b.u[o + k]);
    }
  }
  if (lane == 0) b.lp[row] = live ? (float)((double)lpt + lj) : lpt;
  __syncwarp();
  if (!last && live) {
    const double ljn = row_to_theta_cache(bj, P, b.u + o, b.th + o, b.jc + 3 * o);
    if (lane == 0) b.ljc[row] = ljn;
  }
}

// Metropolis-Hastings: accept when log a < min(0, H0 - H1); a rejected chain
// returns to the trajectory's start. Records theta(u) when asked.
__global__ void k_hmc_end(const BijDev* __restrict__ bj, int P, int B,
                          const HmcDev* __restrict__ ctl, uint64_t seed, HmcBufs b) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * RPB + w;
  if (row >= B) return;
  const size_t o = (size_t)row * P;
  double kin = 0.0;
  for (int k = lane; k < P; k += 32) {
    const double pk = b.p[o + k];
    kin += (double)b.inv_mass[k] * pk * pk;
  }
  kin = warp_sum(kin);
  const double H1 = -(double)b.lp[row] + 0.5 * kin;
  const double dH = (double)b.H0[row] - H1;
  const double log_acc = isfinite(dH) ? fmin(0.0, dH) : -INFINITY;
  const uint64_t base = (ctl->step * (uint64_t)B + (uint64_t)row) * (uint64_t)(2 * P + 2);
  const float a = uniform24(seed, base + 2 * P);
  const bool acc = log((double)a) < log_acc;
  if (!acc) {
    for (int k = lane; k < P; k += 32) {
      b.u[o + k] = b.u0[o + k];
      b.g[o + k] = b.g0[o + k];
    }
    if (lane == 0) b.lp[row] = b.lp0[row];
  }
  if (lane == 0) b.prob[row] = (float)exp(log_acc);
  __syncwarp();
  float* dr = ctl->draws;
  if (dr) row_to_theta(bj, P, b.u + o, dr + ((size_t)ctl->local * B + row) * P);
}

// One block: mean acceptance probability, dual-averaging update, moments of
// u, and the counters.
__global__ void k_hmc_adapt(HmcDev* __restrict__ ctl, const float* __restrict__ prob,
                            const float* __restrict__ u, int B, int P) {
  __shared__ double red[8];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  double s = 0.0;
  for (int r = t; r < B; r += blockDim.x) s += (double)prob[r];
  s = warp_sum(s);
  if (lane == 0) red[w] = s;
  __syncthreads();
  const int flags = ctl->flags;
  if (t == 0) {
    double tot = 0.0;
    for (int k = 0; k < 8; ++k) tot += red[k];
    const double mean = tot / B;
    if (ctl->accept) ctl->accept[ctl->local] = (float)mean;
    if (flags & GL_HMC_ADAPT_STEP) {
      ctl->m += 1;
      const double mm = ctl->m, wgt = 1.0 / (mm + 10.0);
      ctl->hbar = (1.0 - wgt) * ctl->hbar + wgt * (ctl->target - mean);
      ctl->log_eps = ctl->mu - sqrt(mm) / 0.05 * ctl->hbar;
      const double eta = pow(mm, -0.75);
      ctl->log_eps_bar = eta * ctl->log_eps + (1.0 - eta) * ctl->log_eps_bar;
      ctl->eps = (float)exp(ctl->log_eps);
    }
  }
  if (flags & GL_HMC_COLLECT_MOMENTS) {
    for (int k = 0; k < P; ++k) {
      double a = 0.0, a2 = 0.0;
      for (int r = t; r < B; r += blockDim.x) {
        const double x = u[(size_t)r * P + k];
        a += x;
        a2 += x * x;
      }
      a = warp_sum(a);
      a2 = warp_sum(a2);
      __syncthreads();
      if (lane == 0) red[w] = a;
      __syncthreads();
      if (t == 0) {
        double tot = 0.0;
        for (int q = 0; q < 8; ++q) tot += red[q];
        ctl->sum[k] += tot;
      }
      __syncthreads();
      if (lane == 0) red[w] = a2;
      __syncthreads();
      if (t == 0) {
        double tot = 0.0;
        for (int q = 0; q < 8; ++q) tot += red[q];
        ctl->sum2[k] += tot;
      }
    }
  }
  __syncthreads();
  if (t == 0) {
    if (flags & GL_HMC_COLLECT_MOMENTS) ctl->count += B;
    ctl->step += 1;
    ctl->local += 1;
  }
}

__global__ void k_hmc_end_adapt(HmcDev* __restrict__ ctl, float* __restrict__ inv_mass, int P,
                                int set_mass) {
  const int k = threadIdx.x;
  if (set_mass && ctl->count > 1.0 && k < P) {
    const double mean = ctl->sum[k] / ctl->count;
    const double var = ctl->sum2[k] / ctl->count - mean * mean;
    inv_mass[k] = (float)fmax(var, 1e-12);
  }
  __syncthreads();
  if (k == 0) {
    if (ctl->m > 0) ctl->eps = (float)exp(ctl->log_eps_bar);
    // a later adaptation phase restarts the dual averaging from this step
    ctl->mu = log(10.0 * (double)ctl->eps);
    ctl->log_eps = log((double)ctl->eps);
    ctl->log_eps_bar = 0.0;
    ctl->hbar = 0.0;
    ctl->m = 0;
    ctl->count = 0.0;
    for (int q = 0; q < gl::MAX_P; ++q) ctl->sum[q] = ctl->sum2[q] = 0.0;
  }
}

__global__ void k_fill(float* a, int n, float v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

// ------------------------------------------------------------------ SVI ----
struct SviCtl {
  unsigned long long step;  // global step index (generator counter; AdaBelief's t = step + 1)
  int local;                // steps in the current call (ELBO index)
  float lr, b1, b2, eps;
  float* elbo;
};

// Sample i: z ~ N(0, I), u = mu + L z, a = L^-T z, log q(u), theta(u), log|J|.
__global__ void k_svi_draw(const BijDev* __restrict__ bj, int P, int n,
                           const SviCtl* __restrict__ ctl, uint64_t seed,
                           const float* __restrict__ phi, float* __restrict__ z,
                           float* __restrict__ a, float* __restrict__ logq,
                           float* __restrict__ u, float* __restrict__ th,
                           float* __restrict__ logj) {
  __shared__ float zs[RPB][gl::MAX_P];
  __shared__ double Ls[gl::MAX_P][gl::MAX_P];   // L (strict lower part used)
  __shared__ double Li[gl::MAX_P][gl::MAX_P];   // L^{-1} (lower triangular)
  __shared__ double dg[gl::MAX_P];               // exp(log L_kk)
  __shared__ double ldsum;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* mu = phi;
  const float* L = phi + P;  // row-major, diagonal stored as log
  // L is the same for every sample: stage it, its diagonal and its inverse
  // once per block (warp 0 solves L x = e_c for column c in lane c by forward
  // substitution), then each warp's sample needs only products with them.
  for (int k = threadIdx.x; k < P * P; k += blockDim.x) Ls[k / P][k % P] = (double)L[k];
  __syncthreads();
  if (w == 0) {
    double ld = 0.0;
    for (int k = lane; k < P; k += 32) {
      dg[k] = exp(Ls[k][k]);
      ld += Ls[k][k];
    }
    ld = warp_sum(ld);
    if (lane == 0) ldsum = ld;
    __syncwarp();
    for (int c = lane; c < P; c += 32) {
      for (int i = 0; i < c; ++i) Li[i][c] = 0.0;
      for (int i = c; i < P; ++i) {
        double s = i == c ? 1.0 : 0.0;
        for (int j = c; j < i; ++j) s -= Ls[i][j] * Li[j][c];
        Li[i][c] = s / dg[i];
      }
    }
  }
  __syncthreads();
  const int i = blockIdx.x * RPB + w;
  if (i >= n) return;
  const size_t o = (size_t)i * P;
  const uint64_t base = (ctl->step * (uint64_t)n + (uint64_t)i) * (uint64_t)(2 * P);
  double zz = 0.0;
  for (int k = lane; k < P; k += 32) {
    const float zk = normal_bm(seed, base + 2 * k);
    zs[w][k] = zk;
    z[o + k] = zk;
    zz += (double)zk * zk;
  }
  __syncwarp();
  zz = warp_sum(zz);
  for (int k = lane; k < P; k += 32) {
    // u = mu + L z, and a = L^{-T} z (the score of log q w.r.t. mu)
    double s = mu[k];
    for (int j = 0; j < k; ++j) s += Ls[k][j] * zs[w][j];
    s += dg[k] * zs[w][k];
    u[o + k] = (float)s;
    double t = 0.0;
    for (int j = k; j < P; ++j) t += Li[j][k] * zs[w][j];
    a[o + k] = (float)t;
  }
  if (lane == 0) logq[i] = (float)(-0.5 * zz - ldsum - 0.5 * P * LOG_2PI);
  __syncwarp();
  const double lj = row_to_theta(bj, P, u + o, th + o);
  if (lane == 0) logj[i] = (float)lj;
}

// Output k of the gradient sums over the samples: k < P gives
// sum_i w_i a_ik (mu); then the lower triangle (j, c), j >= c, row-major,
// sum_i w_i a_ij z_ic (L); the last output is sum_i w_i and the count.
// w_i = log q_i - log p~_i; non-finite samples are left out.
__global__ void k_svi_sums(int P, int n, const float* __restrict__ a, const float* __restrict__ z,
                           const float* __restrict__ logq, const float* __restrict__ lp,
                           const float* __restrict__ logj, double* __restrict__ sums) {
  __shared__ double red[8], redc[8];
  const int out = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int nL = P * (P + 1) / 2;
  int mode, j = 0, c = 0;
  if (out < P) {
    mode = 0;
    j = out;
  } else if (out < P + nL) {
    mode = 1;
    int r = out - P;
    j = 0;
    while (r > j) { r -= j + 1; ++j; }
    c = r;
  } else {
    mode = 2;
  }
  double s = 0.0, cnt = 0.0;
  for (int i = t; i < n; i += blockDim.x) {
    const double wi = (double)logq[i] - ((double)lp[i] + (double)logj[i]);
    if (!isfinite(wi)) continue;
    const size_t o = (size_t)i * P;
    if (mode == 0) s += wi * a[o + j];
    else if (mode == 1) s += wi * a[o + j] * z[o + c];
    else { s += wi; cnt += 1.0; }
  }
  s = warp_sum(s);
  cnt = warp_sum(cnt);
  if (lane == 0) { red[w] = s; redc[w] = cnt; }
  __syncthreads();
  if (t == 0) {
    double a1 = 0.0, a2 = 0.0;
    for (int q = 0; q < 8; ++q) { a1 += red[q]; a2 += redc[q]; }
    sums[out] = a1;
    if (mode == 2) sums[out + 1] = a2;
  }
}

// The same outputs for the reparameterisation (pathwise) gradient: k < P
// gives sum_i g_ik, then the lower triangle (j, c) sum_i g_ij z_ic, then
// sum_i w_i and the count, with g_i = grad_u log p~(u_i) and
// w_i = log q_i - log p~_i; samples with a non-finite w_i are left out.
__global__ void k_svi_sums_rep(int P, int n, const float* __restrict__ g,
                               const float* __restrict__ z, const float* __restrict__ logq,
                               const float* __restrict__ lpu, double* __restrict__ sums) {
  __shared__ double red[8], redc[8];
  const int out = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int nL = P * (P + 1) / 2;
  int mode, j = 0, c = 0;
  if (out < P) {
    mode = 0;
    j = out;
  } else if (out < P + nL) {
    mode = 1;
    int r = out - P;
    j = 0;
    while (r > j) { r -= j + 1; ++j; }
    c = r;
  } else {
    mode = 2;
  }
  double s = 0.0, cnt = 0.0;
  for (int i = t; i < n; i += blockDim.x) {
    const double wi = (double)logq[i] - (double)lpu[i];
    if (!isfinite(wi)) continue;
    const size_t o = (size_t)i * P;
    if (mode == 0) s += (double)g[o + j];
    else if (mode == 1) s += (double)g[o + j] * z[o + c];
    else { s += wi; cnt += 1.0; }
  }
  s = warp_sum(s);
  cnt = warp_sum(cnt);
  if (lane == 0) { red[w] = s; redc[w] = cnt; }
  __syncthreads();
  if (t == 0) {
    double a1 = 0.0, a2 = 0.0;
    for (int q = 0; q < 8; ++q) { a1 += red[q]; a2 += redc[q]; }
    sums[out] = a1;
    if (mode == 2) sums[out + 1] = a2;
  }
}

// One AdaBelief step (Zhuang et al. 2020) on phi = (mu, L with log diagonal),
// minimising the ELBO loss, from the sums; records the ELBO estimate.
// rep = 0: score-function sums (k_svi_sums), gradients
//   mu: S_k/n, L_jc: S_jc/n, log L_jj: L_jj S_jj/n - W/n;
// rep = 1: pathwise sums (k_svi_sums_rep), gradients
//   mu: -S_k/n, L_jc: -S_jc/n, log L_jj: -L_jj S_jj/n - 1.
__global__ void k_svi_update(int P, float* __restrict__ phi, float* __restrict__ opt,
                             const double* __restrict__ sums, SviCtl* __restrict__ ctl, int rep) {
  const int nL = P * (P + 1) / 2;
  const double W = sums[P + nL], cnt = sums[P + nL + 1];
  const int np = P + P * P;
  float* m = opt;
  float* s = opt + np;
  const SviCtl c = *ctl;
  const double t = (double)c.step + 1.0;
  const double bc1 = 1.0 - pow((double)c.b1, t), bc2 = 1.0 - pow((double)c.b2, t);
  for (int idx = threadIdx.x; idx < np; idx += blockDim.x) {
    const double sgn = rep ? -1.0 : 1.0;
    double g;
    if (idx < P) {
      g = sgn * sums[idx] / cnt;
    } else {
      const int q = idx - P, j = q / P, k = q - j * P;
      if (k > j) continue;  // upper triangle: not a parameter
      const int tri = j * (j + 1) / 2 + k;
      g = sgn * sums[P + tri] / cnt;
      if (k == j) g = g * exp((double)phi[idx]) - (rep ? 1.0 : W / cnt);  // d/d log L_jj
    }
    if (!(cnt > 0.0) || !isfinite(g)) continue;
    const double mk = (double)c.b1 * m[idx] + (1.0 - c.b1) * g;
    const double d = g - mk;
    const double sk = (double)c.b2 * s[idx] + (1.0 - c.b2) * d * d + (double)c.eps;
    m[idx] = (float)mk;
    s[idx] = (float)sk;
    phi[idx] = (float)((double)phi[idx] -
                       (double)c.lr * (mk / bc1) / (sqrt(sk / bc2) + (double)c.eps));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (c.elbo) c.elbo[c.local] = (float)(cnt > 0.0 ? W / cnt : NAN);
    ctl->step = c.step + 1;
    ctl->local = c.local + 1;
  }
}

// ------------------------------------------------ backward intensities ----
// Intensity of light component c sits at theta index 8 + 7c + 6.
__device__ __forceinline__ int intensity_index(int c) { return 8 + 7 * c + 6; }

// Component rows: row (b, c) is theta_b with intensity k set to [k == c].
__global__ void k_bwd_rows(const float* __restrict__ th, int B, int P, int K,
                           float* __restrict__ rows) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t n = (size_t)B * K * P;
  if (i >= n) return;
  const int k = (int)(i % P);
  const size_t bc = i / P;
  const int c = (int)(bc % K);
  const size_t b = bc / K;
  float v = th[b * P + k];
  for (int j = 0; j < K; ++j)
    if (k == intensity_index(j)) v = j == c ? 1.f : 0.f;
  rows[i] = v;
}

// One block per row: A = M^T W M and r = M^T W d over the pixels (compensated
// FP32 per thread, FP64 across threads),
// then A I = r by Cholesky on thread 0; theta* = theta with I. A solve that
// fails (a component with no light in the image) sets every intensity to 0.
template <int K>
__global__ void k_bwd_solve(const float* __restrict__ img, const float* __restrict__ data,
                            const float* __restrict__ w, int npix, int B, int P,
                            const float* __restrict__ th, float* __restrict__ th_star,
                            float* __restrict__ inten) {
  constexpr int KM = K;
  constexpr int NS = K * (K + 1) / 2 + K;
  __shared__ double red[8][NS];
  const int b = blockIdx.x, t = threadIdx.x, lane = t & 31, wp = t >> 5;
  constexpr int nA = K * (K + 1) / 2, ns = NS;
  // Per-thread sums of the products in FP32 with Kahan compensation (the FP64
  // pipe of this GPU is too slow for ~5 FP64 products per pixel and row); the
  // cross-thread reduction and the solve are FP64.
  float acc[NS], cmp[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) acc[q] = cmp[q] = 0.f;
  auto kahan = [&](int q, float x) {
    const float y = x - cmp[q];
    const float tt = acc[q] + y;
    cmp[q] = (tt - acc[q]) - y;
    acc[q] = tt;
  };
  const float* M = img + (size_t)b * K * npix;
  for (int p = t; p < npix; p += blockDim.x) {
    const float wp_ = w[p], dp = data[p];
    float m[K], wm[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      m[k] = M[(size_t)k * npix + p];
      wm[k] = wp_ * m[k];
    }
    int q = 0;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int l = 0; l <= k; ++l) kahan(q++, wm[k] * m[l]);
#pragma unroll
    for (int k = 0; k < K; ++k) kahan(nA + k, wm[k] * dp);
  }
#pragma unroll
  for (int q = 0; q < ns; ++q) {
    double v = (double)acc[q] - (double)cmp[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wp][q] = v;
  }
  __syncthreads();
  __shared__ float I_sh[KM];
  if (t == 0) {
    double A[KM][KM], r[KM], L[KM][KM], y[KM], x[KM];
    int q = 0;
    for (int k = 0; k < K; ++k)
      for (int l = 0; l <= k; ++l) {
        double s = 0.0;
        for (int u = 0; u < 8; ++u) s += red[u][q];
        A[k][l] = A[l][k] = s;
        ++q;
      }
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int u = 0; u < 8; ++u) s += red[u][nA + k];
      r[k] = s;
    }
    bool ok = true;
    for (int k = 0; k < K && ok; ++k) {
      double d = A[k][k];
      for (int j = 0; j < k; ++j) d -= L[k][j] * L[k][j];
      if (!(d > 1e-300) || !isfinite(d)) { ok = false; break; }
      L[k][k] = sqrt(d);
      for (int i = k + 1; i < K; ++i) {
        double s = A[i][k];
        for (int j = 0; j < k; ++j) s -= L[i][j] * L[k][j];
        L[i][k] = s / L[k][k];
      }
    }
    if (ok) {
      for (int k = 0; k < K; ++k) {
        double s = r[k];
        for (int j = 0; j < k; ++j) s -= L[k][j] * y[j];
        y[k] = s / L[k][k];
      }
      for (int k = K - 1; k >= 0; --k) {
        double s = y[k];
        for (int j = k + 1; j < K; ++j) s -= L[j][k] * x[j];
        x[k] = s / L[k][k];
        if (!isfinite(x[k])) ok = false;
      }
    }
    for (int k = 0; k < K; ++k) I_sh[k] = ok ? (float)x[k] : 0.f;
  }
  __syncthreads();
  for (int k = t; k < P; k += blockDim.x) {
    float v = th[(size_t)b * P + k];
    for (int j = 0; j < K; ++j)
      if (k == intensity_index(j)) v = I_sh[j];
    th_star[(size_t)b * P + k] = v;
  }
  if (inten && t < K) inten[(size_t)b * K + t] = I_sh[t];
}

__global__ void k_bwd_zero(float* __restrict__ grad, int B, int P, int K) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * K) return;
  const int b = i / K, c = i - b * K;
  grad[(size_t)b * P + intensity_index(c)] = 0.f;
}

// The backward model's prior: intensities flat on R (no density, no support).
__global__ void k_bwd_prior(gl::PriorDev* __restrict__ pr, int K) {
  const int c = threadIdx.x;
  if (c >= K) return;
  gl::PriorDev& d = pr[intensity_index(c)];
  d.kind = 0;
  d.lo = -INFINITY;
  d.hi = INFINITY;
  d.cnst = 0.0;
}

// Control-block setters: launched on the caller's stream ahead of a graph,
// so a run's parameters need no host staging or synchronisation.
__global__ void k_set_map_ctl(MapCtl* c, MapCtl v) { *c = v; }
__global__ void k_set_svi_ctl(SviCtl* c, SviCtl v) { *c = v; }
__global__ void k_set_hmc_run(HmcDev* c, int flags, float* draws, float* accept) {
  c->flags = flags;
  c->local = 0;
  c->draws = draws;
  c->accept = accept;
}

}  // namespace

// ------------------------------------------------------------ host side ----
struct gl_hmc {
  gl_system* sys = nullptr;
  int B = 0, P = 0, L = 0;
  gl_deflection defl = GL_DEFL_SERIES;
  uint64_t seed = 0;
  HmcBufs b{};
  float* pool = nullptr;
  double* jpool = nullptr;  // Jacobian cache: [B][3 P] + [B] doubles
  HmcDev* ctl = nullptr;
  HmcDev* h_ctl = nullptr;  // pinned staging: initial control block, step-size reads
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  void *key_scratch = nullptr, *key_table = nullptr;
  const void* key_sur = nullptr;
};

namespace gl {

// Per-system inference state: the bijection table and the MAP / SVI graphs.
struct InferState {
  BijDev* bij = nullptr;
  cudaStream_t cap = nullptr;
  // MAP
  cudaGraphExec_t map_exec = nullptr;
  struct MapKey {
    float *u, *m, *v, *logp;
    void *scratch, *table;
    const void* sur;
    int B, n, defl;
  } map_key{};
  float* map_buf = nullptr;  // theta, logp, grad [B(2P + 1)]
  size_t map_buf_floats = 0;
  double* map_jc = nullptr;  // Jacobian terms of theta(u) [B][3 P], then log|J| [B]
  MapCtl* map_ctl = nullptr;
  // SVI
  cudaGraphExec_t svi_exec = nullptr;
  struct SviKey {
    float *phi, *opt;
    void *scratch, *table;
    const void* sur;
    int n, defl, est;
    unsigned long long seed;
  } svi_key{};
  float* svi_buf = nullptr;
  size_t svi_buf_floats = 0;
  double* svi_sums = nullptr;
  SviCtl* svi_ctl = nullptr;
  // backward intensities
  gl::PriorDev* bwd_prior = nullptr;
  float* bwd_buf = nullptr;  // component rows, images, theta*
  size_t bwd_buf_floats = 0;
};

void infer_release(gl_system* s) {
  InferState* f = s->inf;
  if (!f) return;
  if (f->map_exec) cudaGraphExecDestroy(f->map_exec);
  if (f->svi_exec) cudaGraphExecDestroy(f->svi_exec);
  if (f->cap) cudaStreamDestroy(f->cap);
  cudaFree(f->bij);
  cudaFree(f->map_buf);
  cudaFree(f->map_jc);
  cudaFree(f->map_ctl);
  cudaFree(f->svi_buf);
  cudaFree(f->svi_sums);
  cudaFree(f->svi_ctl);
  cudaFree(f->bwd_prior);
  cudaFree(f->bwd_buf);
  delete f;
  s->inf = nullptr;
}

}  // namespace gl

namespace {

gl_status infer_state(gl_system* s, gl::InferState** out) {
  if (!s->inf) {
    auto* f = new gl::InferState();
    s->inf = f;
    const int P = s->sp.P, nc = 1 + s->sp.nL + s->sp.nS;
    GI_CUDA(cudaMalloc(&f->bij, P * sizeof(BijDev)), "bijector allocation");
    k_bij_setup<<<1, 32>>>(s->d_prior, s->d_emax, P, nc, f->bij);
    GI_CUDA(cudaGetLastError(), "bijector set-up");
    GI_CUDA(cudaDeviceSynchronize(), "bijector set-up");
  }
  *out = s->inf;
  return GL_OK;
}

unsigned grid_rows(int B) { return (unsigned)((B + RPB - 1) / RPB); }

gl_status set_dev(gl_system* s) {
  int cur = -1;
  GI_CUDA(cudaGetDevice(&cur), "cudaGetDevice");
  if (cur != s->device) GI_CUDA(cudaSetDevice(s->device), "cudaSetDevice");
  return GL_OK;
}

}  // namespace

extern "C" {

gl_status gl_bijector_forward(gl_system* sys, const float* u, int B, float* theta, float* logdetj,
                              void* stream) {
  if (!sys) return fail(GL_EINVAL, "system is NULL");
  if (B < 0) return fail(GL_EINVAL, "B < 0");
  if (B == 0) return GL_OK;
  if (!u || !theta) return fail(GL_EINVAL, "NULL u or theta");
  gl_status r = set_dev(sys);
  if (r != GL_OK) return r;
  gl::InferState* f;
  if ((r = infer_state(sys, &f)) != GL_OK) return r;
  k_to_theta<<<grid_rows(B), 256, 0, (cudaStream_t)stream>>>(f->bij, sys->sp.P, u, B, theta,
                                                              logdetj);
  GI_CUDA(cudaGetLastError(), "bijector launch");
  return GL_OK;
}

gl_status gl_bijector_inverse(gl_system* sys, const float* theta, int B, float* u, void* stream) {
  if (!sys) return fail(GL_EINVAL, "system is NULL");
  if (B < 0) return fail(GL_EINVAL, "B < 0");
  if (B == 0) return GL_OK;
  if (!u || !theta) return fail(GL_EINVAL, "NULL u or theta");
  gl_status r = set_dev(sys);
  if (r != GL_OK) return r;
  gl::InferState* f;
  if ((r = infer_state(sys, &f)) != GL_OK) return r;
  k_to_u<<<grid_rows(B), 256, 0, (cudaStream_t)stream>>>(f->bij, sys->sp.P, theta, B, u);
  GI_CUDA(cudaGetLastError(), "bijector launch");
  return GL_OK;
}

gl_status gl_logp_grad_unconstrained(gl_system* sys, const float* u, int B, float* logp,
                                     float* grad, gl_deflection defl, void* stream) {
  gl::Range nvtx_range("gl_logp_grad_unconstrained");
  if (!sys) return fail(GL_EINVAL, "system is NULL");
  if (B < 0) return fail(GL_EINVAL, "B < 0");
  if (B == 0) return GL_OK;
  if (!u || !logp || !grad) return fail(GL_EINVAL, "NULL u, logp or grad");
  gl_status r = set_dev(sys);
  if (r != GL_OK) return r;
  gl::InferState* f;
  if ((r = infer_state(sys, &f)) != GL_OK) return r;
  SysParams sp;
  size_t dyn;
  if ((r = gl::eval_prepare(sys, B, defl, true, &sp, &dyn)) != GL_OK) return r;
  const int P = sys->sp.P;
  const size_t need = (size_t)B * (2 * P + 1);
  if (need > f->map_buf_floats) {
    if (f->map_exec) {  // the MAP graph points into the old buffer
      cudaGraphExecDestroy(f->map_exec);
      f->map_exec = nullptr;
    }
    cudaFree(f->map_buf);
    cudaFree(f->map_jc);
    f->map_buf = nullptr;
    f->map_jc = nullptr;
    f->map_buf_floats = 0;
    GI_CUDA(cudaMalloc(&f->map_buf, need * sizeof(float)), "buffer allocation");
    GI_CUDA(cudaMalloc(&f->map_jc, (size_t)B * (3 * P + 1) * sizeof(double)), "buffer allocation");
    f->map_buf_floats = need;
  }
  float* th = f->map_buf;
  float* gth = th + (size_t)B * P;
  float* lpth = gth + (size_t)B * P;
  cudaStream_t st = (cudaStream_t)stream;
  k_to_theta<<<grid_rows(B), 256, 0, st>>>(f->bij, P, u, B, th, nullptr);
  GI_CUDA(cudaGetLastError(), "bijector launch");
  GI_CUDA(gl::eval_launch(sys, sp, dyn, th, B, lpth, gth, defl, st), "gradient launch");
  k_pullback<<<grid_rows(B), 256, 0, st>>>(f->bij, P, u, B, lpth, gth, logp, grad);
  GI_CUDA(cudaGetLastError(), "pull-back launch");
  return GL_OK;
}

gl_status gl_map_adam(gl_system* sys, float* u, float* m, float* v, int B, int n_steps, int t0,
                      float lr, float beta1, float beta2, float eps, float* logp,
                      gl_deflection defl, void* stream) {
  gl::Range nvtx_range("gl_map_adam");
  if (!sys) return fail(GL_EINVAL, "system is NULL");
  if (B < 0 || n_steps < 0 || t0 < 0) return fail(GL_EINVAL, "B, n_steps and t0 must be >= 0");
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f))
    return fail(GL_EINVAL, "need lr > 0, 0 <= beta < 1, eps > 0");
  if (B == 0 || n_steps == 0) return GL_OK;
  if (!u || !m || !v || !logp) return fail(GL_EINVAL, "NULL u, m, v or logp");
  gl_status r = set_dev(sys);
  if (r != GL_OK) return r;
  gl::InferState* f;
  if ((r = infer_state(sys, &f)) != GL_OK) return r;
  SysParams sp;
  size_t dyn;
  if ((r = gl::eval_prepare(sys, B, defl, true, &sp, &dyn)) != GL_OK) return r;
  const int P = sys->sp.P;
  const size_t need = (size_t)B * (2 * P + 1);
  if (need > f->map_buf_floats) {
    if (f->map_exec) {
      cudaGraphExecDestroy(f->map_exec);
      f->map_exec = nullptr;
    }
    cudaFree(f->map_buf);
    cudaFree(f->map_jc);
    f->map_buf = nullptr;
    f->map_jc = nullptr;
    f->map_buf_floats = 0;
    GI_CUDA(cudaMalloc(&f->map_buf, need * sizeof(float)), "buffer allocation");
    GI_CUDA(cudaMalloc(&f->map_jc, (size_t)B * (3 * P + 1) * sizeof(double)), "buffer allocation");
    f->map_buf_floats = need;
  }
  if (!f->map_ctl) GI_CUDA(cudaMalloc(&f->map_ctl, sizeof(MapCtl)), "control allocation");
  cudaStream_t st = (cudaStream_t)stream;
  const MapCtl hc{t0, lr, beta1, beta2, eps};
  k_set_map_ctl<<<1, 1, 0, st>>>(f->map_ctl, hc);
  GI_CUDA(cudaGetLastError(), "control");
  float* th = f->map_buf;
  float* gth = th + (size_t)B * P;
  float* lpth = gth + (size_t)B * P;
  gl::InferState::MapKey key;
  std::memset(&key, 0, sizeof key);
  key.u = u; key.m = m; key.v = v; key.logp = logp;
  key.scratch = sp.scratch;
  key.table = const_cast<float4*>(sp.table);
  key.sur = sys->sur;
  key.B = B; key.n = n_steps; key.defl = (int)defl;
  if (!f->map_exec || std::memcmp(&key, &f->map_key, sizeof key) != 0) {
    if (f->map_exec) {
      cudaGraphExecDestroy(f->map_exec);
      f->map_exec = nullptr;
    }
    if (!f->cap) GI_CUDA(cudaStreamCreateWithFlags(&f->cap, cudaStreamNonBlocking), "stream");
    GI_CUDA(cudaStreamBeginCapture(f->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = cudaSuccess;
    double* jc = f->map_jc;
    double* ljc = jc + (size_t)B * 3 * P;
    k_to_theta_cache<<<grid_rows(B), 256, 0, f->cap>>>(f->bij, P, u, B, th, jc, ljc);
    e = cudaGetLastError();
    for (int k = 0; k < n_steps && e == cudaSuccess; ++k) {
      e = gl::eval_launch(sys, sp, dyn, th, B, lpth, gth, defl, f->cap);
      if (e != cudaSuccess) break;
      k_map_update<<<grid_rows(B), 256, 0, f->cap>>>(f->bij, P, B, u, m, v, lpth, gth, logp,
                                                     f->map_ctl, k, th, jc, ljc);
      e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(f->cap, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e, "MAP capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
    e = cudaGraphInstantiate(&f->map_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      f->map_exec = nullptr;
      return cuda_fail(e, "graph instantiate");
    }
    std::memcpy(&f->map_key, &key, sizeof key);
  }
  GI_CUDA(cudaGraphLaunch(f->map_exec, st), "graph launch");
  return GL_OK;
}

// ------------------------------------------------------------------ HMC ----
gl_status gl_hmc_create(gl_system* sys, const gl_hmc_desc* d, const float* u0, gl_hmc** out,
                        void* stream) {
  if (!out) return fail(GL_EINVAL, "out is NULL");
  *out = nullptr;
  if (!sys || !d || !u0) return fail(GL_EINVAL, "NULL system, desc or u0");
  if (d->chains < 1 || d->n_leapfrog < 1) return fail(GL_EINVAL, "chains and n_leapfrog >= 1");
  if (!(d->step_size > 0.f) || !std::isfinite(d->step_size))
    return fail(GL_EINVAL, "step_size must be positive and finite");
  if (!(d->target_accept > 0.f && d->target_accept < 1.f))
    return fail(GL_EINVAL, "target_accept must be in (0, 1)");
  const gl_deflection defl = (gl_deflection)d->deflection;
  gl_status r = set_dev(sys);
  if (r != GL_OK) return r;
  gl::InferState* f;
  if ((r = infer_state(sys, &f)) != GL_OK) return r;
  SysParams sp;
  size_t dyn;
  const int B = d->chains, P = sys->sp.P;
  if ((r = gl::eval_prepare(sys, B, defl, true, &sp, &dyn)) != GL_OK) return r;
  auto* h = new gl_hmc();
  h->sys = sys;
  h->B = B;
  h->P = P;
  h->L = d->n_leapfrog;
  h->defl = defl;
  h->seed = d->seed;
  const size_t BP = (size_t)B * P;
  const size_t total = 7 * BP + 6 * (size_t)B + P;
  cudaError_t e = cudaMalloc(&h->pool, total * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&h->jpool, (3 * BP + (size_t)B) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->ctl, sizeof(HmcDev));
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_ctl, sizeof(HmcDev));
  if (e != cudaSuccess) {
    gl_hmc_destroy(h);
    return cuda_fail(e, "sampler allocation");
  }
  float* q = h->pool;
  h->b.u = q; q += BP;
  h->b.g = q; q += BP;
  h->b.u0 = q; q += BP;
  h->b.g0 = q; q += BP;
  h->b.p = q; q += BP;
  h->b.th = q; q += BP;
  h->b.g_th = q; q += BP;
  h->b.lp = q; q += B;
  h->b.lp0 = q; q += B;
  h->b.H0 = q; q += B;
  h->b.prob = q; q += B;
  h->b.lp_th = q; q += B;
  q += B;  // spare
  h->b.inv_mass = q;
  h->b.jc = h->jpool;
  h->b.ljc = h->jpool + 3 * BP;
  HmcDev& c = *h->h_ctl;
  std::memset(&c, 0, sizeof c);
  c.eps = d->step_size;
  c.mu = std::log(10.0 * d->step_size);
  c.log_eps = std::log((double)d->step_size);
  c.target = d->target_accept;
  cudaStream_t st = (cudaStream_t)stream;
  e = cudaMemcpyAsync(h->ctl, &c, sizeof c, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->b.u, u0, BP * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) {
    k_fill<<<(P + 63) / 64, 64, 0, st>>>(h->b.inv_mass, P, 1.f);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    k_to_theta<<<grid_rows(B), 256, 0, st>>>(f->bij, P, h->b.u, B, h->b.th, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = gl::eval_launch(sys, sp, dyn, h->b.th, B, h->b.lp_th, h->b.g_th, defl, st);
  if (e == cudaSuccess) {
    k_pullback<<<grid_rows(B), 256, 0, st>>>(f->bij, P, h->b.u, B, h->b.lp_th, h->b.g_th, h->b.lp,
                                             h->b.g);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // creation waits for its evaluation
  if (e != cudaSuccess) {
    gl_hmc_destroy(h);
    return cuda_fail(e, "sampler set-up");
  }
  *out = h;
  return GL_OK;
}

gl_status gl_hmc_set_inv_mass(gl_hmc* h, const float* inv_mass, void* stream) {
  if (!h || !inv_mass) return fail(GL_EINVAL, "NULL sampler or inv_mass");
  gl_status r = set_dev(h->sys);
  if (r != GL_OK) return r;
  GI_CUDA(cudaMemcpyAsync(h->b.inv_mass, inv_mass, h->P * sizeof(float), cudaMemcpyDeviceToDevice,
                          (cudaStream_t)stream),
          "copy inv_mass");
  return GL_OK;
}

gl_status gl_hmc_run(gl_hmc* h, int n, int flags, float* draws, float* accept, void* stream) {
  gl::Range nvtx_range("gl_hmc_run");
  if (!h) return fail(GL_EINVAL, "sampler is NULL");
  if (n < 0) return fail(GL_EINVAL, "n must be >= 0");
  if (flags & ~(GL_HMC_ADAPT_STEP | GL_HMC_COLLECT_MOMENTS)) return fail(GL_EINVAL, "unknown flags");
  if (n == 0) return GL_OK;
  gl_system* sys = h->sys;
  gl_status r = set_dev(sys);
  if (r != GL_OK) return r;
  gl::InferState* f;
  if ((r = infer_state(sys, &f)) != GL_OK) return r;
  SysParams sp;
  size_t dyn;
  if ((r = gl::eval_prepare(sys, h->B, h->defl, true, &sp, &dyn)) != GL_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if (!h->exec || h->key_scratch != (void*)sp.scratch || h->key_table != (const void*)sp.table ||
      h->key_sur != (const void*)sys->sur) {
    if (h->exec) {
      cudaGraphExecDestroy(h->exec);
      h->exec = nullptr;
    }
    if (!h->cap) GI_CUDA(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking), "stream");
    GI_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    const int B = h->B, P = h->P;
    k_hmc_begin<<<grid_rows(B), 256, 0, h->cap>>>(f->bij, P, B, h->ctl, h->seed, h->b);
    cudaError_t e = cudaGetLastError();
    for (int k = 0; k < h->L && e == cudaSuccess; ++k) {
      e = gl::eval_launch(sys, sp, dyn, h->b.th, B, h->b.lp_th, h->b.g_th, h->defl, h->cap);
      if (e != cudaSuccess) break;
      k_hmc_mid<<<grid_rows(B), 256, 0, h->cap>>>(f->bij, P, B, h->ctl, h->b, k == h->L - 1);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_hmc_end<<<grid_rows(B), 256, 0, h->cap>>>(f->bij, P, B, h->ctl, h->seed, h->b);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_hmc_adapt<<<1, 256, 0, h->cap>>>(h->ctl, h->b.prob, h->b.u, B, P);
      e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e, "HMC capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
    e = cudaGraphInstantiate(&h->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->exec = nullptr;
      return cuda_fail(e, "graph instantiate");
    }
    h->key_scratch = sp.scratch;
    h->key_table = const_cast<float4*>(sp.table);
    h->key_sur = sys->sur;
  }
  k_set_hmc_run<<<1, 1, 0, st>>>(h->ctl, flags, draws, accept);
  GI_CUDA(cudaGetLastError(), "control");
  for (int k = 0; k < n; ++k) GI_CUDA(cudaGraphLaunch(h->exec, st), "graph launch");
  return GL_OK;
}

gl_status gl_hmc_end_adaptation(gl_hmc* h, int set_inv_mass, void* stream) {
  if (!h) return fail(GL_EINVAL, "sampler is NULL");
  gl_status r = set_dev(h->sys);
  if (r != GL_OK) return r;
  k_hmc_end_adapt<<<1, 64, 0, (cudaStream_t)stream>>>(h->ctl, h->b.inv_mass, h->P, set_inv_mass);
  GI_CUDA(cudaGetLastError(), "adaptation launch");
  return GL_OK;
}

gl_status gl_hmc_state(gl_hmc* h, float* u, float* logp, float* inv_mass, float* step_size_host,
                       void* stream) {
  if (!h) return fail(GL_EINVAL, "sampler is NULL");
  gl_status r = set_dev(h->sys);
  if (r != GL_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t BP = (size_t)h->B * h->P;
  if (u) GI_CUDA(cudaMemcpyAsync(u, h->b.u, BP * 4, cudaMemcpyDeviceToDevice, st), "copy u");
  if (logp) GI_CUDA(cudaMemcpyAsync(logp, h->b.lp, h->B * 4, cudaMemcpyDeviceToDevice, st), "copy");
  if (inv_mass)
    GI_CUDA(cudaMemcpyAsync(inv_mass, h->b.inv_mass, h->P * 4, cudaMemcpyDeviceToDevice, st), "copy");
  if (step_size_host) {
    GI_CUDA(cudaMemcpyAsync(&h->h_ctl->eps, &h->ctl->eps, sizeof(float), cudaMemcpyDeviceToHost, st),
            "copy step size");
    GI_CUDA(cudaStreamSynchronize(st), "stream");
    *step_size_host = h->h_ctl->eps;
  }
  return GL_OK;
}

gl_status gl_hmc_destroy(gl_hmc* h) {
  if (!h) return GL_OK;
  cudaDeviceSynchronize();
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->cap) cudaStreamDestroy(h->cap);
  cudaFree(h->pool);
  cudaFree(h->jpool);
  cudaFree(h->ctl);
  cudaFreeHost(h->h_ctl);
  delete h;
  return GL_OK;
}

// ------------------------------------------------------------------ SVI ----
gl_status gl_svi_adabelief(gl_system* sys, float* phi, float* opt, int n_samples, int n_steps,
                           int t0, float lr, float beta1, float beta2, float eps,
                           unsigned long long seed, float* elbo, gl_deflection defl,
                           void* stream) {
  return gl_svi_adabelief_ex(sys, phi, opt, n_samples, n_steps, t0, lr, beta1, beta2, eps, seed,
                             elbo, defl, GL_SVI_SCORE, stream);
}

gl_status gl_svi_adabelief_ex(gl_system* sys, float* phi, float* opt, int n_samples, int n_steps,
                              int t0, float lr, float beta1, float beta2, float eps,
                              unsigned long long seed, float* elbo, gl_deflection defl,
                              int estimator, void* stream) {
  gl::Range nvtx_range("gl_svi_adabelief");
  if (!sys) return fail(GL_EINVAL, "system is NULL");
  if (n_samples < 1 || n_steps < 0 || t0 < 0)
    return fail(GL_EINVAL, "need n_samples >= 1, n_steps >= 0, t0 >= 0");
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f))
    return fail(GL_EINVAL, "need lr > 0, 0 <= beta < 1, eps > 0");
  if (!phi || !opt) return fail(GL_EINVAL, "NULL phi or opt");
  if (estimator != GL_SVI_SCORE && estimator != GL_SVI_PATHWISE)
    return fail(GL_EINVAL, "unknown SVI gradient estimator");
  if (n_steps == 0) return GL_OK;
  const bool rep = estimator == GL_SVI_PATHWISE;
  gl_status r = set_dev(sys);
  if (r != GL_OK) return r;
  gl::InferState* f;
  if ((r = infer_state(sys, &f)) != GL_OK) return r;
  SysParams sp;
  size_t dyn;
  const int n = n_samples, P = sys->sp.P;
  if ((r = gl::eval_prepare(sys, n, defl, rep, &sp, &dyn)) != GL_OK) return r;
  const size_t nP = (size_t)n * P;
  const size_t need = 6 * nP + 4 * (size_t)n;
  if (need > f->svi_buf_floats) {
    if (f->svi_exec) {
      cudaGraphExecDestroy(f->svi_exec);
      f->svi_exec = nullptr;
    }
    cudaFree(f->svi_buf);
    f->svi_buf = nullptr;
    f->svi_buf_floats = 0;
    GI_CUDA(cudaMalloc(&f->svi_buf, need * sizeof(float)), "buffer allocation");
    f->svi_buf_floats = need;
  }
  const int nsums = P + P * (P + 1) / 2 + 2;
  if (!f->svi_sums) GI_CUDA(cudaMalloc(&f->svi_sums, (gl::MAX_P + gl::MAX_P * (gl::MAX_P + 1) / 2 + 2) * sizeof(double)), "sums");
  if (!f->svi_ctl) GI_CUDA(cudaMalloc(&f->svi_ctl, sizeof(SviCtl)), "control allocation");
  cudaStream_t st = (cudaStream_t)stream;
  const SviCtl hc{(unsigned long long)t0, 0, lr, beta1, beta2, eps, elbo};
  k_set_svi_ctl<<<1, 1, 0, st>>>(f->svi_ctl, hc);
  GI_CUDA(cudaGetLastError(), "control");
  float* z = f->svi_buf;
  float* a = z + nP;
  float* u = a + nP;
  float* th = u + nP;
  float* gth = th + nP;   // pathwise: d log p / d theta
  float* gu = gth + nP;   // pathwise: d log p~ / d u
  float* logq = gu + nP;
  float* lp = logq + n;
  float* lj = lp + n;
  float* lpu = lj + n;    // pathwise: log p~(u)
  gl::InferState::SviKey key;
  std::memset(&key, 0, sizeof key);
  key.phi = phi; key.opt = opt;
  key.scratch = sp.scratch;
  key.table = const_cast<float4*>(sp.table);
  key.sur = sys->sur;
  key.n = n; key.defl = (int)defl; key.seed = seed; key.est = estimator;
  if (!f->svi_exec || std::memcmp(&key, &f->svi_key, sizeof key) != 0) {
    if (f->svi_exec) {
      cudaGraphExecDestroy(f->svi_exec);
      f->svi_exec = nullptr;
    }
    if (!f->cap) GI_CUDA(cudaStreamCreateWithFlags(&f->cap, cudaStreamNonBlocking), "stream");
    GI_CUDA(cudaStreamBeginCapture(f->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    k_svi_draw<<<grid_rows(n), 256, 0, f->cap>>>(f->bij, P, n, f->svi_ctl, seed, phi, z, a, logq,
                                                  u, th, lj);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = gl::eval_launch(sys, sp, dyn, th, n, lp, rep ? gth : nullptr, defl, f->cap);
    if (e == cudaSuccess && rep) {
      k_pullback<<<grid_rows(n), 256, 0, f->cap>>>(f->bij, P, u, n, lp, gth, lpu, gu);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      if (rep)
        k_svi_sums_rep<<<nsums - 1, 256, 0, f->cap>>>(P, n, gu, z, logq, lpu, f->svi_sums);
      else
        k_svi_sums<<<nsums - 1, 256, 0, f->cap>>>(P, n, a, z, logq, lp, lj, f->svi_sums);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      k_svi_update<<<1, 256, 0, f->cap>>>(P, phi, opt, f->svi_sums, f->svi_ctl, rep ? 1 : 0);
      e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(f->cap, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e, "SVI capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
    e = cudaGraphInstantiate(&f->svi_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      f->svi_exec = nullptr;
      return cuda_fail(e, "graph instantiate");
    }
    std::memcpy(&f->svi_key, &key, sizeof key);
  }
  for (int k = 0; k < n_steps; ++k) GI_CUDA(cudaGraphLaunch(f->svi_exec, st), "graph launch");
  return GL_OK;
}

// ------------------------------------------------ backward intensities ----
gl_status gl_logp_grad_backward(gl_system* sys, const float* theta, int B, float* logp,
                                float* grad, float* intensity, gl_deflection defl, void* stream) {
  gl::Range nvtx_range("gl_logp_grad_backward");
  if (!sys) return fail(GL_EINVAL, "system is NULL");
  if (B < 0) return fail(GL_EINVAL, "B < 0");
  if (B == 0) return GL_OK;
  if (!theta || !logp || !grad) return fail(GL_EINVAL, "NULL theta, logp or grad");
  gl_status r = set_dev(sys);
  if (r != GL_OK) return r;
  gl::InferState* f;
  if ((r = infer_state(sys, &f)) != GL_OK) return r;
  const int P = sys->sp.P, K = sys->sp.nL + sys->sp.nS;
  const size_t npix = (size_t)sys->sp.ny * sys->sp.nx;
  if (!f->bwd_prior) {
    GI_CUDA(cudaMalloc(&f->bwd_prior, P * sizeof(gl::PriorDev)), "prior allocation");
    GI_CUDA(cudaMemcpy(f->bwd_prior, sys->d_prior, P * sizeof(gl::PriorDev),
                       cudaMemcpyDeviceToDevice), "prior copy");
    k_bwd_prior<<<1, 32>>>(f->bwd_prior, K);
    GI_CUDA(cudaGetLastError(), "prior set-up");
    GI_CUDA(cudaDeviceSynchronize(), "prior set-up");
  }
  // prepare both launches before either runs (the second preparation may
  // grow the scratch or table buffers the first one points into)
  SysParams sg, sf;
  size_t dg, df;
  if ((r = gl::eval_prepare(sys, B, defl, true, &sg, &dg)) != GL_OK) return r;
  if ((r = gl::eval_prepare(sys, B * K, defl, false, &sf, &df)) != GL_OK) return r;
  if ((r = gl::eval_prepare(sys, B, defl, true, &sg, &dg)) != GL_OK) return r;
  const size_t need = (size_t)B * K * P + (size_t)B * K * npix + (size_t)B * P;
  if (need > f->bwd_buf_floats) {
    cudaFree(f->bwd_buf);
    f->bwd_buf = nullptr;
    f->bwd_buf_floats = 0;
    GI_CUDA(cudaMalloc(&f->bwd_buf, need * sizeof(float)), "buffer allocation");
    f->bwd_buf_floats = need;
  }
  float* rows = f->bwd_buf;
  float* imgs = rows + (size_t)B * K * P;
  float* th_star = imgs + (size_t)B * K * npix;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nr = (size_t)B * K * P;
  k_bwd_rows<<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(theta, B, P, K, rows);
  GI_CUDA(cudaGetLastError(), "row launch");
  if (sf.table)
    GI_CUDA(gl::launch_table(defl, sys->sur, rows, P, B * K, const_cast<float4*>(sf.table), st),
            "table launch");
  GI_CUDA(gl::launch_component_images(sf, rows, B * K, imgs, df, st), "image launch");
  switch (K) {
#define GL_BWD(k)                                                                          \
  case k:                                                                                  \
    k_bwd_solve<k><<<B, 256, 0, st>>>(imgs, sys->d_data, sys->d_w, (int)npix, B, P, theta, \
                                      th_star, intensity);                                 \
    break;
    GL_BWD(1) GL_BWD(2) GL_BWD(3) GL_BWD(4) GL_BWD(5)
#undef GL_BWD
    default: return fail(GL_EINVAL, "unsupported number of light components");
  }
  GI_CUDA(cudaGetLastError(), "solve launch");
  sg.prior = f->bwd_prior;
  GI_CUDA(gl::eval_launch(sys, sg, dg, th_star, B, logp, grad, defl, st), "gradient launch");
  k_bwd_zero<<<(B * K + 255) / 256, 256, 0, st>>>(grad, B, P, K);
  GI_CUDA(cudaGetLastError(), "launch");
  return GL_OK;
}

}  // extern "C"
