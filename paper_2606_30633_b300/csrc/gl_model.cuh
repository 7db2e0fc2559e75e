// Device-side lens model: per-sample staging of the EPL series deflection and
// the elliptical Sersic profiles, and the conversion of the adjoint's native
// sums to parameter gradients (the sub-pixel evaluations are in
// gl_subpixel.cuh).
//
// Notation (Sec. 3 parameters; Tessore & Metcalf 2015 for the EPL):
//   lens frame  x' = cs dx + sn dy, y' = cs dy - sn dx about the centre,
//               (cs, sn) = (cos, sin) of the position angle atan2(e2, e1)/2;
//   EPL         R^2 = q^2 x'^2 + y'^2, e^{i vphi} = (q x' + i y')/R,
//               w = e^{2 i vphi}, z = -f w (f = |e|), t = gamma - 1,
//               F(z) = 2F1(1, t/2; 2 - t/2; z) = 1 + z E,
//               E = sum_{n>=1} c_n z^{n-1},  c_n = c_{n-1} (2n-2+t)/(2n+2-t),
//               alpha' = A e^{i vphi} F,  A = 2 b^t R^{1-t}/(1+q),  b = theta_E sqrt(q);
//   Sersic      R^2 = q x'^2 + y'^2/q, p = (R/R_e)^{1/n},
//               S = I_e e^{b_n} 2^{-b_n log2(e) p}.
//
// Adjoint identities used (no extra series beyond the t-derivative):
//   * complex shear of a homogeneous deflection, alpha(l z) = l^{1-t} alpha(z):
//       kappa z + gamma zbar = (1 - t) alpha   (Euler's relation, with
//       d alpha = kappa dz + gamma dzbar), so rotating the lens needs no gamma;
//   * for a = 1 the series obeys 2 z (1 - z) F' = (2 - t)(1 - F) + t z F, so
//       F'(z) = [t F - (2 - t) E] / (2 (1 - z))   (no division by z);
//   * dF/dt = z sum_{n>=1} c_n h_n z^{n-1},  h_n = sum_{k<=n} 1/(2k-2+t) + 1/(2k+2-t).
#pragma once

#include <cstddef>

#include "gl_internal.cuh"

namespace gl {

constexpr float R_MIN2 = 1e-12f;   // radius clamp 1e-6 arcsec, squared
constexpr double E_DOMAIN = 0.8;
constexpr double N_SERSIC_MIN = 0.2;
constexpr double LN2 = 0.69314718055994530942;
constexpr double SERIES_EPS = 5.9604644775390625e-08;  // 2^-24

// ---- MUFU primitives (PTX approximate instructions) ----
__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsq(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// ---- paired FP32 arithmetic ----
// The sub-pixel code evaluates two points at a time, one in each lane of a
// float2: the FP32 operations are paired (f32x2) instructions, MUFU ones stay
// per lane.
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// Written as a lane-wise sign change (not a multiply by -1) so that the
// compiler folds it into the consuming paired instruction's operand: 2 % of
// the fused kernel's time on the ground-based workload.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 max2(float2 a, float b) {
  return make_float2(fmaxf(a.x, b), fmaxf(a.y, b));
}
__device__ __forceinline__ float2 ex2_2(float2 a) { return make_float2(ex2(a.x), ex2(a.y)); }
__device__ __forceinline__ float2 lg2_2(float2 a) { return make_float2(lg2(a.x), lg2(a.y)); }
__device__ __forceinline__ float2 rsq2(float2 a) { return make_float2(rsq(a.x), rsq(a.y)); }
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(rcp(a.x), rcp(a.y)); }

// Per-sample constants, each held twice (both lanes of a float2) so that the
// paired code uses them without moves; a leading "n" marks a negated value.
struct EplP {
  float2 nxc, nyc;            // minus the centre
  float2 cs, sn, ncs, nsn;    // position angle
  float2 qcs, qsn;            // q (cos, sin): q x' = qcs dx + qsn dy
  float2 iq, nq;              // 1/q, -q
  float2 f, nf, m2f;          // f = |e|, -f, -2f
  float2 ht, CA;              // (1 - t)/2, 2 b^t / (1 + q)
  float2 t, omt, ntmt;        // t, 1 - t, -(2 - t)
  float2 omtq;                // (1 - t) q
  float2 lnb;
  float2 ndfdq;               // -d f / d q = 2/(1+q)^2
};

// Per-sample constants of one Sersic component (paired).
// The component frame is staged pre-scaled: u = sqrt(q) x', v = y'/sqrt(q) from
// the offset (dx, dy), so that R^2 = q x'^2 + y'^2/q = u^2 + v^2.
struct LightP {
  float2 nxc, nyc;
  float2 ucs, usn;            // sqrt(q) (cos phi, sin phi):  u = ucs dx + usn dy
  float2 vcs, vnsn;           // (cos phi, -sin phi)/sqrt(q): v = vcs dy + vnsn dx
  float2 c1, c0;              // log2 p = c1 log2(R^2) + c0
  float2 nbl;                 // -b_n log2(e)
  float2 Ip;                  // I_e e^{b_n}
  float2 kX1, kX2, kY1, kY2;  // dS/d(X,Y) = S p/R^2 (kX1 u + kX2 v, kY1 u + kY2 v)
};

struct SampleC {
  EplP epl;
  float2 omg1, opg1, ng2;    // 1 - g1, 1 + g1, -g2 (external shear)
  LightP light[MAX_COMP];    // lens lights, then sources
  // the summation loops read two coefficients at a time as float4: 16-byte aligned
  alignas(16) float2 cE[N_MAX];  // E-series coefficients c_n (-f)^{n-1}, n = 1..2 n2 (index n-1), paired
  alignas(16) float2 cT[N_MAX];  // t-derivative coefficients c_n h_n (-f)^{n-1}, paired
  int n2;                    // number of 2-term chunks (N rounded up to a multiple of 2)
  int status;                // 0 ok, 1 outside domain/support (-inf), 2 NaN
  int use_table;             // surrogate table covers this row
  double logprior;
  float dprior[MAX_P];
};

static_assert(offsetof(SampleC, cE) % 16 == 0 && offsetof(SampleC, cT) % 16 == 0,
              "series coefficients must be 16-byte aligned (read as float4)");
static_assert(alignof(SampleC) >= 16, "SampleC must keep its 16-byte members aligned");

__device__ __forceinline__ int ellip_index(int c) { return c == 0 ? 2 : 8 + 7 * (c - 1) + 2; }

// Per-component constants kept for the gradient's chain rule at the end.
struct FinishC {
  float e1, e2, c, cs, sn, q;
  float p0;         // theta_E (EPL) or R_e (Sersic)
  float n, I, bn;   // Sersic index, intensity, b_n (unused for the EPL)
  float t;          // EPL t = gamma - 1
};

// Stages one sample on warp 0 (all 32 lanes call it): NaN, domain and prior
// support checks, the log prior and its gradient (one lane per parameter),
// per-component constants (one lane per component) and the EPL series
// coefficients (a warp prefix product). FP32 with IEEE-accurate library
// functions; the prior's normalisation constants and the log-prior sum are
// FP64. Writes sc.status last (0 ok, 1 -inf, 2 NaN).
__device__ inline void stage_warp(const SysParams& sp, const float* __restrict__ th, SampleC& sc,
                                  FinishC* fin, bool check_prior) {
  const int lane = threadIdx.x & 31;
  const int P = sp.P;
  const int nc = sp.nL + sp.nS;
  // NaN
  bool nan = false;
  for (int k = lane; k < P; k += 32) nan |= isnan(th[k]);
  if (__any_sync(0xffffffffu, nan)) {
    if (lane == 0) sc.status = 2;
    return;
  }
  // domain (one lane per component)
  bool bad = false;
  if (lane <= nc) {
    const int i1 = ellip_index(lane);
    const float e1 = th[i1], e2 = th[i1 + 1];
    const double e = sqrt((double)e1 * e1 + (double)e2 * e2);
    if (!(e < E_DOMAIN)) bad = true;
    if (check_prior && sp.emax) {
      const double em = (double)sp.emax[lane];
      if (em > 0.0 && !(e < em)) bad = true;
    }
    if (lane == 0) {
      if (!(th[0] > 0.f) || !(th[1] > 1.f && th[1] < 3.f)) bad = true;
    } else {
      if (!(th[i1 - 2] > 0.f) || !((double)th[i1 - 1] >= N_SERSIC_MIN)) bad = true;
    }
  }
  // prior (one lane per parameter)
  double lp = 0.0;
  if (check_prior) {
    for (int k = lane; k < P; k += 32) {
      const PriorDev pr = sp.prior[k];
      const float x = th[k];
      float d = 0.f;
      switch (pr.kind) {
        case 0:
          if (!(x >= pr.lo && x <= pr.hi)) bad = true;
          break;
        case 1:
          if (!(x >= pr.lo && x <= pr.hi)) bad = true;
          lp += pr.cnst;
          break;
        case 2: {
          const float z = (x - pr.a) / pr.b;
          lp += (double)(-0.5f * z * z) + pr.cnst;
          d = -z / pr.b;
          break;
        }
        case 3: {
          if (!(x >= pr.lo && x <= pr.hi)) bad = true;
          const float z = (x - pr.a) / pr.b;
          lp += (double)(-0.5f * z * z) + pr.cnst;
          d = -z / pr.b;
          break;
        }
        case 4: {
          if (!(x > 0.f)) { bad = true; break; }
          const float lx = logf(x);
          const float z = (lx - pr.a) / pr.b;
          lp += (double)(-0.5f * z * z) - (double)lx + pr.cnst;
          d = (-z / pr.b - 1.f) / x;
          break;
        }
        default: break;
      }
      sc.dprior[k] = d;
    }
  }
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) sc.status = 1;
    return;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lp += __shfl_xor_sync(0xffffffffu, lp, o);

  // per-component constants
  float t_epl = 0.f, f_epl = 0.f;
  if (lane <= nc) {
    const int i1 = ellip_index(lane);
    const float e1 = th[i1], e2 = th[i1 + 1];
    const float c = sqrtf(e1 * e1 + e2 * e2);
    const float q = (1.f - c) / (1.f + c);
    float sn, cs;
    sincosf(0.5f * atan2f(e2, e1), &sn, &cs);
    FinishC& F = fin[lane];
    F.e1 = e1; F.e2 = e2; F.c = c; F.cs = cs; F.sn = sn; F.q = q;
    if (lane == 0) {
      EplP& E = sc.epl;
      const float t = th[1] - 1.f;
      const float b = th[0] * sqrtf(q);
      E.nxc = f2(-th[4]); E.nyc = f2(-th[5]);
      E.cs = f2(cs); E.sn = f2(sn); E.ncs = f2(-cs); E.nsn = f2(-sn);
      E.qcs = f2(q * cs); E.qsn = f2(q * sn); E.iq = f2(1.f / q); E.nq = f2(-q);
      E.f = f2(c); E.nf = f2(-c); E.m2f = f2(-2.f * c);
      E.ht = f2(0.5f * (1.f - t));
      E.CA = f2(2.f * powf(b, t) / (1.f + q));
      E.t = f2(t); E.omt = f2(1.f - t); E.ntmt = f2(t - 2.f);
      E.omtq = f2((1.f - t) * q);
      E.lnb = f2(logf(b));
      E.ndfdq = f2(2.f / ((1.f + q) * (1.f + q)));
      F.p0 = th[0]; F.t = t; F.n = 0.f; F.I = 0.f; F.bn = 0.f;
      t_epl = t;
      f_epl = c;
      sc.omg1 = f2(1.f - th[6]);
      sc.opg1 = f2(1.f + th[6]);
      sc.ng2 = f2(-th[7]);
      // the table path's rotation term divides d log p / d phi by 2 |e|^2, so
      // nearly round lenses (|e| < TABLE_MIN_E) take the series
      sc.use_table = (sp.table != nullptr || sp.net_wimg != nullptr) && q >= sp.sq_lo &&
                     q <= sp.sq_hi &&
                     th[1] >= sp.sg_lo && th[1] <= sp.sg_hi && c >= TABLE_MIN_E;
    } else {
      LightP& L = sc.light[lane - 1];
      const float* p = th + 8 + 7 * (lane - 1);
      const float Re = p[0], n = p[1];
      const float bn = 1.9992f * n - 0.3271f;
      L.nxc = f2(-p[4]); L.nyc = f2(-p[5]);
      const float rq = sqrtf(q);
      L.ucs = f2(rq * cs); L.usn = f2(rq * sn);
      L.vcs = f2(cs / rq); L.vnsn = f2(-sn / rq);
      L.c1 = f2(0.5f / n);
      L.c0 = f2(-log2f(Re) / n);
      L.nbl = f2(-bn * 1.4426950408889634f);
      L.Ip = f2(p[6] * expf(bn));
      const float m = -bn / n;
      L.kX1 = f2(m * rq * cs); L.kX2 = f2(-m * sn / rq);
      L.kY1 = f2(m * rq * sn); L.kY2 = f2(m * cs / rq);
      F.p0 = Re; F.n = n; F.I = p[6]; F.bn = bn; F.t = 0.f;
    }
  }
  t_epl = __shfl_sync(0xffffffffu, t_epl, 0);
  f_epl = __shfl_sync(0xffffffffu, f_epl, 0);
  // Coefficients e_n = c_n (-f)^{n-1} = prod_{k<=n} rho_k, rho_1 = r_1,
  // rho_k = -f r_k, r_k = (2k-2+t)/(2k+2-t); t_n = e_n h_n, h_n = sum_{k<=n}
  // 1/(2k-2+t) + 1/(2k+2-t): inclusive warp scans of products and sums, 32
  // terms per pass. |e_n| decreases (|rho_k| < f for k >= 2), so the tail
  // after N terms is at most |e_{N+1}| / (1 - f); the series stops at the
  // first N with |e_{N+1}| <= 2^-24 (1-f)^2 / 2, and 2 ceil(N/2) coefficients
  // are staged (zeros past N), the summation loops taking two per step.
  const float tol = (float)SERIES_EPS * (1.f - f_epl) * (1.f - f_epl) * 0.5f;
  float carry_e = 1.f, carry_h = 0.f;
  int N = N_MAX;
  for (int base = 0; base < N_MAX; base += 32) {
    const int n = base + lane + 1;
    const float a = 2.f * n - 2.f + t_epl, bb = 2.f * n + 2.f - t_epl;
    float rho = (n == 1 ? 1.f : -f_epl) * (a / bb);
    float hin = 1.f / a + 1.f / bb;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float r2 = __shfl_up_sync(0xffffffffu, rho, o);
      const float h2 = __shfl_up_sync(0xffffffffu, hin, o);
      if (lane >= o) { rho *= r2; hin += h2; }
    }
    const float en = carry_e * rho, hn = carry_h + hin;
    const unsigned cut = __ballot_sync(0xffffffffu, n >= 2 && fabsf(en) <= tol);
    if (cut) N = base + __ffs(cut) - 1;  // the first n past the cut is N + 1
    sc.cE[n - 1] = f2(n <= N ? en : 0.f);
    sc.cT[n - 1] = f2(n <= N ? en * hn : 0.f);
    if (cut) break;
    carry_e = __shfl_sync(0xffffffffu, en, 31);
    carry_h = __shfl_sync(0xffffffffu, hn, 31);
  }
  const int n2 = (N + 1) >> 1;
  if (lane == 0) {
    sc.n2 = n2;
    sc.logprior = lp;
    sc.status = 0;
  }
}

// Converts a Sersic component's native accumulators a[0..6] to gradients
// w.r.t. [R_e, n, e1, e2, x, y, I_e] (one lane per component).
// amp_deferred: a lens-light component, whose sums a[1..6] were taken without
// the amplitude I_e e^{b_n} (a[0] sums u S / (I_e e^{b_n}) for every component).
__device__ inline void sersic_finish(const FinishC& F, const double* a, float* g,
                                     bool amp_deferred) {
  const float m = -F.bn / F.n;
  const double eb = (double)expf(F.bn);
  const double amp = (double)(F.I * expf(F.bn));  // the staged I_e e^{b_n}
  const double s16 = amp_deferred ? amp : 1.0;
  // a[3], a[5], a[6] hold sums over u^2 - v^2, u, v (u = sqrt(q) x', v = y'/sqrt(q));
  // A3, A5, A6 are the same sums over x'^2 - y'^2/q^2, x', y'
  const float rq = sqrtf(F.q);
  const float A0 = (float)(amp * a[0]), A1 = (float)(s16 * a[1]), A2 = (float)(s16 * a[2]);
  const float A3 = (float)(s16 * a[3]) / F.q;
  const float A4 = (float)(s16 * a[4]), A5 = (float)(s16 * a[5]) / rq, A6 = (float)(s16 * a[6]) * rq;
  // d/dphi = m (q - 1/q) A4 with q - 1/q = -4c/(1-c^2); d phi/d e = (-e2, e1)/(2c^2),
  // so the rotation part of d/de is 2 m A4 (sin 2phi, -cos 2phi)/(1-c^2) (no 1/c)
  const float dq = 0.5f * m * A3;
  const float rot = 2.f * m * A4 / (1.f - F.c * F.c);
  const float Sx = m * F.q * A5, Sy = m * A6 / F.q;  // sum u dS/dx', sum u dS/dy'
  // cos 2phi, sin 2phi of the staged angle phi = atan2(e2, e1)/2: e/|e| for e != 0, and
  // (1, 0) at e = 0, where the gradient is the limit along e1 -> 0+ (the model is
  // smooth in (e1, e2) there)
  const float c2p = F.cs * F.cs - F.sn * F.sn, s2p = 2.f * F.cs * F.sn;
  const float dqdc = -2.f / ((1.f + F.c) * (1.f + F.c));
  g[0] = F.bn / (F.n * F.p0) * A1;
  g[1] = -1.9992f * (A1 - A0) + F.bn * 0.69314718f / F.n * A2;
  g[2] = dq * dqdc * c2p + rot * s2p;
  g[3] = dq * dqdc * s2p - rot * c2p;
  g[4] = -(F.cs * Sx - F.sn * Sy);
  g[5] = -(F.sn * Sx + F.cs * Sy);
  g[6] = (float)(eb * a[0]);  // d S / d I_e = e^{b_n} Se: finite at I_e = 0
}

// EPL + shear native accumulators:
// [0] sum s1 (theta_E), [1] d/dt, [2] d/dq, [3] sum (kappa/Kk) v.(iY) with
// d/dphi = -2 f Kk [3] (exact series; Kk = (2 - t)(1 + q)/4 is applied here)
// or d/dphi itself (surrogate table),
// [4] sum v.d alpha/dx', [5] sum v.d alpha/dy' (lens frame; the centre
// gradient is minus these), [6] d/dg1, [7] d/dg2.
// With f = |e| and d phi/d e = (-e2, e1)/(2 f^2) the rotation part of d/de is
// [3] (sin 2phi, -cos 2phi) for the series: no division by |e|.
__device__ inline void epl_finish(const FinishC& F, const double* a, float* g,
                                  bool rot_is_dphi = false) {
  const float gxl = -(float)a[4], gyl = -(float)a[5];
  const float cc = fmaxf(F.c, 1e-30f);
  const float c2p = F.cs * F.cs - F.sn * F.sn, s2p = 2.f * F.cs * F.sn;  // as in sersic_finish
  const float dqdc = -2.f / ((1.f + F.c) * (1.f + F.c));
  // a[2] holds the q-derivative without its constant part a0 sum s1, a0 =
  // t/(2q) - 1/(1+q) (the derivative of ln of the deflection prefactor)
  const double a0 = (double)F.t / (2.0 * F.q) - 1.0 / (1.0 + F.q);
  // the series path sums kappa/Kk v.(iY) in a[3]; Kk = (2 - t)(1 + q)/4 per sample
  const double Kk = (2.0 - (double)F.t) * (1.0 + (double)F.q) * 0.25;
  const float dq = (float)(a[2] + a0 * a[0]), rot = (float)(rot_is_dphi ? a[3] : Kk * a[3]);
  g[0] = F.t / F.p0 * (float)a[0];
  g[1] = (float)a[1];
  if (rot_is_dphi) {
    const float k = rot / (2.f * cc * cc);
    g[2] = dq * dqdc * c2p - k * F.e2;
    g[3] = dq * dqdc * s2p + k * F.e1;
  } else {
    g[2] = dq * dqdc * c2p + rot * s2p;
    g[3] = dq * dqdc * s2p - rot * c2p;
  }
  g[4] = F.cs * gxl - F.sn * gyl;
  g[5] = F.sn * gxl + F.cs * gyl;
  g[6] = (float)a[6];
  g[7] = (float)a[7];
}

}  // namespace gl
