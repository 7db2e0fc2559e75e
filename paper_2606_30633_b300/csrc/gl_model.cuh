// Device-side lens model: per-sample staging, the EPL series deflection, the
// elliptical Sersic profile, and their hand-written adjoints.
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

// Per-sample constants of one Sersic component.
struct LightC {
  float xc, yc, cs, sn;
  float q, iq, iq2;     // q, 1/q, 1/q^2
  float c1, c0;         // log2 p = c1 log2(R^2) + c0
  float bl;             // b_n log2(e)
  float Ip;             // I_e e^{b_n}
  float kX1, kX2, kY1, kY2;  // dS/d(X,Y) = S p/R^2 (kX1 x' + kX2 y', kY1 x' + kY2 y')
};

// Per-sample constants of the EPL.
struct EplC {
  float xc, yc, cs, sn;
  float q, q2, f, ht;   // ht = (1 - t)/2
  float CA;             // 2 b^t / (1 + q)
  float t, omt, tmt;    // t, 1 - t, 2 - t
  float Kk;             // kappa = Kk A / R
  float a0;             // t/(2q) - 1/(1+q)
  float lnb;
  float dfdq;           // -2/(1+q)^2
};

struct SampleC {
  EplC epl;
  float g1, g2;
  LightC light[MAX_COMP];  // lens lights, then sources
  float4 cE[N_MAX / 4];    // E-series coefficients c_n (-f)^{n-1}, n = 1..N (index n-1)
  float4 cT[N_MAX / 4];    // t-derivative coefficients c_n h_n (-f)^{n-1}
  int nq;                  // number of float4 chunks (N rounded up to a multiple of 4)
  int status;              // 0 ok, 1 outside domain/support (-inf), 2 NaN
  double logprior;
  float dprior[MAX_P];
};

__device__ __forceinline__ int ellip_index(int c) { return c == 0 ? 2 : 8 + 7 * (c - 1) + 2; }

// Stages one sample: checks NaN, domain and prior support, evaluates the log
// prior (and its gradient), and the per-sample constants of every component.
// Runs on one thread in double precision. check_prior = false skips the
// prior (model-image rendering).
__device__ inline void stage_sample(const SysParams& sp, const float* __restrict__ th,
                                    SampleC& sc, bool check_prior) {
  const int P = sp.P;
  const int nc = sp.nL + sp.nS;
  double v[MAX_P];
  for (int k = 0; k < P; ++k) {
    v[k] = (double)th[k];
    if (isnan(v[k])) { sc.status = 2; return; }
  }
  sc.status = 1;
  if (!(v[0] > 0.0)) return;
  if (!(v[1] > 1.0 && v[1] < 3.0)) return;
  for (int c = 0; c <= nc; ++c) {
    const int i1 = ellip_index(c);
    const double e = sqrt(v[i1] * v[i1] + v[i1 + 1] * v[i1 + 1]);
    if (!(e < E_DOMAIN)) return;
    if (check_prior && sp.emax) {
      const double em = (double)sp.emax[c];
      if (em > 0.0 && !(e < em)) return;
    }
    if (c > 0) {
      if (!(v[i1 - 2] > 0.0)) return;
      if (!(v[i1 - 1] >= N_SERSIC_MIN)) return;
    }
  }
  double lp = 0.0;
  if (check_prior) {
    for (int k = 0; k < P; ++k) {
      const PriorDev pr = sp.prior[k];
      const double x = v[k], a = pr.a, b = pr.b;
      double d = 0.0;
      switch (pr.kind) {
        case 0:
          if (!(x >= (double)pr.lo && x <= (double)pr.hi)) return;
          break;
        case 1:
          if (!(x >= (double)pr.lo && x <= (double)pr.hi)) return;
          lp += pr.cnst;
          break;
        case 2: {
          const double z = (x - a) / b;
          lp += -0.5 * z * z + pr.cnst;
          d = -z / b;
          break;
        }
        case 3: {
          if (!(x >= (double)pr.lo && x <= (double)pr.hi)) return;
          const double z = (x - a) / b;
          lp += -0.5 * z * z + pr.cnst;
          d = -z / b;
          break;
        }
        case 4: {
          if (!(x > 0.0)) return;
          const double lx = log(x);
          const double z = (lx - a) / b;
          lp += -0.5 * z * z - lx + pr.cnst;
          d = (-z / b - 1.0) / x;
          break;
        }
        default: break;
      }
      sc.dprior[k] = (float)d;
    }
  }
  sc.logprior = lp;

  // EPL
  {
    EplC& E = sc.epl;
    const double e1 = v[2], e2 = v[3];
    const double c = sqrt(e1 * e1 + e2 * e2);
    const double q = (1.0 - c) / (1.0 + c);
    const double phi = 0.5 * atan2(e2, e1);
    const double t = v[1] - 1.0;
    const double b = v[0] * sqrt(q);
    E.xc = (float)v[4];
    E.yc = (float)v[5];
    E.cs = (float)cos(phi);
    E.sn = (float)sin(phi);
    E.q = (float)q;
    E.q2 = (float)(q * q);
    E.f = (float)c;
    E.ht = (float)(0.5 * (1.0 - t));
    E.CA = (float)(2.0 * pow(b, t) / (1.0 + q));
    E.t = (float)t;
    E.omt = (float)(1.0 - t);
    E.tmt = (float)(2.0 - t);
    E.Kk = (float)((2.0 - t) * (1.0 + q) / 4.0);
    E.a0 = (float)(t / (2.0 * q) - 1.0 / (1.0 + q));
    E.lnb = (float)log(b);
    E.dfdq = (float)(-2.0 / ((1.0 + q) * (1.0 + q)));
    // terms: smallest N >= 1 with f^N <= 2^-24 (1-f)^2 / 2 (tails of E, F and F')
    const double tol = SERIES_EPS * (1.0 - c) * (1.0 - c) * 0.5;
    int N = 1;
    double fn = c;
    while (fn > tol && N < N_MAX) { fn *= c; ++N; }
    const int nq = (N + 3) / 4;
    sc.nq = nq;
    float* ce = reinterpret_cast<float*>(sc.cE);
    float* ct = reinterpret_cast<float*>(sc.cT);
    double cn = 1.0, hn = 0.0, pw = 1.0;
    for (int n = 1; n <= 4 * nq; ++n) {
      if (n <= N) {
        cn *= (2.0 * n - 2.0 + t) / (2.0 * n + 2.0 - t);
        hn += 1.0 / (2.0 * n - 2.0 + t) + 1.0 / (2.0 * n + 2.0 - t);
        ce[n - 1] = (float)(cn * pw);
        ct[n - 1] = (float)(cn * hn * pw);
        pw *= -c;
      } else {
        ce[n - 1] = 0.f;
        ct[n - 1] = 0.f;
      }
    }
  }
  sc.g1 = (float)v[6];
  sc.g2 = (float)v[7];
  for (int k = 0; k < nc; ++k) {
    LightC& L = sc.light[k];
    const double* p = v + 8 + 7 * k;
    const double e1 = p[2], e2 = p[3];
    const double c = sqrt(e1 * e1 + e2 * e2);
    const double q = (1.0 - c) / (1.0 + c);
    const double phi = 0.5 * atan2(e2, e1);
    const double n = p[1], Re = p[0];
    const double bn = 1.9992 * n - 0.3271;
    const double cs = cos(phi), sn = sin(phi);
    L.xc = (float)p[4];
    L.yc = (float)p[5];
    L.cs = (float)cs;
    L.sn = (float)sn;
    L.q = (float)q;
    L.iq = (float)(1.0 / q);
    L.iq2 = (float)(1.0 / (q * q));
    L.c1 = (float)(0.5 / n);
    L.c0 = (float)(-log2(Re) / n);
    L.bl = (float)(bn / LN2);
    L.Ip = (float)(p[6] * exp(bn));
    const double m = -bn / n;
    L.kX1 = (float)(m * q * cs);
    L.kX2 = (float)(-m * sn / q);
    L.kY1 = (float)(m * q * sn);
    L.kY2 = (float)(m * cs / q);
  }
  sc.status = 0;
}

// ---- forward pieces ----

__device__ __forceinline__ float sersic_fwd(const LightC& c, float X, float Y) {
  const float dx = X - c.xc, dy = Y - c.yc;
  const float xp = fmaf(c.cs, dx, c.sn * dy);
  const float yp = fmaf(c.cs, dy, -c.sn * dx);
  const float R2 = fmaxf(fmaf(c.q * xp, xp, c.iq * yp * yp), R_MIN2);
  const float p = ex2(fmaf(c.c1, lg2(R2), c.c0));
  return c.Ip * ex2(-c.bl * p);
}

// Horner sum E = sum_{n=1}^{N} cE[n-1] w^{n-1}, coefficients in float4 chunks.
__device__ __forceinline__ void horner1(const float4* __restrict__ cE, int nq, float wr, float wi,
                                        float& Er, float& Ei) {
  float er = 0.f, ei = 0.f;
  for (int k = nq - 1; k >= 0; --k) {
    const float4 c = cE[k];
#define GL_H1(cc)                                      \
  {                                                    \
    const float nr = fmaf(wr, er, fmaf(-wi, ei, cc));  \
    ei = fmaf(wr, ei, wi * er);                        \
    er = nr;                                           \
  }
    GL_H1(c.w) GL_H1(c.z) GL_H1(c.y) GL_H1(c.x)
#undef GL_H1
  }
  Er = er;
  Ei = ei;
}

// The same for E and the t-derivative sum together.
__device__ __forceinline__ void horner2(const float4* __restrict__ cE, const float4* __restrict__ cT,
                                        int nq, float wr, float wi, float& Er, float& Ei,
                                        float& Tr, float& Ti) {
  float er = 0.f, ei = 0.f, tr = 0.f, ti = 0.f;
  for (int k = nq - 1; k >= 0; --k) {
    const float4 c = cE[k];
    const float4 d = cT[k];
#define GL_H2(cc, dd)                                  \
  {                                                    \
    const float nr = fmaf(wr, er, fmaf(-wi, ei, cc));  \
    ei = fmaf(wr, ei, wi * er);                        \
    er = nr;                                           \
    const float mr = fmaf(wr, tr, fmaf(-wi, ti, dd));  \
    ti = fmaf(wr, ti, wi * tr);                        \
    tr = mr;                                           \
  }
    GL_H2(c.w, d.w) GL_H2(c.z, d.z) GL_H2(c.y, d.y) GL_H2(c.x, d.x)
#undef GL_H2
  }
  Er = er;
  Ei = ei;
  Tr = tr;
  Ti = ti;
}

// EPL deflection (world frame) at (x, y).
__device__ __forceinline__ void epl_alpha(const EplC& e, const float4* __restrict__ cE, int nq,
                                          float x, float y, float& ax, float& ay) {
  const float dx = x - e.xc, dy = y - e.yc;
  const float xp = fmaf(e.cs, dx, e.sn * dy);
  const float yp = fmaf(e.cs, dy, -e.sn * dx);
  const float R2 = fmaxf(fmaf(e.q2 * xp, xp, yp * yp), R_MIN2);
  const float ir = rsq(R2);
  const float cph = e.q * xp * ir, sph = yp * ir;
  const float wr = fmaf(cph, cph, -sph * sph), wi = 2.f * cph * sph;
  float Er, Ei;
  horner1(cE, nq, wr, wi, Er, Ei);
  const float zr = -e.f * wr, zi = -e.f * wi;
  const float Fr = 1.f + fmaf(zr, Er, -zi * Ei);
  const float Fi = fmaf(zr, Ei, zi * Er);
  const float A = e.CA * ex2(e.ht * lg2(R2));
  const float aLr = A * fmaf(cph, Fr, -sph * Fi);
  const float aLi = A * fmaf(cph, Fi, sph * Fr);
  ax = fmaf(e.cs, aLr, -e.sn * aLi);
  ay = fmaf(e.sn, aLr, e.cs * aLi);
}

// ---- adjoint pieces ----
// Native accumulators of a Sersic component (converted to parameter
// gradients once per sample): [0] sum uS, [1] sum uSp, [2] sum uSp log2 p,
// [3] sum uSp/R^2 (x'^2 - y'^2/q^2), [4] sum uSp/R^2 x'y',
// [5] sum uSp/R^2 x', [6] sum uSp/R^2 y'.
// Returns S; if grad_pos, adds dS/dX, dS/dY (without u) to gX, gY.
template <bool grad_pos>
__device__ __forceinline__ float sersic_adj(const LightC& c, float X, float Y, float u,
                                            float* __restrict__ a, float& gX, float& gY) {
  const float dx = X - c.xc, dy = Y - c.yc;
  const float xp = fmaf(c.cs, dx, c.sn * dy);
  const float yp = fmaf(c.cs, dy, -c.sn * dx);
  const float R2raw = fmaf(c.q * xp, xp, c.iq * yp * yp);
  const float R2 = fmaxf(R2raw, R_MIN2);
  const float l2p = fmaf(c.c1, lg2(R2), c.c0);
  const float p = ex2(l2p);
  const float S = c.Ip * ex2(-c.bl * p);
  const float Sp = S * p;
  // d R^2 / d(position) vanishes where the radius is clamped
  const float Dh = R2raw > R_MIN2 ? Sp * rcp(R2) : 0.f;
  const float uS = u * S, uSp = u * Sp, kD = u * Dh;
  a[0] += uS;
  a[1] += uSp;
  a[2] = fmaf(uSp, l2p, a[2]);
  a[3] = fmaf(kD, fmaf(xp, xp, -c.iq2 * yp * yp), a[3]);
  a[4] = fmaf(kD * xp, yp, a[4]);
  a[5] = fmaf(kD, xp, a[5]);
  a[6] = fmaf(kD, yp, a[6]);
  if (grad_pos) {
    gX = fmaf(Dh, fmaf(c.kX1, xp, c.kX2 * yp), gX);
    gY = fmaf(Dh, fmaf(c.kY1, xp, c.kY2 * yp), gY);
  }
  return S;
}

// Converts a Sersic component's native accumulators to gradients w.r.t.
// [R_e, n, e1, e2, x, y, I_e] (double precision, once per sample).
__device__ inline void sersic_finish(const double* p, const double* a, double* g) {
  const double Re = p[0], n = p[1], e1 = p[2], e2 = p[3], I = p[6];
  const double c = sqrt(e1 * e1 + e2 * e2);
  const double q = (1.0 - c) / (1.0 + c);
  const double phi = 0.5 * atan2(e2, e1);
  const double cs = cos(phi), sn = sin(phi);
  const double bn = 1.9992 * n - 0.3271;
  const double m = -bn / n;
  const double dI = a[0] / I;
  const double dRe = bn / (n * Re) * a[1];
  const double dn = -1.9992 * (a[1] - a[0]) + bn * LN2 / n * a[2];
  const double dq = 0.5 * m * a[3];
  const double dphi = m * (q - 1.0 / q) * a[4];
  const double Sx = m * q * a[5], Sy = m * a[6] / q;  // sum u dS/dx', sum u dS/dy'
  const double dxc = -(cs * Sx - sn * Sy);
  const double dyc = -(sn * Sx + cs * Sy);
  const double cc = c > 1e-30 ? c : 1e-30;
  const double dqdc = -2.0 / ((1.0 + c) * (1.0 + c));
  g[0] = dRe;
  g[1] = dn;
  g[2] = dq * dqdc * (e1 / cc) - dphi * e2 / (2.0 * cc * cc);
  g[3] = dq * dqdc * (e2 / cc) + dphi * e1 / (2.0 * cc * cc);
  g[4] = dxc;
  g[5] = dyc;
  g[6] = dI;
}

// EPL + shear native accumulators:
// [0] sum s1 (theta_E), [1] d/dt, [2] d/dq, [3] d/dphi, [4] sum v.d alpha/dx',
// [5] sum v.d alpha/dy' (lens frame; the centre gradient is minus these),
// [6] d/dg1, [7] d/dg2.
__device__ inline void epl_finish(const double* v, const double* a, double* g) {
  const double thetaE = v[0], t = v[1] - 1.0, e1 = v[2], e2 = v[3];
  const double c = sqrt(e1 * e1 + e2 * e2);
  const double phi = 0.5 * atan2(e2, e1);
  const double cs = cos(phi), sn = sin(phi);
  const double gxl = -a[4], gyl = -a[5];
  const double cc = c > 1e-30 ? c : 1e-30;
  const double dqdc = -2.0 / ((1.0 + c) * (1.0 + c));
  g[0] = t / thetaE * a[0];
  g[1] = a[1];
  g[2] = a[2] * dqdc * (e1 / cc) - a[3] * e2 / (2.0 * cc * cc);
  g[3] = a[2] * dqdc * (e2 / cc) + a[3] * e1 / (2.0 * cc * cc);
  g[4] = cs * gxl - sn * gyl;
  g[5] = sn * gxl + cs * gyl;
  g[6] = a[6];
  g[7] = a[7];
}

}  // namespace gl
