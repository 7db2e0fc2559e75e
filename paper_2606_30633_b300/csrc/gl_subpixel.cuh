// Sub-pixel evaluations of the lens model (forward surface brightness and its
// adjoint), two points at a time in the lanes of float2 values: every FP32
// operation is one paired instruction, which halves the issue slots of the
// FP32 work (the FP32 pipe's lane throughput is unchanged); MUFU operations
// and the table gathers stay per lane.
//
// Notation as in gl_model.cuh. The EPL deflection comes from the exact
// series (Horner in w over the staged coefficients) or, for rows that the
// surrogate covers, from the row's table (F and its derivatives).
#pragma once

#include "gl_model.cuh"

namespace gl {

// v through an index the compiler cannot see is zero: the constants are then
// read from shared memory where they are used instead of being hoisted out of
// the pixel loops into registers (and spilled).
template <class T>
__device__ __forceinline__ const T& reload(const T& v) {
  int z;
  asm volatile("mov.b32 %0, 0;" : "=r"(z));
  return (&v)[z];
}

// ------------------------------------------------------ EPL geometry ----
struct Geo2 {
  float2 xp, yp, R2, ir, cph, sph, nsph, wr, wi, nwi;
};

__device__ __forceinline__ Geo2 epl_geometry2(const EplP& e, float2 x, float2 y) {
  Geo2 g;
  const float2 dx = add2(x, e.nxc), dy = add2(y, e.nyc);
  g.xp = fma2(e.cs, dx, mul2(e.sn, dy));
  g.yp = fma2(e.cs, dy, mul2(e.nsn, dx));
  g.R2 = max2(fma2(mul2(e.q2, g.xp), g.xp, mul2(g.yp, g.yp)), R_MIN2);
  g.ir = rsq2(g.R2);
  g.cph = mul2(mul2(e.q, g.xp), g.ir);
  g.sph = mul2(g.yp, g.ir);
  g.nsph = neg2(g.sph);
  g.wr = fma2(g.cph, g.cph, mul2(g.nsph, g.sph));
  const float2 cs = mul2(g.cph, g.sph);
  g.wi = add2(cs, cs);
  g.nwi = neg2(g.wi);
  return g;
}

// ------------------------------------------------------ Horner sums ----
// One Horner step of e <- w e + c (complex w, real coefficient c).
__device__ __forceinline__ void horner_step(const Geo2& g, float2 c, float2& er, float2& ei) {
  const float2 nr = fma2(g.wr, er, fma2(g.nwi, ei, c));
  ei = fma2(g.wr, ei, mul2(g.wi, er));
  er = nr;
}

// E = sum_{n=1}^{4 nq} cE[n-1] w^{n-1} at two points.
__device__ __forceinline__ void horner_E(const float2* __restrict__ cE, int nq, const Geo2& g,
                                         float2& Er, float2& Ei) {
  const float4* c4 = reinterpret_cast<const float4*>(cE);
  float2 er = f2(0.f), ei = f2(0.f);
  for (int k = 2 * nq - 1; k >= 0; --k) {
    const float4 c = c4[k];  // terms 2k+2 (z, w) and 2k+1 (x, y)
    horner_step(g, make_float2(c.z, c.w), er, ei);
    horner_step(g, make_float2(c.x, c.y), er, ei);
  }
  Er = er;
  Ei = ei;
}

// The same at four points (two pairs interleaved for instruction-level parallelism).
__device__ __forceinline__ void horner_E2(const float2* __restrict__ cE, int nq, const Geo2& g0,
                                          const Geo2& g1, float2& Er0, float2& Ei0, float2& Er1,
                                          float2& Ei1) {
  const float4* c4 = reinterpret_cast<const float4*>(cE);
  float2 er0 = f2(0.f), ei0 = f2(0.f), er1 = f2(0.f), ei1 = f2(0.f);
  for (int k = 2 * nq - 1; k >= 0; --k) {
    const float4 c = c4[k];
    const float2 chi = make_float2(c.z, c.w), clo = make_float2(c.x, c.y);
    horner_step(g0, chi, er0, ei0);
    horner_step(g1, chi, er1, ei1);
    horner_step(g0, clo, er0, ei0);
    horner_step(g1, clo, er1, ei1);
  }
  Er0 = er0; Ei0 = ei0; Er1 = er1; Ei1 = ei1;
}

// E and the t-derivative sum T together.
__device__ __forceinline__ void horner_ET(const float2* __restrict__ cE,
                                          const float2* __restrict__ cT, int nq, const Geo2& g,
                                          float2& Er, float2& Ei, float2& Tr, float2& Ti) {
  const float4* c4 = reinterpret_cast<const float4*>(cE);
  const float4* d4 = reinterpret_cast<const float4*>(cT);
  float2 er = f2(0.f), ei = f2(0.f), tr = f2(0.f), ti = f2(0.f);
  for (int k = 2 * nq - 1; k >= 0; --k) {
    const float4 c = c4[k];
    const float4 d = d4[k];
    horner_step(g, make_float2(c.z, c.w), er, ei);
    horner_step(g, make_float2(d.z, d.w), tr, ti);
    horner_step(g, make_float2(c.x, c.y), er, ei);
    horner_step(g, make_float2(d.x, d.y), tr, ti);
  }
  Er = er; Ei = ei; Tr = tr; Ti = ti;
}

// ------------------------------------------------- surrogate table lookup ----
// Table of row b: TABLE_M nodes uniform in the pseudo-angle
//   pa = 1 - cos(vphi) / (|cos(vphi)| + sin(vphi)),  vphi folded into [0, pi)
// (F has period pi in vphi; pa is monotonic, in [0, 2), with
// d pa / d vphi = 1 / (|cos| + sin)^2), two float4 per node:
// (F, dF/dpa) and (dF/dq, dF/dt). Cubic Hermite interpolation in pa for F and
// its derivative, linear for the rest. One point (the gathers are per lane).
struct TabF {
  float Fr, Fi, Pr, Pi, Qr, Qi, Tr, Ti;  // F, dF/dvphi, dF/dq, dF/dt
};
template <bool DERIV>
__device__ __forceinline__ TabF table_eval(const float4* __restrict__ tab, float cph, float sph) {
  const float fl = sph < 0.f ? -1.f : 1.f;  // fold vphi into [0, pi)
  const float c = cph * fl, sn = sph * fl;
  const float rd = rcp(fmaxf(fabsf(c) + sn, 1e-20f));  // 0 only at the clamped centre
  const float pa = fmaf(-c, rd, 1.f);
  const float u = pa * (0.5f * TABLE_M);
  const int i0 = min((int)u, TABLE_M - 1);
  const float t = u - (float)i0;
  const int i1 = (i0 + 1) & (TABLE_M - 1);
  const float4 a0 = tab[2 * i0], a1 = tab[2 * i1];
  const float h = 2.f / TABLE_M;
  const float t2 = t * t, omt = 1.f - t;
  const float h00 = (1.f + 2.f * t) * omt * omt, h10 = t * omt * omt;
  const float h01 = t2 * (3.f - 2.f * t), h11 = t2 * (t - 1.f);
  TabF o;
  o.Fr = h00 * a0.x + h01 * a1.x + h * (h10 * a0.z + h11 * a1.z);
  o.Fi = h00 * a0.y + h01 * a1.y + h * (h10 * a0.w + h11 * a1.w);
  if (DERIV) {
    const float d00 = 6.f * (t2 - t) / h, d10 = 3.f * t2 - 4.f * t + 1.f, d11 = 3.f * t2 - 2.f * t;
    const float k = rd * rd;  // d pa / d vphi
    o.Pr = k * (d00 * (a0.x - a1.x) + d10 * a0.z + d11 * a1.z);
    o.Pi = k * (d00 * (a0.y - a1.y) + d10 * a0.w + d11 * a1.w);
    const float4 b0 = tab[2 * i0 + 1], b1 = tab[2 * i1 + 1];
    o.Qr = omt * b0.x + t * b1.x;
    o.Qi = omt * b0.y + t * b1.y;
    o.Tr = omt * b0.z + t * b1.z;
    o.Ti = omt * b0.w + t * b1.w;
  }
  return o;
}

// ------------------------------------------------------ forward pieces ----
// F = 1 + z E with z = -f w:  Fr = 1 - f (wr Er - wi Ei),  Fi = -f (wr Ei + wi Er).
__device__ __forceinline__ void series_F(const EplP& e, const Geo2& g, float2 Er, float2 Ei,
                                         float2& Fr, float2& Fi) {
  Fr = fma2(e.nf, fma2(g.wr, Er, mul2(g.nwi, Ei)), f2(1.f));
  Fi = mul2(e.nf, fma2(g.wr, Ei, mul2(g.wi, Er)));
}

// The source-plane position beta = theta - alpha - (g1 x + g2 y, g2 x - g1 y)
// from F (A e^{i vphi} F is the lens-frame deflection).
__device__ __forceinline__ void lens_equation2(const SampleC& sc, const Geo2& g, float2 x, float2 y,
                                               float2 Fr, float2 Fi, float2& bx, float2& by) {
  const EplP& e = sc.epl;
  const float2 A = mul2(e.CA, ex2_2(mul2(e.ht, lg2_2(g.R2))));
  const float2 aLr = mul2(A, fma2(g.cph, Fr, mul2(g.nsph, Fi)));
  const float2 aLi = mul2(A, fma2(g.cph, Fi, mul2(g.sph, Fr)));
  const float2 nax = fma2(e.ncs, aLr, mul2(e.sn, aLi));   // -(cs aLr - sn aLi)
  const float2 nay = fma2(e.nsn, aLr, mul2(e.ncs, aLi));  // -(sn aLr + cs aLi)
  bx = fma2(sc.omg1, x, fma2(sc.ng2, y, nax));
  by = fma2(sc.ng2, x, fma2(sc.opg1, y, nay));
}

__device__ __forceinline__ float2 sersic_fwd2(const LightP& c, float2 X, float2 Y) {
  const float2 dx = add2(X, c.nxc), dy = add2(Y, c.nyc);
  const float2 xp = fma2(c.cs, dx, mul2(c.sn, dy));
  const float2 yp = fma2(c.cs, dy, mul2(c.nsn, dx));
  const float2 R2 = max2(fma2(mul2(c.q, xp), xp, mul2(mul2(c.iq, yp), yp)), R_MIN2);
  const float2 p = ex2_2(fma2(c.c1, lg2_2(R2), c.c0));
  return mul2(c.Ip, ex2_2(mul2(c.nbl, p)));
}

// Lens light at theta plus sources at beta.
template <int NL, int NS>
__device__ __forceinline__ float2 light_sum2(const SampleC& sc, float2 x, float2 y, float2 bx,
                                             float2 by) {
  float2 sb = sersic_fwd2(sc.light[0], NL > 0 ? x : bx, NL > 0 ? y : by);
#pragma unroll
  for (int c = 1; c < NL; ++c) sb = add2(sb, sersic_fwd2(sc.light[c], x, y));
#pragma unroll
  for (int c = (NL > 0 ? 0 : 1); c < NS; ++c) sb = add2(sb, sersic_fwd2(sc.light[NL + c], bx, by));
  return sb;
}

template <bool TAB>
__device__ __forceinline__ void deflection_F(const SampleC& sc, const float4* tab, const Geo2& g,
                                             float2& Fr, float2& Fi) {
  if (TAB) {
    const TabF t0 = table_eval<false>(tab, g.cph.x, g.sph.x);
    const TabF t1 = table_eval<false>(tab, g.cph.y, g.sph.y);
    Fr = make_float2(t0.Fr, t1.Fr);
    Fi = make_float2(t0.Fi, t1.Fi);
  } else {
    float2 Er, Ei;
    horner_E(sc.cE, sc.nq, g, Er, Ei);
    series_F(sc.epl, g, Er, Ei, Fr, Fi);
  }
}

// Surface brightness at two points.
template <int NL, int NS, bool TAB>
__device__ __forceinline__ float2 surface_brightness2(const SampleC& sc, const float4* tab, float2 x,
                                                      float2 y) {
  const Geo2 g = epl_geometry2(sc.epl, x, y);
  float2 Fr, Fi, bx, by;
  deflection_F<TAB>(sc, tab, g, Fr, Fi);
  lens_equation2(sc, g, x, y, Fr, Fi, bx, by);
  return light_sum2<NL, NS>(sc, x, y, bx, by);
}

// Surface brightness at four points (two pairs; the series sums interleaved).
template <int NL, int NS, bool TAB>
__device__ __forceinline__ void surface_brightness4(const SampleC& sc, const float4* tab, float2 x0,
                                                    float2 y0, float2 x1, float2 y1, float2& sb0,
                                                    float2& sb1) {
  const Geo2 g0 = epl_geometry2(sc.epl, x0, y0);
  const Geo2 g1 = epl_geometry2(sc.epl, x1, y1);
  float2 Fr0, Fi0, Fr1, Fi1;
  if (TAB) {
    deflection_F<true>(sc, tab, g0, Fr0, Fi0);
    deflection_F<true>(sc, tab, g1, Fr1, Fi1);
  } else {
    float2 Er0, Ei0, Er1, Ei1;
    horner_E2(sc.cE, sc.nq, g0, g1, Er0, Ei0, Er1, Ei1);
    series_F(sc.epl, g0, Er0, Ei0, Fr0, Fi0);
    series_F(sc.epl, g1, Er1, Ei1, Fr1, Fi1);
  }
  float2 bx, by;
  lens_equation2(sc, g0, x0, y0, Fr0, Fi0, bx, by);
  sb0 = light_sum2<NL, NS>(sc, x0, y0, bx, by);
  lens_equation2(sc, g1, x1, y1, Fr1, Fi1, bx, by);
  sb1 = light_sum2<NL, NS>(sc, x1, y1, bx, by);
}

// ------------------------------------------------------ adjoint pieces ----
// Per-thread adjoint sums: a float2 (one sum per lane, added at the flush)
// where the registers allow, else a float that takes both lanes at once.
__device__ __forceinline__ void acc_add(float2& a, float2 v) { a = add2(a, v); }
__device__ __forceinline__ void acc_add(float& a, float2 v) { a += v.x + v.y; }
__device__ __forceinline__ void acc_fma(float2& a, float2 x, float2 y) { a = fma2(x, y, a); }
__device__ __forceinline__ void acc_fma(float& a, float2 x, float2 y) {
  a = fmaf(x.x, y.x, fmaf(x.y, y.y, a));
}
__device__ __forceinline__ float acc_total(float2 a) { return a.x + a.y; }
__device__ __forceinline__ float acc_total(float a) { return a; }
template <class AccT> __device__ __forceinline__ AccT acc_zero();
template <> __device__ __forceinline__ float2 acc_zero<float2>() { return f2(0.f); }
template <> __device__ __forceinline__ float acc_zero<float>() { return 0.f; }

// Native accumulators of a Sersic component (converted to parameter
// gradients once per sample): [0] sum uS, [1] sum uSp, [2] sum uSp log2 p,
// [3] sum uSp/R^2 (x'^2 - y'^2/q^2), [4] sum uSp/R^2 x'y',
// [5] sum uSp/R^2 x', [6] sum uSp/R^2 y' (one sum per lane).
// If grad_pos, adds dS/dX, dS/dY (without u) to gX, gY.
template <bool grad_pos, class AccT>
__device__ __forceinline__ void sersic_adj2(const LightP& c, float2 X, float2 Y, float2 u,
                                            AccT* __restrict__ a, float2& gX, float2& gY) {
  const float2 dx = add2(X, c.nxc), dy = add2(Y, c.nyc);
  const float2 xp = fma2(c.cs, dx, mul2(c.sn, dy));
  const float2 yp = fma2(c.cs, dy, mul2(c.nsn, dx));
  const float2 R2raw = fma2(mul2(c.q, xp), xp, mul2(mul2(c.iq, yp), yp));
  const float2 R2 = max2(R2raw, R_MIN2);
  const float2 l2p = fma2(c.c1, lg2_2(R2), c.c0);
  const float2 p = ex2_2(l2p);
  const float2 S = mul2(c.Ip, ex2_2(mul2(c.nbl, p)));
  const float2 Sp = mul2(S, p);
  // d R^2 / d(position) vanishes where the radius is clamped
  float2 Dh = mul2(Sp, rcp2(R2));
  Dh.x = R2raw.x > R_MIN2 ? Dh.x : 0.f;
  Dh.y = R2raw.y > R_MIN2 ? Dh.y : 0.f;
  const float2 uSp = mul2(u, Sp), kD = mul2(u, Dh);
  acc_fma(a[0], u, S);
  acc_add(a[1], uSp);
  acc_fma(a[2], uSp, l2p);
  acc_fma(a[3], kD, fma2(xp, xp, mul2(mul2(c.niq2, yp), yp)));
  acc_fma(a[4], mul2(kD, xp), yp);
  acc_fma(a[5], kD, xp);
  acc_fma(a[6], kD, yp);
  if (grad_pos) {
    gX = fma2(Dh, fma2(c.kX1, xp, mul2(c.kX2, yp)), gX);
    gY = fma2(Dh, fma2(c.kY1, xp, mul2(c.kY2, yp)), gY);
  }
}

// Adds u x d SB / d(native parameters) at two sub-pixels to acc (see
// epl_finish / sersic_finish for the accumulator meanings). EPL + shear:
// [0] theta_E, [1] d/dt, [2] d/dq, [3] rotation, [4], [5] lens-frame
// position, [6], [7] shear; then 7 per Sersic component.
template <int NL, int NS, bool TAB, class AccT>
__device__ __forceinline__ void subpixel_adjoint2(const SampleC& sc, const float4* tab, float2 x,
                                                  float2 y, float2 u, AccT* acc) {
  const EplP& e = sc.epl;
  const Geo2 g = epl_geometry2(e, x, y);
  const float2 iR2 = mul2(g.ir, g.ir);
  float2 Fr, Fi, Er, Ei, Tr, Ti, zr, zi, nzi;
  TabF t0, t1;
  if (TAB) {
    t0 = table_eval<true>(tab, g.cph.x, g.sph.x);
    t1 = table_eval<true>(tab, g.cph.y, g.sph.y);
    Fr = make_float2(t0.Fr, t1.Fr);
    Fi = make_float2(t0.Fi, t1.Fi);
  } else {
    horner_ET(sc.cE, sc.cT, sc.nq, g, Er, Ei, Tr, Ti);
    zr = mul2(e.nf, g.wr);
    zi = mul2(e.nf, g.wi);
    nzi = mul2(e.f, g.wi);
    Fr = fma2(zr, Er, fma2(nzi, Ei, f2(1.f)));
    Fi = fma2(zr, Ei, mul2(zi, Er));
  }
  const float2 Lm = lg2_2(g.R2);
  const float2 A = mul2(e.CA, ex2_2(mul2(e.ht, Lm)));
  const float2 Qr = mul2(A, g.cph), Qi = mul2(A, g.sph), nQi = mul2(A, g.nsph);  // A e^{i vphi}
  const float2 aLr = fma2(Qr, Fr, mul2(nQi, Fi));
  const float2 aLi = fma2(Qr, Fi, mul2(Qi, Fr));
  const float2 nax = fma2(e.ncs, aLr, mul2(e.sn, aLi));
  const float2 nay = fma2(e.nsn, aLr, mul2(e.ncs, aLi));
  const float2 bx = fma2(sc.omg1, x, fma2(sc.ng2, y, nax));
  const float2 by = fma2(sc.ng2, x, fma2(sc.opg1, y, nay));

  float2 gX = f2(0.f), gY = f2(0.f);
#pragma unroll
  for (int c = 0; c < NL; ++c) sersic_adj2<false>(sc.light[c], x, y, u, acc + 8 + 7 * c, gX, gY);
#pragma unroll
  for (int c = 0; c < NS; ++c)
    sersic_adj2<true>(sc.light[NL + c], bx, by, u, acc + 8 + 7 * (NL + c), gX, gY);
  // adjoint of the deflection: v = d logp / d alpha = -u grad_beta S
  const float2 nu = neg2(u);
  const float2 vx = mul2(nu, gX), vy = mul2(nu, gY), nvy = mul2(u, gY);
  acc_fma(acc[6], nvy, y);
  acc_fma(acc[6], vx, x);
  acc_fma(acc[7], vy, x);
  acc_fma(acc[7], vx, y);
  // lens frame
  const float2 vLx = fma2(e.cs, vx, mul2(e.sn, vy));
  const float2 vLy = fma2(e.cs, vy, mul2(e.nsn, vx));
  const float2 nvLx = neg2(vLx);
  const float2 s1 = fma2(vLx, aLr, mul2(vLy, aLi));    // v . alpha
  const float2 s1i = fma2(vLy, aLr, mul2(nvLx, aLi));  // v . (i alpha)
  const float2 lnbR = fma2(f2(-0.34657359027997264f), Lm, e.lnb);  // ln b - ln R
  const float2 dphq = mul2(mul2(g.xp, g.yp), neg2(iR2));           // d vphi / d ln q
  const float2 aq = fma2(mul2(mul2(e.omtq, g.xp), g.xp), iR2, e.a0);
  if (TAB) {
    // table derivatives at fixed (the other) arguments: dF/dvphi, dF/dq, dF/dt
    const float2 Pr = make_float2(t0.Pr, t1.Pr), Pi = make_float2(t0.Pi, t1.Pi);
    const float2 Qtr = make_float2(t0.Qr, t1.Qr), Qti = make_float2(t0.Qi, t1.Qi);
    const float2 Ttr = make_float2(t0.Tr, t1.Tr), Tti = make_float2(t0.Ti, t1.Ti);
    const float2 PFr = fma2(Qr, Pr, mul2(nQi, Pi)), PFi = fma2(Qr, Pi, mul2(Qi, Pr));
    const float2 QFr = fma2(Qr, Qtr, mul2(nQi, Qti)), QFi = fma2(Qr, Qti, mul2(Qi, Qtr));
    const float2 TFr = fma2(Qr, Ttr, mul2(nQi, Tti)), TFi = fma2(Qr, Tti, mul2(Qi, Ttr));
    const float2 S13 = add2(s1i, fma2(vLx, PFr, mul2(vLy, PFi)));
    const float2 sQ = fma2(vLx, QFr, mul2(vLy, QFi)), sT = fma2(vLx, TFr, mul2(vLy, TFi));
    acc_add(acc[0], s1);
    acc_add(acc[1], sT);
    acc_fma(acc[1], s1, lnbR);
    acc_add(acc[2], sQ);
    acc_fma(acc[2], S13, dphq);
    acc_fma(acc[2], s1, aq);
    const float2 Dx = mul2(iR2, fma2(mul2(e.omtq2, g.xp), s1, mul2(mul2(e.nq, g.yp), S13)));
    const float2 Dy = mul2(iR2, fma2(mul2(e.omt, g.yp), s1, mul2(mul2(e.q, g.xp), S13)));
    acc_add(acc[3], fma2(g.yp, Dx, fma2(neg2(g.xp), Dy, s1i)));  // d alpha/d phi
    acc_add(acc[4], Dx);
    acc_add(acc[5], Dy);
    return;
  }
  // dF/dt = z (Tr + i Ti)
  const float2 TFr = fma2(zr, Tr, mul2(nzi, Ti)), TFi = fma2(zr, Ti, mul2(zi, Tr));
  const float2 QTr = fma2(Qr, TFr, mul2(nQi, TFi)), QTi = fma2(Qr, TFi, mul2(Qi, TFr));
  const float2 sT = fma2(vLx, QTr, mul2(vLy, QTi));
  // F'(z) = [t F - (2-t) E] / (2 (1 - z))
  const float2 nr = fma2(e.t, Fr, mul2(e.ntmt, Er)), ni = fma2(e.t, Fi, mul2(e.ntmt, Ei));
  const float2 ozr = fma2(e.f, g.wr, f2(1.f));  // 1 - z = (ozr, -zi)
  const float2 inv = mul2(f2(0.5f), rcp2(fma2(ozr, ozr, mul2(zi, zi))));
  const float2 Fpr = mul2(fma2(nr, ozr, mul2(ni, nzi)), inv);
  const float2 Fpi = mul2(fma2(ni, ozr, mul2(nr, zi)), inv);
  const float2 P2r = fma2(Qr, Fpr, mul2(nQi, Fpi)), P2i = fma2(Qr, Fpi, mul2(Qi, Fpr));
  const float2 P3r = fma2(P2r, g.wr, mul2(P2i, g.nwi)), P3i = fma2(P2r, g.wi, mul2(P2i, g.wr));
  const float2 s3 = fma2(vLx, P3r, mul2(vLy, P3i));
  const float2 s3i = fma2(vLy, P3r, mul2(nvLx, P3i));
  const float2 S13 = fma2(e.m2f, s3i, s1i);
  acc_add(acc[0], s1);
  acc_add(acc[1], sT);
  acc_fma(acc[1], s1, lnbR);
  acc_fma(acc[2], e.ndfdq, s3);
  acc_fma(acc[2], S13, dphq);
  acc_fma(acc[2], s1, aq);
  // rotation: d alpha'/d phi = i X with X = (2-t) alpha' - 2 kappa z' =
  // -2 kappa f (z' w E + conj(z') F), which is O(f); acc[3] = sum kappa v.(iY)
  const float2 kap = mul2(mul2(e.Kk, A), g.ir);
  const float2 zwr = fma2(g.xp, g.wr, mul2(g.yp, g.nwi)), zwi = fma2(g.xp, g.wi, mul2(g.yp, g.wr));
  const float2 Yr = fma2(zwr, Er, fma2(neg2(zwi), Ei, fma2(g.xp, Fr, mul2(g.yp, Fi))));
  const float2 Yi = fma2(zwr, Ei, fma2(zwi, Er, fma2(g.xp, Fi, mul2(neg2(g.yp), Fr))));
  acc_fma(acc[3], kap, fma2(vLy, Yr, mul2(nvLx, Yi)));
  acc_fma(acc[4], iR2, fma2(mul2(e.omtq2, g.xp), s1, mul2(mul2(e.nq, g.yp), S13)));
  acc_fma(acc[5], iR2, fma2(mul2(e.omt, g.yp), s1, mul2(mul2(e.q, g.xp), S13)));
}

}  // namespace gl
