// Sub-pixel evaluations of the lens model (forward surface brightness and its
// adjoint), two points at a time in the lanes of float2 values: every FP32
// operation is one paired instruction, which halves the issue slots of the
// FP32 work (the FP32 pipe's lane throughput is unchanged); MUFU operations
// and the table gathers stay per lane.
//
// Notation as in gl_model.cuh. The EPL deflection comes from the exact
// series (Clenshaw's recurrence in w over the staged coefficients) or, for rows that the
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
// qx = q x' and yp = y' in the lens frame (R^2 = q^2 x'^2 + y'^2 = qx^2 + yp^2).
struct Geo2 {
  float2 qx, yp, R2, ir, cph, sph, nsph, wr, wi, nwi;
};

__device__ __forceinline__ Geo2 epl_geometry2(const EplP& e, float2 x, float2 y) {
  Geo2 g;
  const float2 dx = add2(x, e.nxc), dy = add2(y, e.nyc);
  g.qx = fma2(e.qcs, dx, mul2(e.qsn, dy));
  g.yp = fma2(e.cs, dy, mul2(e.nsn, dx));
  g.R2 = max2(fma2(g.qx, g.qx, mul2(g.yp, g.yp)), R_MIN2);
  g.ir = rsq2(g.R2);
  g.cph = mul2(g.qx, g.ir);
  g.sph = mul2(g.yp, g.ir);
  g.nsph = neg2(g.sph);
  g.wr = fma2(g.cph, g.cph, mul2(g.nsph, g.sph));
  const float2 cs = mul2(g.cph, g.sph);
  g.wi = add2(cs, cs);
  g.nwi = neg2(g.wi);
  return g;
}

// -------------------------------------------------- series summation ----
// The series are real-coefficient power series in w = e^{i theta} (theta =
// 2 vphi, |w| = 1), summed with Clenshaw's recurrence (Clenshaw 1955):
//   b_k = a_k + 2 cos(theta) b_{k+1} - b_{k+2},  b_M = b_{M+1} = 0,
//   sum_{k<M} a_k w^k = (b_0 - cos(theta) b_1) + i sin(theta) b_1,
// two operations per term where a complex Horner step takes four, and one
// FMA latency per term on the dependency chain. With a_k = c_{k+1}:
//   E = sum_{n>=1} c_n w^{n-1} = (b_0 - wr b_1, wi b_1),
//   w E = (wr b_0 - b_1, wi b_0)       (using |w|^2 = 1).
struct Clen2 {
  float2 b0, b1;
};

// One Clenshaw step: returns a + tw b1 - b2.
__device__ __forceinline__ float2 clen_step(float2 tw, float2 b1, float2 b2, float2 a) {
  return fma2(tw, b1, fma2(f2(-1.f), b2, a));
}

// The sum over the staged coefficients c[0 .. 2 n2) at two points.
__device__ __forceinline__ Clen2 clenshaw(const float2* __restrict__ c, int n2, const Geo2& g) {
  const float4* c4 = reinterpret_cast<const float4*>(c);
  const float2 tw = add2(g.wr, g.wr);
  float2 b1 = f2(0.f), b2 = f2(0.f);
#pragma unroll 2  // two chunks per trip: less loop overhead in the forward
  for (int k = n2 - 1; k >= 0; --k) {
    const float4 a = c4[k];  // a_{2k+1} in (z, w), a_{2k} in (x, y)
    const float2 bh = clen_step(tw, b1, b2, make_float2(a.z, a.w));
    const float2 bl = clen_step(tw, bh, b1, make_float2(a.x, a.y));
    b2 = bh;
    b1 = bl;
  }
  return Clen2{b1, b2};
}

// The same at four points (two pairs interleaved for instruction-level parallelism).
__device__ __forceinline__ void clenshaw2(const float2* __restrict__ c, int n2, const Geo2& g0,
                                          const Geo2& g1, Clen2& s0, Clen2& s1) {
  const float4* c4 = reinterpret_cast<const float4*>(c);
  const float2 tw0 = add2(g0.wr, g0.wr), tw1 = add2(g1.wr, g1.wr);
  float2 p1 = f2(0.f), p2 = f2(0.f), q1 = f2(0.f), q2 = f2(0.f);
#pragma unroll 2  // two chunks per trip: less loop overhead in the forward
  for (int k = n2 - 1; k >= 0; --k) {
    const float4 a = c4[k];
    const float2 ah = make_float2(a.z, a.w), al = make_float2(a.x, a.y);
    const float2 ph = clen_step(tw0, p1, p2, ah);
    const float2 qh = clen_step(tw1, q1, q2, ah);
    const float2 pl = clen_step(tw0, ph, p1, al);
    const float2 ql = clen_step(tw1, qh, q1, al);
    p2 = ph; p1 = pl;
    q2 = qh; q1 = ql;
  }
  s0 = Clen2{p1, p2};
  s1 = Clen2{q1, q2};
}

// The same at six points (three pairs interleaved).
__device__ __forceinline__ void clenshaw3(const float2* __restrict__ c, int n2, const Geo2* g,
                                          Clen2* out) {
  const float4* c4 = reinterpret_cast<const float4*>(c);
  float2 tw[3], b1[3], b2[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    tw[m] = add2(g[m].wr, g[m].wr);
    b1[m] = f2(0.f);
    b2[m] = f2(0.f);
  }
#pragma unroll 2  // two chunks per trip: less loop overhead in the forward
  for (int k = n2 - 1; k >= 0; --k) {
    const float4 a = c4[k];
    const float2 ah = make_float2(a.z, a.w), al = make_float2(a.x, a.y);
    float2 bh[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) bh[m] = clen_step(tw[m], b1[m], b2[m], ah);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const float2 bl = clen_step(tw[m], bh[m], b1[m], al);
      b2[m] = bh[m];
      b1[m] = bl;
    }
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) out[m] = Clen2{b1[m], b2[m]};
}

// E and the t-derivative sum T together.
__device__ __forceinline__ void clenshaw_ET(const float2* __restrict__ cE,
                                            const float2* __restrict__ cT, int n2, const Geo2& g,
                                            Clen2& sE, Clen2& sT) {
  const float4* c4 = reinterpret_cast<const float4*>(cE);
  const float4* d4 = reinterpret_cast<const float4*>(cT);
  const float2 tw = add2(g.wr, g.wr);
  float2 e1 = f2(0.f), e2 = f2(0.f), t1 = f2(0.f), t2 = f2(0.f);
  for (int k = n2 - 1; k >= 0; --k) {
    const float4 a = c4[k];
    const float4 d = d4[k];
    const float2 eh = clen_step(tw, e1, e2, make_float2(a.z, a.w));
    const float2 th = clen_step(tw, t1, t2, make_float2(d.z, d.w));
    const float2 el = clen_step(tw, eh, e1, make_float2(a.x, a.y));
    const float2 tl = clen_step(tw, th, t1, make_float2(d.x, d.y));
    e2 = eh; e1 = el;
    t2 = th; t1 = tl;
  }
  sE = Clen2{e1, e2};
  sT = Clen2{t1, t2};
}

// ------------------------------------------------- surrogate table lookup ----
// Table of row b: TABLE_M intervals uniform in the pseudo-angle
//   pa = 1 - cos(vphi) / (|cos(vphi)| + sin(vphi)),  vphi folded into [0, pi)
// (F has period pi in vphi; pa is monotonic, in [0, 2), with
// d pa / d vphi = 1 / (|cos| + sin)^2). Interval j holds four float4 (in
// four arrays of TABLE_M): the cubic F(t) = a + b t + c t^2 + d t^3 in the
// local coordinate t = pa TABLE_M/2 - j as (a, b), (c, d), then
// (dF/dq, dF/dt) at its start and their change across it (linear in t).
struct TabF {
  float Fr, Fi, Pr, Pi, Qr, Qi, Tr, Ti;  // F, dF/dvphi, dF/dq, dF/dt
};

template <bool DERIV>
__device__ __forceinline__ TabF table_interval(const float4* __restrict__ tab, int j, float t,
                                               float k) {
  const float4 p0 = tab[j], p1 = tab[TABLE_M + j];
  TabF o;
  o.Fr = fmaf(t, fmaf(t, fmaf(t, p1.z, p1.x), p0.z), p0.x);
  o.Fi = fmaf(t, fmaf(t, fmaf(t, p1.w, p1.y), p0.w), p0.y);
  if (DERIV) {
    // dF/dvphi = (b + 2c t + 3d t^2) (TABLE_M/2) (d pa / d vphi) = (...) k
    const float t3 = 3.f * t;
    o.Pr = k * fmaf(t, fmaf(t3, p1.z, p1.x + p1.x), p0.z);
    o.Pi = k * fmaf(t, fmaf(t3, p1.w, p1.y + p1.y), p0.w);
    const float4 g0 = tab[2 * TABLE_M + j], g1 = tab[3 * TABLE_M + j];
    o.Qr = fmaf(t, g1.x, g0.x);
    o.Qi = fmaf(t, g1.y, g0.y);
    o.Tr = fmaf(t, g1.z, g0.z);
    o.Ti = fmaf(t, g1.w, g0.w);
  }
  return o;
}

// Table values at two points (e^{i vphi} = cph + i sph per lane). The
// interval index comes from rounding in the float format: (u + 1/2) + 2^23
// holds round(u + 1/2) = floor(u) + 1 in its low mantissa bits (ties land on
// a neighbouring interval at t = 0 or 1, the same point; u = TABLE_M and a
// rounding below 0 wrap through the periodic table).
template <bool DERIV>
__device__ __forceinline__ void table_eval2(const float4* __restrict__ tab, const Geo2& g,
                                            TabF& o0, TabF& o1) {
  // fold vphi into [0, pi): nc = -cos, sn = |sin| of the folded angle
  const float2 nsgn = make_float2(g.sph.x < 0.f ? 1.f : -1.f, g.sph.y < 0.f ? 1.f : -1.f);
  const float2 nc = mul2(g.cph, nsgn);
  const float2 rd = make_float2(rcp(fmaxf(fabsf(nc.x) + fabsf(g.sph.x), 1e-20f)),
                                rcp(fmaxf(fabsf(nc.y) + fabsf(g.sph.y), 1e-20f)));
  constexpr float HM = 0.5f * TABLE_M;
  const float2 rdm = mul2(rd, f2(HM));
  const float2 u = fma2(nc, rdm, f2(HM));  // pa TABLE_M/2
  const float2 v = add2(add2(u, f2(0.5f)), f2(8388608.f));
  const float2 t = fma2(add2(v, f2(-8388609.f)), f2(-1.f), u);  // u - (floor(u))
  const int j0 = (__float_as_int(v.x) - 1) & (TABLE_M - 1);
  const int j1 = (__float_as_int(v.y) - 1) & (TABLE_M - 1);
  float2 k = f2(0.f);
  if (DERIV) k = mul2(rd, rdm);  // (TABLE_M/2) d pa / d vphi
  o0 = table_interval<DERIV>(tab, j0, t.x, k.x);
  o1 = table_interval<DERIV>(tab, j1, t.y, k.y);
}

// ------------------------------------------------------ forward pieces ----
// F = 1 + z E = 1 - f w E with z = -f w:  Fr = 1 - f (wr b_0 - b_1),  Fi = -f wi b_0.
__device__ __forceinline__ void series_F(const EplP& e, const Geo2& g, const Clen2& sE, float2& Fr,
                                         float2& Fi) {
  Fr = fma2(e.nf, fma2(g.wr, sE.b0, neg2(sE.b1)), f2(1.f));
  Fi = mul2(e.nf, mul2(g.wi, sE.b0));
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
  const float2 u = fma2(c.ucs, dx, mul2(c.usn, dy));
  const float2 v = fma2(c.vcs, dy, mul2(c.vnsn, dx));
  const float2 R2 = max2(fma2(u, u, mul2(v, v)), R_MIN2);
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
    TabF t0, t1;
    table_eval2<false>(tab, g, t0, t1);
    Fr = make_float2(t0.Fr, t1.Fr);
    Fi = make_float2(t0.Fi, t1.Fi);
  } else {
    series_F(sc.epl, g, clenshaw(sc.cE, sc.n2, g), Fr, Fi);
  }
}

// Brightness at two points whose light light(x, y, bx, by) depends on the
// image-plane position (x, y) and the lensed position (bx, by).
template <bool TAB, class Light>
__device__ __forceinline__ float2 lensed_brightness2(const SampleC& sc, const float4* tab, float2 x,
                                                     float2 y, Light light) {
  const Geo2 g = epl_geometry2(sc.epl, x, y);
  float2 Fr, Fi, bx, by;
  deflection_F<TAB>(sc, tab, g, Fr, Fi);
  lens_equation2(sc, g, x, y, Fr, Fi, bx, by);
  return light(x, y, bx, by);
}

// The same at four points (two pairs; the series sums interleaved).
template <bool TAB, class Light>
__device__ __forceinline__ void lensed_brightness4(const SampleC& sc, const float4* tab, float2 x0,
                                                   float2 y0, float2 x1, float2 y1, float2& sb0,
                                                   float2& sb1, Light light) {
  const Geo2 g0 = epl_geometry2(sc.epl, x0, y0);
  const Geo2 g1 = epl_geometry2(sc.epl, x1, y1);
  float2 Fr0, Fi0, Fr1, Fi1;
  if (TAB) {
    deflection_F<true>(sc, tab, g0, Fr0, Fi0);
    deflection_F<true>(sc, tab, g1, Fr1, Fi1);
  } else {
    Clen2 s0, s1;
    clenshaw2(sc.cE, sc.n2, g0, g1, s0, s1);
    series_F(sc.epl, g0, s0, Fr0, Fi0);
    series_F(sc.epl, g1, s1, Fr1, Fi1);
  }
  float2 bx, by;
  lens_equation2(sc, g0, x0, y0, Fr0, Fi0, bx, by);
  sb0 = light(x0, y0, bx, by);
  lens_equation2(sc, g1, x1, y1, Fr1, Fi1, bx, by);
  sb1 = light(x1, y1, bx, by);
}

// Surface brightness (lens light and sources) at two points.
template <int NL, int NS, bool TAB>
__device__ __forceinline__ float2 surface_brightness2(const SampleC& sc, const float4* tab, float2 x,
                                                      float2 y) {
  return lensed_brightness2<TAB>(sc, tab, x, y, [&](float2 px, float2 py, float2 bx, float2 by) {
    return light_sum2<NL, NS>(sc, px, py, bx, by);
  });
}

// The same at four points.
template <int NL, int NS, bool TAB>
__device__ __forceinline__ void surface_brightness4(const SampleC& sc, const float4* tab, float2 x0,
                                                    float2 y0, float2 x1, float2 y1, float2& sb0,
                                                    float2& sb1) {
  lensed_brightness4<TAB>(sc, tab, x0, y0, x1, y1, sb0, sb1,
                          [&](float2 px, float2 py, float2 bx, float2 by) {
                            return light_sum2<NL, NS>(sc, px, py, bx, by);
                          });
}

// The same at six points (three pairs x[m], y[m]; the series sums interleaved).
template <int NL, int NS, bool TAB>
__device__ __forceinline__ void surface_brightness6(const SampleC& sc, const float4* tab,
                                                    const float2* x, const float2* y, float2* sb) {
  Geo2 g[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) g[m] = epl_geometry2(sc.epl, x[m], y[m]);
  float2 Fr[3], Fi[3];
  if (TAB) {
#pragma unroll
    for (int m = 0; m < 3; ++m) deflection_F<true>(sc, tab, g[m], Fr[m], Fi[m]);
  } else {
    Clen2 cs[3];
    clenshaw3(sc.cE, sc.n2, g, cs);
#pragma unroll
    for (int m = 0; m < 3; ++m) series_F(sc.epl, g[m], cs[m], Fr[m], Fi[m]);
  }
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    float2 bx, by;
    lens_equation2(sc, g[m], x[m], y[m], Fr[m], Fi[m], bx, by);
    sb[m] = light_sum2<NL, NS>(sc, x[m], y[m], bx, by);
  }
}

// One light component at four points (two pairs): a lens-light component on
// the image plane, a source component at the lensed position (the only
// case that needs the deflection).
template <bool TAB>
__device__ __forceinline__ void component_brightness4(const SampleC& sc, const float4* tab, int c,
                                                      bool source, float2 x0, float2 y0, float2 x1,
                                                      float2 y1, float2& sb0, float2& sb1) {
  const LightP& L = sc.light[c];
  if (!source) {
    sb0 = sersic_fwd2(L, x0, y0);
    sb1 = sersic_fwd2(L, x1, y1);
    return;
  }
  lensed_brightness4<TAB>(sc, tab, x0, y0, x1, y1, sb0, sb1,
                          [&](float2, float2, float2 bx, float2 by) { return sersic_fwd2(L, bx, by); });
}

// The same at two points.
template <bool TAB>
__device__ __forceinline__ float2 component_brightness2(const SampleC& sc, const float4* tab, int c,
                                                        bool source, float2 x, float2 y) {
  const LightP& L = sc.light[c];
  if (!source) return sersic_fwd2(L, x, y);
  return lensed_brightness2<TAB>(sc, tab, x, y, [&](float2, float2, float2 bx, float2 by) {
    return sersic_fwd2(L, bx, by);
  });
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
// gradients once per sample), in the scaled frame us = sqrt(q) x',
// vs = y'/sqrt(q): [0] sum u Se (Se = S / (I_e e^{b_n})), [1] sum uSp, [2] sum uSp log2 p,
// [3] sum uSp/R^2 (us^2 - vs^2), [4] sum uSp/R^2 us vs,
// [5] sum uSp/R^2 us, [6] sum uSp/R^2 vs (one sum per lane); for a lens-light
// component [1..6] also hold S / (I_e e^{b_n}) in place of S.
// If grad_pos, adds dS/dX, dS/dY (without u) to gX, gY.
template <bool grad_pos, class AccT>
__device__ __forceinline__ void sersic_adj2(const LightP& c, float2 X, float2 Y, float2 u,
                                            AccT* __restrict__ a, float2& gX, float2& gY) {
  const float2 dx = add2(X, c.nxc), dy = add2(Y, c.nyc);
  const float2 us = fma2(c.ucs, dx, mul2(c.usn, dy));   // sqrt(q) x'
  const float2 vs = fma2(c.vcs, dy, mul2(c.vnsn, dx));  // y' / sqrt(q)
  const float2 R2raw = fma2(us, us, mul2(vs, vs));
  const float2 R2 = max2(R2raw, R_MIN2);
  const float2 l2p = fma2(c.c1, lg2_2(R2), c.c0);
  const float2 p = ex2_2(l2p);
  // Se: the profile without its amplitude I_e e^{b_n}. A lens-light component
  // (no position gradient) accumulates everything without the amplitude, which
  // sersic_finish applies per sample; a source keeps it, since its position
  // gradient feeds the deflection's adjoint. a[0] always sums u Se.
  const float2 Se = ex2_2(mul2(c.nbl, p));
  const float2 S = grad_pos ? mul2(c.Ip, Se) : Se;
  const float2 Sp = mul2(S, p);
  // d R^2 / d(position) vanishes where the radius is clamped
  float2 rR2 = rcp2(R2);
  rR2.x = R2raw.x > R_MIN2 ? rR2.x : 0.f;
  rR2.y = R2raw.y > R_MIN2 ? rR2.y : 0.f;
  const float2 uSp = mul2(u, Sp), kD = mul2(uSp, rR2);
  acc_fma(a[0], u, Se);
  acc_add(a[1], uSp);
  acc_fma(a[2], uSp, l2p);
  acc_fma(a[3], kD, fma2(us, us, mul2(neg2(vs), vs)));
  acc_fma(a[4], mul2(kD, us), vs);
  acc_fma(a[5], kD, us);
  acc_fma(a[6], kD, vs);
  if (grad_pos) {
    const float2 Dh = mul2(Sp, rR2);
    gX = fma2(Dh, fma2(c.kX1, us, mul2(c.kX2, vs)), gX);
    gY = fma2(Dh, fma2(c.kY1, us, mul2(c.kY2, vs)), gY);
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
  float2 Fr, Fi, Er, Ei, dtFr, dtFi;  // dtF = dF/dt
  TabF t0, t1;
  if (TAB) {
    table_eval2<true>(tab, g, t0, t1);
    Fr = make_float2(t0.Fr, t1.Fr);
    Fi = make_float2(t0.Fi, t1.Fi);
  } else {
    Clen2 sE, sT;
    clenshaw_ET(sc.cE, sc.cT, sc.n2, g, sE, sT);
    const float2 nwr = neg2(g.wr);
    Er = fma2(nwr, sE.b1, sE.b0);
    Ei = mul2(g.wi, sE.b1);
    Fr = fma2(e.f, fma2(nwr, sE.b0, sE.b1), f2(1.f));
    Fi = mul2(e.nf, mul2(g.wi, sE.b0));
    // dF/dt = z T = -f w T
    dtFr = mul2(e.f, fma2(nwr, sT.b0, sT.b1));
    dtFi = mul2(e.nf, mul2(g.wi, sT.b0));
  }
  const float2 Lm = lg2_2(g.R2);
  const float2 A = mul2(e.CA, ex2_2(mul2(e.ht, Lm)));
  const float2 Qr = mul2(A, g.cph), Qi = mul2(A, g.sph), nQi = neg2(Qi);  // A e^{i vphi}
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
  const float2 vx = mul2(nu, gX), vy = mul2(nu, gY), nvy = neg2(vy);
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
  // G = conj(vL) A e^{i vphi}: for any lens-frame factor X of the deflection,
  // v . (A e^{i vphi} X) = Re(G X) and v . (i A e^{i vphi} X) = -Im(G X)
  const float2 Gr = fma2(vLx, Qr, mul2(vLy, Qi)), Gi = fma2(vLx, Qi, mul2(neg2(vLy), Qr));
  const float2 nGi = neg2(Gi);
  const float2 lnbR = fma2(f2(-0.34657359027997264f), Lm, e.lnb);  // ln b - ln R
  const float2 xp = mul2(g.qx, e.iq);                               // x'
  const float2 xR = mul2(iR2, xp);
  // acc[2] (d/dq) takes S13 d vphi/d ln q + s1 ((1-t) q x'^2/R^2 + a0) with
  // d vphi/d ln q = -x'y'/R^2: x'/R^2 ((1-t) q x' s1 - y' S13) per sub-pixel;
  // the constant part a0 sum s1 = a0 acc[0] is added per sample (epl_finish)
  if (TAB) {
    // table derivatives at fixed (the other) arguments: dF/dvphi, dF/dq, dF/dt
    const float2 Pr = make_float2(t0.Pr, t1.Pr), Pi = make_float2(t0.Pi, t1.Pi);
    const float2 Qtr = make_float2(t0.Qr, t1.Qr), Qti = make_float2(t0.Qi, t1.Qi);
    const float2 Ttr = make_float2(t0.Tr, t1.Tr), Tti = make_float2(t0.Ti, t1.Ti);
    const float2 S13 = add2(s1i, fma2(Gr, Pr, mul2(nGi, Pi)));
    const float2 sQ = fma2(Gr, Qtr, mul2(nGi, Qti)), sT = fma2(Gr, Ttr, mul2(nGi, Tti));
    acc_add(acc[0], s1);
    acc_add(acc[1], sT);
    acc_fma(acc[1], s1, lnbR);
    acc_add(acc[2], sQ);
    const float2 yS = mul2(g.yp, S13);
    acc_fma(acc[2], xR, fma2(mul2(e.omtq, xp), s1, neg2(yS)));
    const float2 Dx = mul2(iR2, fma2(mul2(e.omtq, g.qx), s1, mul2(e.nq, yS)));
    const float2 Dy = mul2(iR2, fma2(mul2(e.omt, g.yp), s1, mul2(g.qx, S13)));
    acc_add(acc[3], fma2(g.yp, Dx, fma2(neg2(xp), Dy, s1i)));  // d alpha/d phi
    acc_add(acc[4], Dx);
    acc_add(acc[5], Dy);
    return;
  }
  const float2 sT = fma2(Gr, dtFr, mul2(nGi, dtFi));  // v . (A e^{i vphi} dF/dt)
  // H = F'(z) w with F'(z) = [t F - (2-t) E] / (2 (1 - z)), 1 - z = 1 + f w and
  // |w| = 1: H = n / (2 (conj(w) + f)), n = t F - (2-t) E
  const float2 nr = fma2(e.t, Fr, mul2(e.ntmt, Er)), ni = fma2(e.t, Fi, mul2(e.ntmt, Ei));
  // (the floor only acts at the clamped lens centre, where e^{i vphi} = 0 and G = 0)
  const float2 dr = add2(g.wr, e.f);  // conj(w) + f = (dr, -wi)
  const float2 inv = mul2(f2(0.5f), rcp2(max2(fma2(dr, dr, mul2(g.wi, g.wi)), 1e-30f)));
  const float2 Hr = mul2(fma2(nr, dr, mul2(ni, g.nwi)), inv);
  const float2 Hi = mul2(fma2(nr, g.wi, mul2(ni, dr)), inv);
  const float2 s3 = fma2(Gr, Hr, mul2(nGi, Hi));  // v . (A e^{i vphi} F' w)
  const float2 t3 = fma2(Gr, Hi, mul2(Gi, Hr));   // -v . (i A e^{i vphi} F' w)
  const float2 S13 = fma2(neg2(e.m2f), t3, s1i);
  acc_add(acc[0], s1);
  acc_add(acc[1], sT);
  acc_fma(acc[1], s1, lnbR);
  acc_fma(acc[2], e.ndfdq, s3);
  const float2 yS = mul2(g.yp, S13);
  acc_fma(acc[2], xR, fma2(mul2(e.omtq, xp), s1, neg2(yS)));
  // rotation: d alpha'/d phi = i X with X = (2-t) alpha' - 2 kappa z' =
  // -2 kappa f (z' w E + conj(z') F), which is O(f); acc[3] = sum (kappa/Kk) v.(iY)
  const float2 kap = mul2(A, g.ir);  // kappa / Kk, Kk = (2 - t)(1 + q)/4 applied per sample
  const float2 zwr = fma2(xp, g.wr, mul2(g.yp, g.nwi)), zwi = fma2(xp, g.wi, mul2(g.yp, g.wr));
  const float2 Yr = fma2(zwr, Er, fma2(neg2(zwi), Ei, fma2(xp, Fr, mul2(g.yp, Fi))));
  const float2 Yi = fma2(zwr, Ei, fma2(zwi, Er, fma2(xp, Fi, mul2(neg2(g.yp), Fr))));
  acc_fma(acc[3], kap, fma2(vLy, Yr, mul2(nvLx, Yi)));
  acc_fma(acc[4], iR2, fma2(mul2(e.omtq, g.qx), s1, mul2(e.nq, yS)));  // (1-t) q^2 x' = (1-t) q qx
  acc_fma(acc[5], iR2, fma2(mul2(e.omt, g.yp), s1, mul2(g.qx, S13)));
}

}  // namespace gl
