// Paired FP32 evaluation of the sub-pixel forward model: two pixels per
// thread, one in each lane of a float2, so every FP32 operation is one paired
// instruction (fma/mul/add .f32x2 on sm_100+) and the FP32 work takes half the
// issue slots; MUFU operations stay per lane.
//
// Per-sample constants are kept in shared memory duplicated into both lanes
// ((v, v) pairs), with the negated ones precomputed, so that the pair code
// needs no broadcast moves and no negations; it produces -alpha directly.
// The arithmetic is the scalar path's (gl_model.cuh) operation for operation.
#pragma once

#include "gl_model.cuh"

namespace gl {

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 max2(float2 a, float b) {
  return make_float2(fmaxf(a.x, b), fmaxf(a.y, b));
}
__device__ __forceinline__ float2 ex2_2(float2 a) { return make_float2(ex2(a.x), ex2(a.y)); }
__device__ __forceinline__ float2 lg2_2(float2 a) { return make_float2(lg2(a.x), lg2(a.y)); }
__device__ __forceinline__ float2 rsq2(float2 a) { return make_float2(rsq(a.x), rsq(a.y)); }

// Duplicated per-sample constants (see LightC / EplC for the meanings).
struct LightC2 {
  float2 nxc, nyc, cs, sn, nsn, q, iq, c1, c0, nbl, Ip;
};
struct EplC2 {
  float2 nxc, nyc, cs, sn, ncs, nsn, q, q2, f, nf, ht, CA;
};
struct PairC {
  EplC2 epl;
  float2 omg1, opg1, ng2;  // 1 - g1, 1 + g1, -g2
  LightC2 light[MAX_COMP];
  float4 cE2[N_MAX / 2];  // (c_n, c_n, c_{n+1}, c_{n+1}) of the E series, n = 1, 3, ...
};

// pc through an index the compiler cannot see is zero: the constants are then
// read from shared memory where they are used instead of being hoisted out of
// the pixel loops into registers (and spilled).
__device__ __forceinline__ const PairC& reload(const PairC& pc) {
  int z;
  asm volatile("mov.b32 %0, 0;" : "=r"(z));
  return (&pc)[z];
}

// Fills PairC from SampleC (threads 0, 32.., 64..; no barrier inside).
__device__ __forceinline__ void fill_pair_consts(const SampleC& sc, int ncomp, PairC& pc) {
  const int t = threadIdx.x;
  if (t == 0) {
    const EplC& e = sc.epl;
    EplC2& E = pc.epl;
    E.nxc = f2(-e.xc); E.nyc = f2(-e.yc); E.cs = f2(e.cs); E.sn = f2(e.sn);
    E.ncs = f2(-e.cs); E.nsn = f2(-e.sn); E.q = f2(e.q); E.q2 = f2(e.q2);
    E.f = f2(e.f); E.nf = f2(-e.f); E.ht = f2(e.ht); E.CA = f2(e.CA);
    pc.omg1 = f2(1.f - sc.g1); pc.opg1 = f2(1.f + sc.g1); pc.ng2 = f2(-sc.g2);
  }
  if (t >= 32 && t < 32 + ncomp) {
    const LightC& L = sc.light[t - 32];
    LightC2& P = pc.light[t - 32];
    P.nxc = f2(-L.xc); P.nyc = f2(-L.yc); P.cs = f2(L.cs); P.sn = f2(L.sn); P.nsn = f2(-L.sn);
    P.q = f2(L.q); P.iq = f2(L.iq); P.c1 = f2(L.c1); P.c0 = f2(L.c0); P.nbl = f2(-L.bl);
    P.Ip = f2(L.Ip);
  }
  const float* ce = reinterpret_cast<const float*>(sc.cE);
  for (int k = t - 64; k >= 0 && k < 2 * sc.nq; k += THREADS - 64) {
    const float a = ce[2 * k], b = ce[2 * k + 1];
    pc.cE2[k] = make_float4(a, a, b, b);
  }
}

__device__ __forceinline__ float2 sersic_fwd2(const LightC2& c, float2 X, float2 Y) {
  const float2 dx = add2(X, c.nxc), dy = add2(Y, c.nyc);
  const float2 xp = fma2(c.cs, dx, mul2(c.sn, dy));
  const float2 yp = fma2(c.cs, dy, mul2(c.nsn, dx));
  const float2 R2 = max2(fma2(mul2(c.q, xp), xp, mul2(mul2(c.iq, yp), yp)), R_MIN2);
  const float2 p = ex2_2(fma2(c.c1, lg2_2(R2), c.c0));
  return mul2(c.Ip, ex2_2(mul2(c.nbl, p)));
}

// E = sum_{n=1}^{N} c_n w^{n-1} for two points (Horner, duplicated coefficients).
__device__ __forceinline__ void horner1_2(const float4* __restrict__ cE2, int nq, float2 wr,
                                          float2 wi, float2 nwi, float2& Er, float2& Ei) {
  float2 er = f2(0.f), ei = f2(0.f);
  for (int k = 2 * nq - 1; k >= 0; --k) {
    const float4 c = cE2[k];  // coefficients of terms 2k+2 (z, w) and 2k+1 (x, y)
    float2 nr = fma2(wr, er, fma2(nwi, ei, make_float2(c.z, c.w)));
    ei = fma2(wr, ei, mul2(wi, er));
    er = nr;
    nr = fma2(wr, er, fma2(nwi, ei, make_float2(c.x, c.y)));
    ei = fma2(wr, ei, mul2(wi, er));
    er = nr;
  }
  Er = er;
  Ei = ei;
}

// Lens-frame geometry of the EPL at two points.
struct EplPt2 {
  float2 R2, cph, sph, nsph, wr, wi, nwi;
};

__device__ __forceinline__ EplPt2 epl_geometry2(const EplC2& e, float2 x, float2 y) {
  EplPt2 g;
  const float2 dx = add2(x, e.nxc), dy = add2(y, e.nyc);
  const float2 xp = fma2(e.cs, dx, mul2(e.sn, dy));
  const float2 yp = fma2(e.cs, dy, mul2(e.nsn, dx));
  g.R2 = max2(fma2(mul2(e.q2, xp), xp, mul2(yp, yp)), R_MIN2);
  const float2 ir = rsq2(g.R2);
  g.cph = mul2(mul2(e.q, xp), ir);
  g.sph = mul2(yp, ir);
  g.nsph = mul2(f2(-1.f), g.sph);
  g.wr = fma2(g.cph, g.cph, mul2(g.nsph, g.sph));
  const float2 cs = mul2(g.cph, g.sph);
  g.wi = mul2(f2(2.f), cs);
  g.nwi = mul2(f2(-2.f), cs);
  return g;
}

// Minus the EPL deflection (world frame) from the geometry and E.
__device__ __forceinline__ void epl_nalpha2_finish(const EplC2& e, const EplPt2& g, float2 Er,
                                                   float2 Ei, float2& nax, float2& nay) {
  // z = -f w:  F = 1 + z E,  Fr = 1 - f (wr Er - wi Ei),  Fi = -f (wr Ei + wi Er)
  const float2 Fr = fma2(e.nf, fma2(g.wr, Er, mul2(g.nwi, Ei)), f2(1.f));
  const float2 Fi = mul2(e.nf, fma2(g.wr, Ei, mul2(g.wi, Er)));
  const float2 A = mul2(e.CA, ex2_2(mul2(e.ht, lg2_2(g.R2))));
  const float2 aLr = mul2(A, fma2(g.cph, Fr, mul2(g.nsph, Fi)));
  const float2 aLi = mul2(A, fma2(g.cph, Fi, mul2(g.sph, Fr)));
  nax = fma2(e.ncs, aLr, mul2(e.sn, aLi));   // -(cs aLr - sn aLi)
  nay = fma2(e.nsn, aLr, mul2(e.ncs, aLi));  // -(sn aLr + cs aLi)
}

// Two Horner chains (four points) interleaved, for instruction-level parallelism.
__device__ __forceinline__ void horner1_2x2(const float4* __restrict__ cE2, int nq,
                                            const EplPt2& g0, const EplPt2& g1, float2& Er0,
                                            float2& Ei0, float2& Er1, float2& Ei1) {
  float2 er0 = f2(0.f), ei0 = f2(0.f), er1 = f2(0.f), ei1 = f2(0.f);
  for (int k = 2 * nq - 1; k >= 0; --k) {
    const float4 c = cE2[k];
    const float2 chi = make_float2(c.z, c.w), clo = make_float2(c.x, c.y);
    float2 nr0 = fma2(g0.wr, er0, fma2(g0.nwi, ei0, chi));
    float2 nr1 = fma2(g1.wr, er1, fma2(g1.nwi, ei1, chi));
    ei0 = fma2(g0.wr, ei0, mul2(g0.wi, er0));
    ei1 = fma2(g1.wr, ei1, mul2(g1.wi, er1));
    er0 = nr0;
    er1 = nr1;
    nr0 = fma2(g0.wr, er0, fma2(g0.nwi, ei0, clo));
    nr1 = fma2(g1.wr, er1, fma2(g1.nwi, ei1, clo));
    ei0 = fma2(g0.wr, ei0, mul2(g0.wi, er0));
    ei1 = fma2(g1.wr, ei1, mul2(g1.wi, er1));
    er0 = nr0;
    er1 = nr1;
  }
  Er0 = er0; Ei0 = ei0; Er1 = er1; Ei1 = ei1;
}

// beta = theta - alpha - (g1 x + g2 y, g2 x - g1 y), from -alpha.
__device__ __forceinline__ void lens_equation2(const PairC& pc, float2 x, float2 y, float2 nax,
                                               float2 nay, float2& bx, float2& by) {
  bx = fma2(pc.omg1, x, fma2(pc.ng2, y, nax));
  by = fma2(pc.ng2, x, fma2(pc.opg1, y, nay));
}

template <int NL, int NS>
__device__ __forceinline__ float2 light_sum2(const PairC& pc, float2 x, float2 y, float2 bx,
                                             float2 by) {
  float2 sb = sersic_fwd2(pc.light[0], NL > 0 ? x : bx, NL > 0 ? y : by);
#pragma unroll
  for (int c = 1; c < NL; ++c) sb = add2(sb, sersic_fwd2(pc.light[c], x, y));
#pragma unroll
  for (int c = (NL > 0 ? 0 : 1); c < NS; ++c) sb = add2(sb, sersic_fwd2(pc.light[NL + c], bx, by));
  return sb;
}

// Surface brightness at two points (exact series).
template <int NL, int NS>
__device__ __forceinline__ float2 surface_brightness2(const PairC& pc, int nq, float2 x, float2 y) {
  const EplPt2 g = epl_geometry2(pc.epl, x, y);
  float2 Er, Ei, nax, nay, bx, by;
  horner1_2(pc.cE2, nq, g.wr, g.wi, g.nwi, Er, Ei);
  epl_nalpha2_finish(pc.epl, g, Er, Ei, nax, nay);
  lens_equation2(pc, x, y, nax, nay, bx, by);
  return light_sum2<NL, NS>(pc, x, y, bx, by);
}

// Surface brightness at four points (two pairs, interleaved).
template <int NL, int NS>
__device__ __forceinline__ void surface_brightness2x2(const PairC& pc, int nq, float2 x0, float2 y0,
                                                      float2 x1, float2 y1, float2& sb0,
                                                      float2& sb1) {
  const EplPt2 g0 = epl_geometry2(pc.epl, x0, y0);
  const EplPt2 g1 = epl_geometry2(pc.epl, x1, y1);
  float2 Er0, Ei0, Er1, Ei1;
  horner1_2x2(pc.cE2, nq, g0, g1, Er0, Ei0, Er1, Ei1);
  float2 nax, nay, bx, by;
  epl_nalpha2_finish(pc.epl, g0, Er0, Ei0, nax, nay);
  lens_equation2(pc, x0, y0, nax, nay, bx, by);
  sb0 = light_sum2<NL, NS>(pc, x0, y0, bx, by);
  epl_nalpha2_finish(pc.epl, g1, Er1, Ei1, nax, nay);
  lens_equation2(pc, x1, y1, nax, nay, bx, by);
  sb1 = light_sum2<NL, NS>(pc, x1, y1, bx, by);
}

}  // namespace gl
