// Learned EPL deflection surrogate: a 4 -> 64 -> 64 -> 64 -> 64 -> 2 SiLU MLP
// on BF16 tensor cores (mma.sync m16n8k16, FP32 accumulate), evaluated one
// 16-row tile per warp.
//
// Inputs (q, gamma, log(R/theta_E), vphi) are normalised to
//   x0 = (q - 0.75)/0.25, x1 = (gamma - 2)/0.3, x2 = log(R/theta_E)/2.3,
//   x3 = (vphi - pi)/pi,
// with vphi the angle of q x' + i y' in [0, 2 pi). The network predicts the
// hypergeometric factor F = 2F1(1, t/2; 2 - t/2; z), z = -f e^{2 i vphi}, beyond
// its first two series terms, with the factor z^3 taken out:
//   F = 1 + c1 z + c2 z^2 + z^3 y / OUT_SCALE,  c1 = t/(4-t),  c2 = c1 (2+t)/(6-t),
//   y ~ OUT_SCALE sum_{n>=3} c_n z^{n-3}   (complex y = y0 + i y1, |y| ~ 0.3-1.4).
// The network's error (set by BF16 rounding of its activations) is then
// multiplied by |z|^3 = f^3 <= 1/27 on q >= 0.5, and vanishes as q -> 1
// where F tends to its analytic terms.
//
// Fragment layouts (PTX mma.m16n8k16, g = lane/4, c = lane%4):
//   A 16x16: a0 (row g, cols 2c..2c+1), a1 (row g+8), a2 (row g, cols 2c+8..), a3 (row g+8, cols 2c+8..)
//   B 16x8 : b0 (rows 2c..2c+1, col g), b1 (rows 2c+8.., col g)
//   C 16x8 : c0,c1 (row g, cols 2c, 2c+1), c2,c3 (row g+8, cols 2c, 2c+1)
// The C tiles of columns 16k..16k+15 are exactly the A fragment of k-step k,
// so a layer's output feeds the next layer from registers.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace gl {
namespace mlp {

constexpr int H = 64;          // hidden width
constexpr int NIN = 4;         // inputs
constexpr int NOUT = 2;        // outputs
constexpr float OUT_SCALE = 4.f;
constexpr float PI_F = 3.14159265358979f;

// FP32 parameter vector (master weights), row-major W[out][in]:
constexpr int OFF_W1 = 0;                    // [64][4]
constexpr int OFF_B1 = OFF_W1 + H * NIN;     // [64]
constexpr int OFF_W2 = OFF_B1 + H;           // [64][64]
constexpr int OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H;
constexpr int OFF_B3 = OFF_W3 + H * H;
constexpr int OFF_W4 = OFF_B3 + H;
constexpr int OFF_B4 = OFF_W4 + H * H;
constexpr int OFF_W5 = OFF_B4 + H;           // [2][64]
constexpr int OFF_B5 = OFF_W5 + NOUT * H;    // [2]
constexpr int NPARAM = OFF_B5 + NOUT;        // 12930

// BF16 operand layouts packed from the FP32 parameters:
//   P1 [64][16]  W1 with inputs padded to 16
//   P2..P4 [64][64]
//   P5 [8][64]   W5 with outputs padded to 8
//   T2..T4 [64][64] transposes (W^T [in][out]) for the backward pass
//   T5 [64][16]  W5^T with outputs padded to 16
constexpr int BOFF_P1 = 0;
constexpr int BOFF_P2 = BOFF_P1 + H * 16;
constexpr int BOFF_P3 = BOFF_P2 + H * H;
constexpr int BOFF_P4 = BOFF_P3 + H * H;
constexpr int BOFF_P5 = BOFF_P4 + H * H;
constexpr int BOFF_T2 = BOFF_P5 + 8 * H;
constexpr int BOFF_T3 = BOFF_T2 + H * H;
constexpr int BOFF_T4 = BOFF_T3 + H * H;
constexpr int BOFF_T5 = BOFF_T4 + H * H;
constexpr int NBF16 = BOFF_T5 + H * 16;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// sigmoid by the MUFU exponential and reciprocal
__device__ __forceinline__ float sigm(float z) {
  float e, r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-1.4426950408889634f * z));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.f + e));
  return r;
}

// D[16 x 64] = A[16 x K] W^T with W [64][K] bf16 row-major (K = 16 * KSTEPS).
template <int KSTEPS>
__device__ __forceinline__ void layer_mma(const uint32_t (&a)[KSTEPS][4],
                                          const __nv_bfloat16* __restrict__ W, float (&d)[8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  constexpr int K = 16 * KSTEPS;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.f;
    const __nv_bfloat16* w = W + (nt * 8 + g) * K + 2 * c;
#pragma unroll
    for (int kk = 0; kk < KSTEPS; ++kk) {
      const uint32_t b0 = *reinterpret_cast<const uint32_t*>(w + kk * 16);
      const uint32_t b1 = *reinterpret_cast<const uint32_t*>(w + kk * 16 + 8);
      mma16816(d[nt], a[kk], b0, b1);
    }
  }
}

// Output layer: D[16 x 8] = A[16 x 64] P5^T (cols 0, 1 real).
__device__ __forceinline__ void out_mma(const uint32_t (&a)[4][4],
                                        const __nv_bfloat16* __restrict__ P5, float (&d)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  d[0] = d[1] = d[2] = d[3] = 0.f;
  const __nv_bfloat16* w = P5 + g * H + 2 * c;
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    const uint32_t b0 = *reinterpret_cast<const uint32_t*>(w + kk * 16);
    const uint32_t b1 = *reinterpret_cast<const uint32_t*>(w + kk * 16 + 8);
    mma16816(d, a[kk], b0, b1);
  }
}

// Input A fragment (K = 16, inputs in cols 0..3) for rows g and g+8.
__device__ __forceinline__ void input_frag(const float (&xg)[4], const float (&xg8)[4],
                                           uint32_t (&a)[1][4]) {
  const int c = threadIdx.x & 3;
  a[0][0] = c == 0 ? pack_bf16(xg[0], xg[1]) : (c == 1 ? pack_bf16(xg[2], xg[3]) : 0u);
  a[0][1] = c == 0 ? pack_bf16(xg8[0], xg8[1]) : (c == 1 ? pack_bf16(xg8[2], xg8[3]) : 0u);
  a[0][2] = 0u;
  a[0][3] = 0u;
}

// C tiles of a 64-wide layer -> A fragments for the next layer.
__device__ __forceinline__ void c_to_a(const float (&v)[8][4], uint32_t (&a)[4][4]) {
#pragma unroll
  for (int kk = 0; kk < 4; ++kk) {
    a[kk][0] = pack_bf16(v[2 * kk][0], v[2 * kk][1]);
    a[kk][1] = pack_bf16(v[2 * kk][2], v[2 * kk][3]);
    a[kk][2] = pack_bf16(v[2 * kk + 1][0], v[2 * kk + 1][1]);
    a[kk][3] = pack_bf16(v[2 * kk + 1][2], v[2 * kk + 1][3]);
  }
}

// bias + SiLU in place on C tiles; column of element j of tile nt: nt*8 + 2c + (j & 1)
__device__ __forceinline__ void bias_silu(float (&v)[8][4], const float* __restrict__ b) {
  const int c = threadIdx.x & 3;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float z = v[nt][j] + b[nt * 8 + 2 * c + (j & 1)];
      v[nt][j] = z * sigm(z);
    }
}

// Forward pass of one 16-row tile with one forward-mode tangent: (xg, xg8)
// are the normalised inputs of rows g and g+8, (tg, tg8) their tangents.
// Returns y (C layout of the output tile: cols 0, 1 real) and dy.
__device__ __forceinline__ void forward_jvp(const __nv_bfloat16* __restrict__ wb,
                                            const float* __restrict__ params,
                                            const float (&xg)[4], const float (&xg8)[4],
                                            const float (&tg)[4], const float (&tg8)[4],
                                            float (&y)[4], float (&dy)[4]) {
  const int c = threadIdx.x & 3;
  uint32_t a1[1][4], t1[1][4];
  input_frag(xg, xg8, a1);
  input_frag(tg, tg8, t1);
  float z[8][4], dz[8][4];
  layer_mma<1>(a1, wb + BOFF_P1, z);
  layer_mma<1>(t1, wb + BOFF_P1, dz);
  uint32_t a[4][4], t[4][4];
  const float* bias[4] = {params + OFF_B1, params + OFF_B2, params + OFF_B3, params + OFF_B4};
  const __nv_bfloat16* Wl[3] = {wb + BOFF_P2, wb + BOFF_P3, wb + BOFF_P4};
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    if (l > 0) {
      layer_mma<4>(a, Wl[l - 1], z);
      layer_mma<4>(t, Wl[l - 1], dz);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float zz = z[nt][j] + bias[l][nt * 8 + 2 * c + (j & 1)];
        const float s = sigm(zz);
        z[nt][j] = zz * s;
        dz[nt][j] *= s * (1.f + zz * (1.f - s));
      }
    c_to_a(z, a);
    c_to_a(dz, t);
  }
  out_mma(a, wb + BOFF_P5, y);
  out_mma(t, wb + BOFF_P5, dy);
  const float b0 = params[OFF_B5], b1 = params[OFF_B5 + 1];
  if (c == 0) {
    y[0] += b0;
    y[1] += b1;
    y[2] += b0;
    y[3] += b1;
  }
}

// Normalised network inputs.
__device__ __forceinline__ void features(float q, float gamma, float lr, float vphi, float (&x)[4]) {
  x[0] = (q - 0.75f) * 4.f;
  x[1] = (gamma - 2.f) * (1.f / 0.3f);
  x[2] = lr * (1.f / 2.3f);
  x[3] = (vphi - PI_F) * (1.f / PI_F);
}

// The analytic part 1 + c1 z + c2 z^2 and its derivatives w.r.t. vphi, q, t
// at fixed (the others); z = -f e^{2 i vphi}, f = (1 - q)/(1 + q).
struct Base {
  float Fr, Fi, Pr, Pi, Qr, Qi, Tr, Ti;  // F, dF/dvphi, dF/dq, dF/dt
};
__device__ __forceinline__ Base base_terms(float q, float t, float vphi) {
  float s2, c2;
  sincosf(2.f * vphi, &s2, &c2);
  const float f = (1.f - q) / (1.f + q);
  const float dfdq = -2.f / ((1.f + q) * (1.f + q));
  const float zr = -f * c2, zi = -f * s2;
  const float c1 = t / (4.f - t);
  const float k2 = (2.f + t) / (6.f - t);
  const float cc2 = c1 * k2;
  const float dc1 = 4.f / ((4.f - t) * (4.f - t));
  const float dc2 = dc1 * k2 + c1 * 8.f / ((6.f - t) * (6.f - t));
  const float z2r = zr * zr - zi * zi, z2i = 2.f * zr * zi;
  Base b;
  b.Fr = 1.f + c1 * zr + cc2 * z2r;
  b.Fi = c1 * zi + cc2 * z2i;
  // dF/dz = c1 + 2 c2 z; dz/dvphi = 2 i z; dz/dq = -e^{2i vphi} df/dq
  const float gr = c1 + 2.f * cc2 * zr, gi = 2.f * cc2 * zi;
  const float dzr = -2.f * zi, dzi = 2.f * zr;
  b.Pr = gr * dzr - gi * dzi;
  b.Pi = gr * dzi + gi * dzr;
  const float qzr = -c2 * dfdq, qzi = -s2 * dfdq;
  b.Qr = gr * qzr - gi * qzi;
  b.Qi = gr * qzi + gi * qzr;
  b.Tr = dc1 * zr + dc2 * z2r;
  b.Ti = dc1 * zi + dc2 * z2i;
  return b;
}

// F and its derivatives w.r.t. vphi, q, t from the analytic part b, the
// network output y (complex, y0 + i y1) and y's derivatives dy[0..2] w.r.t.
// (vphi, q, t): with u = -e^{2 i vphi} and z = f u,
//   F    = b + z^3 y / S
//   F_vp = b_vp + z^3 (6 i y + y_vp) / S              (dz/dvphi = 2 i z)
//   F_q  = b_q + u^3 (3 f^2 f'(q) y + f^3 y_q) / S     (dz/dq = u f'(q))
//   F_t  = b_t + z^3 y_t / S
__device__ __forceinline__ Base compose(const Base& b, float q, float vphi, const float (&y)[2],
                                        const float (&dy)[3][2]) {
  float s2, c2;
  sincosf(2.f * vphi, &s2, &c2);
  const float f = (1.f - q) / (1.f + q);
  const float dfdq = -2.f / ((1.f + q) * (1.f + q));
  const float ur = -c2, ui = -s2;
  const float u2r = ur * ur - ui * ui, u2i = 2.f * ur * ui;
  const float u3r = u2r * ur - u2i * ui, u3i = u2r * ui + u2i * ur;
  const float k3 = f * f * f * (1.f / OUT_SCALE), kq = 3.f * f * f * dfdq * (1.f / OUT_SCALE);
  const float zr = k3 * u3r, zi = k3 * u3i;  // z^3 / S
  Base o;
  o.Fr = b.Fr + (zr * y[0] - zi * y[1]);
  o.Fi = b.Fi + (zr * y[1] + zi * y[0]);
  const float pr = dy[0][0] - 6.f * y[1], pi = dy[0][1] + 6.f * y[0];  // 6 i y + y_vp
  o.Pr = b.Pr + (zr * pr - zi * pi);
  o.Pi = b.Pi + (zr * pi + zi * pr);
  const float qr = kq * y[0] + k3 * dy[1][0], qi = kq * y[1] + k3 * dy[1][1];
  o.Qr = b.Qr + (u3r * qr - u3i * qi);
  o.Qi = b.Qi + (u3r * qi + u3i * qr);
  o.Tr = b.Tr + (zr * dy[2][0] - zi * dy[2][1]);
  o.Ti = b.Ti + (zr * dy[2][1] + zi * dy[2][0]);
  return o;
}

}  // namespace mlp
}  // namespace gl
