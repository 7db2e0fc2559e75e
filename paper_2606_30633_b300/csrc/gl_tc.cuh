// The surrogate network on the 5th-generation tensor cores, per row of
// parameters: the building blocks (shared-memory operand layout, tcgen05 MMA
// and TMEM access, bounded mbarrier waits) and net_row, which evaluates the
// network at the 128 table nodes of one row with three forward-mode tangents
// and leaves each node's (F, dF/dpa, dF/dq, dF/dt). Used by the stand-alone
// table build (k_table_tc) and by the fused gradient kernel (k_grad_fused),
// which therefore build bit-identical tables.
//
// Per row, the 128 nodes are the M = 128 rows of every layer's MMA
// (tcgen05.mma kind::f16, BF16 operands in shared memory, FP32 accumulators in
// tensor memory), for the primal pass and the three tangents (d/dvphi, d/dq,
// d/dgamma) as four accumulators of 64 columns. One thread per node reads its
// accumulator row back (tcgen05.ld), applies bias and SiLU (and SiLU' to the
// tangents) and writes the next layer's BF16 operand (two warpgroups split
// the columns). Operands use the
// canonical K-major layout without swizzle: 8 x 16-byte core matrices,
// K-adjacent ones 128 B apart (LBO), row-group-adjacent ones K/8 x 128 B apart
// (SBO).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gl_internal.cuh"
#include "gl_mlp.cuh"

namespace gl {
namespace tc {

using namespace gl::mlp;

constexpr uint32_t TMEM_COLS = 256;     // 4 streams x 64 columns
constexpr int A0_BYTES = 128 * 16 * 2;  // layer-1 operand [128][16]
constexpr int A_BYTES = 128 * 64 * 2;   // hidden operands [128][64]
constexpr int W1_BYTES = 64 * 16 * 2;
constexpr int WH_BYTES = 64 * 64 * 2;
constexpr int W5_BYTES = 16 * 64 * 2;   // output layer padded to N = 16
constexpr int TB_W1 = 0;  // shared-memory byte offsets of the network's operands
constexpr int TB_WH = TB_W1 + W1_BYTES;
constexpr int TB_W5 = TB_WH + 3 * WH_BYTES;
constexpr int TB_A0 = TB_W5 + W5_BYTES;
constexpr int TB_A = TB_A0 + A0_BYTES;
constexpr int TB_NODE = TB_A + 4 * A_BYTES;
// the network's shared memory with its own node array (k_table_tc) and with
// the node array over the first hidden operand, free once the last layer's
// MMAs have completed (k_grad_fused)
constexpr int SMEM_BYTES = TB_NODE + TABLE_M * 2 * 16;
constexpr int NET_SMEM_BYTES = TB_NODE;
constexpr long long WAIT_LIMIT = 1ll << 22;
// accumulator columns a thread reads per tcgen05.ld in the layer epilogues
// (8: 92 registers in the table build, 16: 123 and 2 % slower)
constexpr int NET_CHUNK = 8;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of element (r, k) of an [R][K] BF16 operand.
__device__ __forceinline__ uint32_t core_off(int r, int k, int K) {
  return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor (no swizzle, base offset 0, version 1).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor, kind::f16: FP32 D, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(bar)));
}

// Bounded wait for the barrier's phase; false on timeout.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t phase) {
  uint32_t done = 0;
  for (long long it = 0; it < WAIT_LIMIT && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase));
  }
  return done != 0;
}

__device__ __forceinline__ void ld16(uint32_t addr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void ld8(uint32_t addr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(addr));
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void ld2(uint32_t addr, float (&v)[2]) {
  uint32_t r0, r1;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];"
               : "=r"(r0), "=r"(r1)
               : "r"(addr));
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
}

__device__ __forceinline__ void ldc(uint32_t addr, float (&v)[8]) { ld8(addr, v); }
__device__ __forceinline__ void ldc(uint32_t addr, float (&v)[16]) { ld16(addr, v); }

__device__ __forceinline__ void wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Operand writes by the threads are made visible to the tensor cores, and the
// accumulator reads finished, before thread 0 issues the next MMAs.
__device__ __forceinline__ void to_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Copies an [N][K] BF16 row-major matrix (rows >= n_src zero) into the operand
// layout, by the NTH threads of the CTA.
template <int NTH>
__device__ __forceinline__ void load_operand(unsigned char* dst, const __nv_bfloat16* __restrict__ src,
                                             int N, int K, int n_src) {
  for (int i = threadIdx.x; i < N * K; i += NTH) {
    const int n = i / K, k = i - n * K;
    *reinterpret_cast<__nv_bfloat16*>(dst + core_off(n, k, K)) =
        n < n_src ? src[n * K + k] : __float2bfloat16(0.f);
  }
}

// The network's weight operands into shared memory at sm (TB_* offsets):
// layers 1-4 from the packed image (wimg, the training kernel's layout of the
// same bytes), the output layer padded to N = 16 from the BF16 operands.
template <int NTH>
__device__ __forceinline__ void load_weights(unsigned char* sm, const unsigned char* __restrict__ wimg,
                                             const __nv_bfloat16* __restrict__ wb) {
  const uint4* src = reinterpret_cast<const uint4*>(wimg);
  uint4* dst = reinterpret_cast<uint4*>(sm + TB_W1);
#pragma unroll 4
  for (int k = threadIdx.x; k < TB_W5 / 16; k += NTH) dst[k] = src[k];
  load_operand<NTH>(sm + TB_W5, wb + BOFF_P5, 16, 64, 8);
}

// 8 consecutive BF16 values of row r at column k0 (a multiple of 8), one store.
__device__ __forceinline__ void put8(unsigned char* base, int r, int k0, int K, const float* v) {
  uint4 u;
  u.x = pack_bf16(v[0], v[1]);
  u.y = pack_bf16(v[2], v[3]);
  u.z = pack_bf16(v[4], v[5]);
  u.w = pack_bf16(v[6], v[7]);
  *reinterpret_cast<uint4*>(base + core_off(r, k0, K)) = u;
}

}  // namespace tc

// Node j of a table: pseudo-angle pa_j = 2j/TABLE_M and its angle vphi_j in
// [0, pi) (inverse of pa = 1 - cos/(|cos| + sin)), with d vphi/d pa = (|cos| + sin)^2.
__device__ __forceinline__ void table_node(int j, float& vphi, float& dvdpa) {
  const float pa = 2.f * j / TABLE_M;
  vphi = pa <= 1.f ? atan2f(pa, 1.f - pa) : mlp::PI_F - atan2f(2.f - pa, pa - 1.f);
  float s, c;
  sincosf(vphi, &s, &c);
  const float d = fabsf(c) + s;
  dvdpa = d * d;
}

// Writes a row's interval table from its node values (node j: (F, dF/dpa)
// and (dF/dq, dF/dt), complex, in shared memory). Interval j covers pa in
// [pa_j, pa_j + h), h = 2/TABLE_M, with local t = (pa - pa_j)/h, and holds
//   (a, b), (c, d):  F(t) = a + b t + c t^2 + d t^3, the cubic Hermite
//                    through nodes j and j+1 (the nodes are periodic);
//   G0, G1 - G0:     (dF/dq, dF/dt) at node j and its change to node j+1,
// stored as four arrays of TABLE_M float4 (lanes reading different intervals
// then hit different shared-memory banks). out is global or shared memory.
__device__ __forceinline__ void write_intervals(const float4 (*node)[2], float4* __restrict__ out) {
  const float h = 2.f / TABLE_M;
  for (int j = threadIdx.x; j < TABLE_M; j += blockDim.x) {
    const int k = (j + 1) & (TABLE_M - 1);
    const float4 n0 = node[j][0], n1 = node[k][0];
    const float ar = n0.x, ai = n0.y, br = h * n0.z, bi = h * n0.w;
    const float er = h * n1.z, ei = h * n1.w;  // h dF/dpa at node j+1
    const float dr = n1.x - n0.x, di = n1.y - n0.y;
    const float cr = 3.f * dr - 2.f * br - er, ci = 3.f * di - 2.f * bi - ei;
    const float d3r = br + er - 2.f * dr, d3i = bi + ei - 2.f * di;
    const float4 m0 = node[j][1], m1 = node[k][1];
    out[j] = make_float4(ar, ai, br, bi);
    out[TABLE_M + j] = make_float4(cr, ci, d3r, d3i);
    out[2 * TABLE_M + j] = m0;
    out[3 * TABLE_M + j] = make_float4(m1.x - m0.x, m1.y - m0.y, m1.z - m0.z, m1.w - m0.w);
  }
}

// The network at the 128 nodes of one row (EPL axis ratio q, slope gamma) with
// three forward-mode tangents: node j's (F, dv dF/dvphi) and (dF/dq, dF/dt)
// into node[j]; (vp, dv) is table_node(t mod 128), the same for every row. All NTH threads of the CTA call it. Thread t serves node
// t mod 128: with one warpgroup it does all 64 columns of the four streams in
// each layer epilogue, with two (NTH = 256) the first warpgroup does columns
// 0-31 and the second 32-63 (warps w and w + 4 reach the same TMEM lanes), so
// no accumulator is read twice. The first warpgroup alone writes the inputs and
// reads the output layer. The
// weights are in shared memory at sm (load_weights); tb is the CTA's
// 256-column TMEM allocation, bar an initialised mbarrier whose parity is
// phase. Returns false (the block's common decision) when a bounded wait ran
// out or forced is set: the commit of parity phase is then still outstanding
// and the caller drains it before freeing the tensor memory.
template <int NTH>
__device__ __forceinline__ bool net_row(const __nv_bfloat16* __restrict__ wb,
                                        const float* __restrict__ params, float q, float gamma,
                                        float vp, float dv, unsigned char* sm,
                                        float4 (*node)[2], uint32_t tb,
                                        uint64_t* bar, uint32_t& phase, bool forced) {
  using namespace tc;
  static_assert(NTH == 128 || NTH == 256, "one or two warpgroups");
  const int t = threadIdx.x, nd = t & 127;
  const bool worker = t < 128;  // the first warpgroup
  const uint32_t lane_addr = tb + ((uint32_t)(32 * ((t >> 5) & 3)) << 16);
  unsigned char* A0 = sm + TB_A0;
  unsigned char* A = sm + TB_A;
  const uint32_t a0 = smem_u32(A0), aa = smem_u32(A), w1 = smem_u32(sm + TB_W1);
  const uint32_t wh = smem_u32(sm + TB_WH), w5 = smem_u32(sm + TB_W5);
  // tangent seeds of the normalised inputs, rounded to BF16 like every operand
  const float seed[3] = {__bfloat162float(__float2bfloat16(1.f / PI_F)), 4.f,
                         __bfloat162float(__float2bfloat16(1.f / 0.3f))};
  const int seed_in[3] = {3, 0, 1};
  float x[4];
  features(q, gamma, 0.f, vp, x);
  if (worker) {
    const float v[8] = {x[0], x[1], x[2], x[3], 0.f, 0.f, 0.f, 0.f};
    const float zero[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    put8(A0, nd, 0, 16, v);
    put8(A0, nd, 8, 16, zero);
  }
  to_async();
  // layer 1 (primal only: the tangents' first pre-activations are W1 seed)
  if (t == 0) {
    mma(tb, sdesc(a0, 256), sdesc(w1, 256), idesc(128, 64), 0u);
    commit(bar);
  }
  for (int layer = 1; layer <= 5; ++layer) {
    // the decision is the block's (a thread leaving alone would desert a barrier)
    if (!__syncthreads_and(!forced && wait_phase(bar, phase))) return false;
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (layer == 5) break;
    // epilogue of layer `layer`: bias, SiLU, SiLU' on the tangents, BF16 operands
    const float* bias = params + (layer == 1 ? OFF_B1 : layer == 2 ? OFF_B2
                                                      : layer == 3 ? OFF_B3 : OFF_B4);
    constexpr int CW = 64 / (NTH / 128);  // columns per thread
    constexpr int CH = NET_CHUNK;         // columns per accumulator read
    const int cb = (t >> 7) * CW;
#pragma unroll 1
    for (int c0 = cb; c0 < cb + CW; c0 += CH) {
      // the global loads (biases, layer 1's tangent seeds) go out before the
      // accumulator reads, whose wait would otherwise hold them back
      float z[CH], d1[CH], d2[CH], d3[CH], bz[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) bz[j] = bias[c0 + j];
      if (layer == 1) {
#pragma unroll
        for (int j = 0; j < CH; ++j) {
          const __nv_bfloat16* wrow = wb + BOFF_P1 + (c0 + j) * 16;
          d1[j] = __bfloat162float(wrow[seed_in[0]]) * seed[0];
          d2[j] = __bfloat162float(wrow[seed_in[1]]) * seed[1];
          d3[j] = __bfloat162float(wrow[seed_in[2]]) * seed[2];
        }
      }
      ldc(lane_addr + c0, z);
      if (layer > 1) {
        ldc(lane_addr + 64 + c0, d1);
        ldc(lane_addr + 128 + c0, d2);
        ldc(lane_addr + 192 + c0, d3);
      }
      wait_ld();
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const float zz = z[j] + bz[j];
        const float sg = sigm(zz);
        const float dsl = sg * (1.f + zz * (1.f - sg));
        z[j] = zz * sg;
        d1[j] *= dsl;
        d2[j] *= dsl;
        d3[j] *= dsl;
      }
#pragma unroll
      for (int h = 0; h < CH; h += 8) {
        put8(A, nd, c0 + h, 64, z + h);
        put8(A + A_BYTES, nd, c0 + h, 64, d1 + h);
        put8(A + 2 * A_BYTES, nd, c0 + h, 64, d2 + h);
        put8(A + 3 * A_BYTES, nd, c0 + h, 64, d3 + h);
      }
    }
    to_async();
    if (t == 0) {
      const bool out = layer == 4;
      const uint32_t wl = out ? w5 : wh + (uint32_t)(layer - 1) * WH_BYTES;
      const uint32_t id = out ? idesc(128, 16) : idesc(128, 64);
      for (int s = 0; s < 4; ++s)
        for (int kk = 0; kk < 4; ++kk)
          mma(tb + 64u * s, sdesc(aa + s * A_BYTES + kk * 256, 1024), sdesc(wl + kk * 256, 1024),
              id, kk > 0 ? 1u : 0u);
      commit(bar);
    }
  }
  // output layer: y (primal) and the three tangents' dy, two columns each
  if (worker) {
    float y[2], dy[3][2];
    ld2(lane_addr, y);
    ld2(lane_addr + 64, dy[0]);
    ld2(lane_addr + 128, dy[1]);
    ld2(lane_addr + 192, dy[2]);
    wait_ld();
    y[0] += params[OFF_B5];
    y[1] += params[OFF_B5 + 1];
    const Base bt = compose(base_terms(q, gamma - 1.f, vp), q, vp, y, dy);
    node[nd][0] = make_float4(bt.Fr, bt.Fi, dv * bt.Pr, dv * bt.Pi);
    node[nd][1] = make_float4(bt.Qr, bt.Qi, bt.Tr, bt.Ti);
  }
  return true;
}

}  // namespace gl
