// Fused per-sample kernels of the lens log-posterior: one CTA per parameter
// vector. Phases (all in one launch, per CTA):
//   1  sub-pixel ray-shoot (EPL series + shear), lens and source Sersic light,
//      binned to pixels (each thread owns whole pixels: no atomics);
//   2  PSF convolution of the binned image, chi^2 against the data
//      (Kahan-compensated FP32 per thread, FP64 across threads);
//   3  (gradient only) g = sigma^-2 (d - m) correlated with the PSF (the
//      convolution's adjoint), times D^2/s^2;
//   4  (gradient only) sub-pixel adjoint: recompute the forward chain and
//      accumulate the native gradient sums in registers; block reduction; the
//      per-sample chain rule to the Eq. sim-dist parameters plus the prior.
// The binned image and g live in zero-padded buffers (dynamic shared memory
// when they fit, else a per-CTA slot of global scratch).
#pragma once

#include <type_traits>

#include "gl_subpixel.cuh"

namespace gl {

// ---------------------------------------------------------------- conv ----
// Correlation of a zero-padded buffer: out(i, j) = sum_{u,v} k[u][v] in(i+u, j+v),
// by a CTA of T threads.
// Each thread computes ROWS_STRIP outputs of one column; lanes own adjacent
// columns (conflict-free loads); taps are compile-time indices into the
// kernel's parameter block.
// RELOAD (parameter block in shared memory): the tap columns are a loop
// unrolled by 3, so a few columns of taps are live (fully unrolled, the
// compiler hoisted all K^2 shared-memory taps into registers and spilled).
template <int T, int K, bool CONV, bool RELOAD, class Epi>
__device__ __forceinline__ void correlate_fixed(const SysParams& sp, const float* in, Epi epi) {
  constexpr int RS = ROWS_STRIP;
  const int ny = sp.ny, nx = sp.nx, Wp = sp.Wp;
  const int nrb = (ny + RS - 1) / RS;
  const int total = nrb * nx;
  for (int s = threadIdx.x; s < total; s += T) {
    const int rb = s / nx;
    const int j = s - rb * nx;
    const int i0 = rb * RS;
    float acc[RS];
#pragma unroll
    for (int r = 0; r < RS; ++r) acc[r] = 0.f;
    const float* base = in + (size_t)i0 * Wp + j;
    auto column = [&](int v, const float* taps) {
      float col[RS + K - 1];
#pragma unroll
      for (int m = 0; m < RS + K - 1; ++m) col[m] = base[m * Wp + v];
#pragma unroll
      for (int u = 0; u < K; ++u) {
        const float kv = taps[u * K + v];
#pragma unroll
        for (int r = 0; r < RS; ++r) acc[r] = fmaf(kv, col[u + r], acc[r]);
      }
    };
    if constexpr (RELOAD) {
      const float* taps = CONV ? sp.kconv : sp.kcorr;
#pragma unroll 3
      for (int v = 0; v < K; ++v) column(v, taps);
    } else {
#pragma unroll
      for (int v = 0; v < K; ++v) column(v, CONV ? sp.kconv : sp.kcorr);
    }
#pragma unroll
    for (int r = 0; r < RS; ++r)
      if (i0 + r < ny) epi(i0 + r, j, acc[r]);
  }
}

template <int T, bool CONV, class Epi>
__device__ __forceinline__ void correlate_generic(const SysParams& sp, const float* in, Epi epi) {
  const int ny = sp.ny, nx = sp.nx, Wp = sp.Wp, ky = sp.ky, kx = sp.kx;
  for (int s = threadIdx.x; s < ny * nx; s += T) {
    const int i = s / nx;
    const int j = s - i * nx;
    float acc = 0.f;
    for (int u = 0; u < ky; ++u)
      for (int v = 0; v < kx; ++v)
        acc = fmaf(CONV ? sp.kconv[u * kx + v] : sp.kcorr[u * kx + v],
                   in[(size_t)(i + u) * Wp + j + v], acc);
    epi(i, j, acc);
  }
}

template <int T, bool CONV, bool RELOAD = false, class Epi>
__device__ __forceinline__ void correlate(const SysParams& sp, const float* in, Epi epi) {
  if (sp.ky == 11 && sp.kx == 11)
    correlate_fixed<T, 11, CONV, RELOAD>(sp, in, epi);
  else if (sp.ky == 21 && sp.kx == 21)
    correlate_fixed<T, 21, CONV, RELOAD>(sp, in, epi);
  else
    correlate_generic<T, CONV>(sp, in, epi);
}

// Zero the halo of a padded buffer (the interior is written by a phase).
// first_thread: the threads taking part start at this index (warp 0 may be busy);
// T threads in the CTA.
template <int T>
__device__ __forceinline__ void zero_halo(const SysParams& sp, float* buf, int first_thread) {
  const int Hp = sp.Hp, Wp = sp.Wp;
  const int t0 = (int)threadIdx.x - first_thread, nt = T - first_thread;
  if (t0 < 0) return;
  const int top = sp.cy * Wp;                        // rows [0, cy)
  const int bot0 = (sp.cy + sp.ny) * Wp, bot = Hp * Wp - bot0;  // rows [cy+ny, Hp)
  for (int k = t0; k < top; k += nt) buf[k] = 0.f;
  for (int k = t0; k < bot; k += nt) buf[bot0 + k] = 0.f;
  const int side = Wp - sp.nx;                       // halo columns per interior row
  if (side > 0) {
    for (int k = t0; k < sp.ny * side; k += nt) {
      const int r = k / side, c = k - r * side;
      const int col = c < sp.cx ? c : c + sp.nx;
      buf[(size_t)(r + sp.cy) * Wp + col] = 0.f;
    }
  }
}

// Pixel (i, j) walk for p = threadIdx.x + it * step without a division per step.
struct PixelWalk {
  int i, j, di, dj, nx;
  __device__ __forceinline__ PixelWalk(int nx_, int step) : nx(nx_) {
    i = (int)threadIdx.x / nx_;
    j = (int)threadIdx.x - i * nx_;
    di = step / nx_;
    dj = step - di * nx_;
  }
  __device__ __forceinline__ void next() {
    i += di;
    j += dj;
    if (j >= nx) { j -= nx; ++i; }
  }
};

// ---------------------------------------------------------- reductions ----
template <int NW>
__device__ __forceinline__ double block_sum_double(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < NW; ++k) s += red[k];
  return s;  // valid on thread 0
}

// ---------------------------------------------------------------- kernels ----
// Shared memory of a CTA of NW warps.
template <int NW>
struct AdjSums {
  float redP[NW][MAX_P];
  double gsum[MAX_P];
};
// Static shared memory of the kernels (static_smem_bytes() tells the host).
template <int NW>
struct SmemStatic {
  SampleC sc;
  FinishC fin[MAX_COMP + 1];
  double red[NW];
  AdjSums<NW> adj;
};

__device__ __forceinline__ void buffers(const SysParams& sp, float* dsm, bool two, float*& A,
                                        float*& Bf, int slot_index) {
  const size_t nbuf = ((size_t)sp.Hp * sp.Wp + 3) & ~(size_t)3;
  float* slot = sp.scratch ? sp.scratch + (size_t)slot_index * sp.slot_floats : nullptr;
  size_t soff = 0, goff = 0;
  if (sp.bufA_smem) { A = dsm; soff += nbuf; } else { A = slot; goff += nbuf; }
  Bf = nullptr;
  if (two) {
    if (sp.bufB_smem) Bf = dsm + soff; else Bf = slot + goff;
  }
}

// Phase 1: bin the sub-pixel surface brightness into the padded buffer A.
// Pixels go in the lanes of float2 pairs: four pixels per thread (p, p + T,
// p + 2T, p + 3T; two interleaved pairs) while all four exist, then pairs,
// where a missing second pixel repeats the first and is not written.
// eval4(x0, y0, x1, y1, sb0, sb1) and eval2(x, y) give the brightness at two
// pairs and at one pair of sub-pixel centres. T threads in the CTA.
template <int T, class Eval2>
__device__ __forceinline__ void bin_tail(const SysParams& sp, float* A, PixelWalk w0, int p,
                                         Eval2 eval2) {
  const int s = sp.s, npix = sp.ny * sp.nx, Wp = sp.Wp, cy = sp.cy, cx = sp.cx;
  const float2 D = f2(sp.D), scale = f2(sp.scale);
  for (; p < npix; p += 2 * T) {
    PixelWalk w1 = w0;
    w1.next();
    const bool v1 = p + T < npix;
    const int i1 = v1 ? w1.i : w0.i, j1 = v1 ? w1.j : w0.j;
    const float2 xj = make_float2((float)w0.j + sp.xg0, (float)j1 + sp.xg0);
    const float2 yi = make_float2((float)w0.i + sp.yg0, (float)i1 + sp.yg0);
    float2 acc = f2(0.f);
    for (int k = 0; k < s; ++k) {
      const float2 y = mul2(add2(yi, f2(sp.off[k])), D);
      for (int l = 0; l < s; ++l) {
        const float2 x = mul2(add2(xj, f2(sp.off[l])), D);
        acc = add2(acc, eval2(x, y));
      }
    }
    acc = mul2(acc, scale);
    A[(size_t)(w0.i + cy) * Wp + w0.j + cx] = acc.x;
    if (v1) A[(size_t)(w1.i + cy) * Wp + w1.j + cx] = acc.y;
    w0 = w1;
    w0.next();
  }
}

template <int T, class Eval4, class Eval2>
__device__ __forceinline__ void bin_loop(const SysParams& sp, float* A, Eval4 eval4, Eval2 eval2) {
  const int s = sp.s, npix = sp.ny * sp.nx, Wp = sp.Wp, cy = sp.cy, cx = sp.cx;
  const float2 D = f2(sp.D), scale = f2(sp.scale);
  PixelWalk w0(sp.nx, T);
  int p = threadIdx.x;
  for (; p + 3 * T < npix; p += 4 * T) {
    PixelWalk w1 = w0;
    w1.next();
    PixelWalk w2 = w1;
    w2.next();
    PixelWalk w3 = w2;
    w3.next();
    const float2 xj0 = make_float2((float)w0.j + sp.xg0, (float)w1.j + sp.xg0);
    const float2 yi0 = make_float2((float)w0.i + sp.yg0, (float)w1.i + sp.yg0);
    const float2 xj1 = make_float2((float)w2.j + sp.xg0, (float)w3.j + sp.xg0);
    const float2 yi1 = make_float2((float)w2.i + sp.yg0, (float)w3.i + sp.yg0);
    float2 acc0 = f2(0.f), acc1 = f2(0.f);
    for (int k = 0; k < s; ++k) {
      const float2 ok = f2(sp.off[k]);
      const float2 y0 = mul2(add2(yi0, ok), D), y1 = mul2(add2(yi1, ok), D);
      for (int l = 0; l < s; ++l) {
        const float2 ol = f2(sp.off[l]);
        const float2 x0 = mul2(add2(xj0, ol), D), x1 = mul2(add2(xj1, ol), D);
        float2 sb0, sb1;
        eval4(x0, y0, x1, y1, sb0, sb1);
        acc0 = add2(acc0, sb0);
        acc1 = add2(acc1, sb1);
      }
    }
    acc0 = mul2(acc0, scale);
    acc1 = mul2(acc1, scale);
    A[(size_t)(w0.i + cy) * Wp + w0.j + cx] = acc0.x;
    A[(size_t)(w1.i + cy) * Wp + w1.j + cx] = acc0.y;
    A[(size_t)(w2.i + cy) * Wp + w2.j + cx] = acc1.x;
    A[(size_t)(w3.i + cy) * Wp + w3.j + cx] = acc1.y;
    w0 = w3;
    w0.next();
  }
  bin_tail<T>(sp, A, w0, p, eval2);
}

// The same with six pixels per thread (three interleaved pairs) while all six
// exist: eval6(x, y, sb) gives the brightness at the three pairs x[k], y[k].
// More independent work per thread for the forward's MUFU/FP32 latency chain.
template <int T, class Eval6, class Eval2>
__device__ __forceinline__ void bin_loop6(const SysParams& sp, float* A, Eval6 eval6, Eval2 eval2) {
  const int s = sp.s, npix = sp.ny * sp.nx, Wp = sp.Wp, cy = sp.cy, cx = sp.cx;
  const float2 D = f2(sp.D), scale = f2(sp.scale);
  PixelWalk w0(sp.nx, T);
  int p = threadIdx.x;
  for (; p + 5 * T < npix; p += 6 * T) {
    int wi[6], wj[6];
    {
      PixelWalk t = w0;
#pragma unroll
      for (int m = 0; m < 6; ++m) {
        wi[m] = t.i;
        wj[m] = t.j;
        if (m < 5) t.next();
      }
      w0 = t;
    }
    float2 xj[3], yi[3], acc[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      xj[m] = make_float2((float)wj[2 * m] + sp.xg0, (float)wj[2 * m + 1] + sp.xg0);
      yi[m] = make_float2((float)wi[2 * m] + sp.yg0, (float)wi[2 * m + 1] + sp.yg0);
      acc[m] = f2(0.f);
    }
    for (int k = 0; k < s; ++k) {
      const float2 ok = f2(sp.off[k]);
      float2 y[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) y[m] = mul2(add2(yi[m], ok), D);
      for (int l = 0; l < s; ++l) {
        const float2 ol = f2(sp.off[l]);
        float2 x[3], sb[3];
#pragma unroll
        for (int m = 0; m < 3; ++m) x[m] = mul2(add2(xj[m], ol), D);
        eval6(x, y, sb);
#pragma unroll
        for (int m = 0; m < 3; ++m) acc[m] = add2(acc[m], sb[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      acc[m] = mul2(acc[m], scale);
      A[(size_t)(wi[2 * m] + cy) * Wp + wj[2 * m] + cx] = acc[m].x;
      A[(size_t)(wi[2 * m + 1] + cy) * Wp + wj[2 * m + 1] + cx] = acc[m].y;
    }
    w0.next();
  }
  bin_tail<T>(sp, A, w0, p, eval2);
}

// Phase 1 with NPR pixel pairs per thread in flight (2 or 3). Every pixel sums
// its sub-pixels in the same order whatever NPR is, so the binned image (and
// everything after it) does not depend on NPR.
template <int T, int NPR, int NL, int NS, bool TAB>
__device__ __forceinline__ void bin_pixels(const SysParams& sp, const SampleC& sc,
                                           const float4* tab, float* A) {
  if constexpr (NPR == 3) {
    bin_loop6<T>(
        sp, A,
        [&](const float2* x, const float2* y, float2* sb) {
          surface_brightness6<NL, NS, TAB>(reload(sc), tab, x, y, sb);
        },
        [&](float2 x, float2 y) { return surface_brightness2<NL, NS, TAB>(reload(sc), tab, x, y); });
    return;
  }
  bin_loop<T>(
      sp, A,
      [&](float2 x0, float2 y0, float2 x1, float2 y1, float2& sb0, float2& sb1) {
        surface_brightness4<NL, NS, TAB>(reload(sc), tab, x0, y0, x1, y1, sb0, sb1);
      },
      [&](float2 x, float2 y) { return surface_brightness2<NL, NS, TAB>(reload(sc), tab, x, y); });
}

// Phase 1 for the image of one light component c (a source when source is
// set): the same walk with only that component evaluated.
template <int T, bool TAB>
__device__ __forceinline__ void bin_component(const SysParams& sp, const SampleC& sc,
                                              const float4* tab, float* A, int c, bool source) {
  bin_loop<T>(
      sp, A,
      [&](float2 x0, float2 y0, float2 x1, float2 y1, float2& sb0, float2& sb1) {
        component_brightness4<TAB>(reload(sc), tab, c, source, x0, y0, x1, y1, sb0, sb1);
      },
      [&](float2 x, float2 y) {
        return component_brightness2<TAB>(reload(sc), tab, c, source, x, y);
      });
}

// Phase 4: sub-pixel adjoint over pixel pairs (p, p + T) in float2 lanes (a
// missing second pixel repeats the first with u = 0). Per-lane FP32 sums are
// flushed into the per-warp sums redP every FLUSH_IT pairs, which bounds the
// FP32 accumulation length (near the mode the gradient is a small difference
// of large sums).
template <int T, int NL, int NS, bool TAB>
__device__ __forceinline__ void adjoint_pixels(const SysParams& sp, const SampleC& sc,
                                               const float4* tab, const float* A,
                                               float (*redP)[MAX_P]) {
  constexpr int P = 8 + 7 * (NL + NS);
  constexpr int FLUSH_IT = 2;
  // float2 sums (one per lane) up to 22 parameters, else lane-summed floats
  using AccT = typename std::conditional<(P <= 22), float2, float>::type;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = sp.s, npix = sp.ny * sp.nx, Wp = sp.Wp, cy = sp.cy, cx = sp.cx;
  const float2 D = f2(sp.D);
  AccT acc[P];
#pragma unroll
  for (int k = 0; k < P; ++k) acc[k] = acc_zero<AccT>();
  const int iters = (npix + 2 * T - 1) / (2 * T);  // the same in every lane
  PixelWalk w0(sp.nx, T);
  for (int it = 0; it < iters; ++it) {
    const int p = threadIdx.x + 2 * it * T;
    PixelWalk w1 = w0;
    w1.next();
    if (p < npix) {
      const bool v1 = p + T < npix;
      const int i1 = v1 ? w1.i : w0.i, j1 = v1 ? w1.j : w0.j;
      const float u0 = A[(size_t)(w0.i + cy) * Wp + w0.j + cx];
      const float u1 = v1 ? A[(size_t)(i1 + cy) * Wp + j1 + cx] : 0.f;
      const float2 u = make_float2(u0, u1);
      const float2 xj = make_float2((float)w0.j + sp.xg0, (float)j1 + sp.xg0);
      const float2 yi = make_float2((float)w0.i + sp.yg0, (float)i1 + sp.yg0);
      for (int k = 0; k < s; ++k) {
        const float2 y = mul2(add2(yi, f2(sp.off[k])), D);
        for (int l = 0; l < s; ++l) {
          const float2 x = mul2(add2(xj, f2(sp.off[l])), D);
          subpixel_adjoint2<NL, NS, TAB, AccT>(reload(sc), tab, x, y, u, acc);
        }
      }
    }
    w0 = w1;
    w0.next();
    if ((it + 1) % FLUSH_IT == 0 || it + 1 == iters) {
      if constexpr (P <= 32) {
        // reduce-scatter over the warp: each xor step halves the values a
        // lane holds (it keeps the half its lane bit selects and adds the
        // partner's copy of it), so lane k ends with the warp sum of value k;
        // 31 shuffles for all P sums instead of 5 per sum
        float v[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = k < P ? acc_total(acc[k]) : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const bool up = (lane & o) != 0;
#pragma unroll
          for (int i = 0; i < o; ++i) {
            const float keep = up ? v[i + o] : v[i];
            const float give = up ? v[i] : v[i + o];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, give, o);
          }
        }
        if (lane < P) redP[warp][lane] += v[0];
#pragma unroll
        for (int k = 0; k < P; ++k) acc[k] = acc_zero<AccT>();
      } else {
#pragma unroll
        for (int k = 0; k < P; ++k) {
          float v = acc_total(acc[k]);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) redP[warp][k] += v;
          acc[k] = acc_zero<AccT>();
        }
      }
    }
  }
}

// The row's surrogate table into shared memory (when the row uses it).
template <int T, bool SURR>
__device__ __forceinline__ void load_table(const float4* src, const SampleC& sc, float4* tab) {
  if (SURR && sc.use_table) {
    for (int k = threadIdx.x; k < TABLE_ROW; k += T) tab[k] = src[k];
  }
  __syncthreads();
}

// A table build whose tensor-core wait ran out leaves the row's table NaN; the
// row's results are then NaN (NaN positions would otherwise be clamped to a
// finite radius by the fmax in the radius floor and give finite brightness).
template <bool SURR>
__device__ __forceinline__ bool table_failed(const SampleC& sc, const float4* tab) {
  return SURR && sc.use_table && isnan(tab[0].x);
}

// Forward: log p per row, or (img != nullptr) the model image per row.
template <int NL, int NS, bool SURR>
__global__ void __launch_bounds__(THREADS, 2)
k_forward(const __grid_constant__ SysParams sp, const float* __restrict__ theta, int B,
          float* __restrict__ logp, float* __restrict__ img) {
  extern __shared__ __align__(16) float dsm[];
  __shared__ SmemStatic<NWARPS> st;
  __shared__ float4 tab[SURR ? TABLE_ROW : 1];
  SampleC& sc = st.sc;
  const int b = blockIdx.x;
  if (b >= B) return;
  const bool want_img = img != nullptr;
  float *A, *Bf;
  buffers(sp, dsm, false, A, Bf, blockIdx.x);
  if (threadIdx.x < 32)
    stage_warp(sp, theta + (size_t)b * sp.P, sc, st.fin, !want_img);
  else
    zero_halo<THREADS>(sp, A, 32);
  __syncthreads();
  const int npix = sp.ny * sp.nx;
  if (sc.status != 0) {
    if (want_img) {
      for (int p = threadIdx.x; p < npix; p += THREADS) img[(size_t)b * npix + p] = __int_as_float(0x7fc00000);
    } else if (threadIdx.x == 0) {
      logp[b] = sc.status == 2 ? __int_as_float(0x7fc00000) : -__int_as_float(0x7f800000);
    }
    return;
  }
  load_table<THREADS, SURR>(sp.table + (size_t)blockIdx.x * TABLE_ROW, sc, tab);
  if (table_failed<SURR>(sc, tab)) {
    if (want_img) {
      for (int p = threadIdx.x; p < npix; p += THREADS) img[(size_t)b * npix + p] = __int_as_float(0x7fc00000);
    } else if (threadIdx.x == 0) {
      logp[b] = __int_as_float(0x7fc00000);
    }
    return;
  }
  if (SURR && sc.use_table)
    bin_pixels<THREADS, 3, NL, NS, true>(sp, sc, tab, A);
  else
    bin_pixels<THREADS, 3, NL, NS, false>(sp, sc, tab, A);
  __syncthreads();
  float csum = 0.f, ccomp = 0.f;
  float* out = want_img ? img + (size_t)b * npix : nullptr;
  correlate<THREADS, true>(sp, A, [&](int i, int j, float m) {
    const int idx = i * sp.nx + j;
    if (want_img) {
      out[idx] = m;
    } else {
      const float r = sp.data[idx] - m;
      const float y = fmaf(sp.w[idx] * r, r, -ccomp);
      const float t = csum + y;
      ccomp = (t - csum) - y;
      csum = t;
    }
  });
  if (want_img) return;
  const double chi2 = block_sum_double<NWARPS>((double)csum - (double)ccomp, st.red);
  if (threadIdx.x == 0) logp[b] = (float)(-0.5 * chi2 + sc.logprior);
}

// Model images of single light components (the linear intensity solve):
// each row has one component with non-zero intensity, and only that one is
// evaluated (a lens-light row needs no deflection). A row with none gives a
// zero image; a row outside the model domain or with a NaN gives NaN.
template <bool SURR>
__global__ void __launch_bounds__(THREADS, 2)
k_component_images(const __grid_constant__ SysParams sp, const float* __restrict__ theta, int B,
                   float* __restrict__ img) {
  extern __shared__ __align__(16) float dsm[];
  __shared__ SmemStatic<NWARPS> st;
  __shared__ float4 tab[SURR ? TABLE_ROW : 1];
  SampleC& sc = st.sc;
  const int b = blockIdx.x;
  if (b >= B) return;
  float *A, *Bf;
  buffers(sp, dsm, false, A, Bf, blockIdx.x);
  if (threadIdx.x < 32)
    stage_warp(sp, theta + (size_t)b * sp.P, sc, st.fin, false);
  else
    zero_halo<THREADS>(sp, A, 32);
  __syncthreads();
  const int npix = sp.ny * sp.nx;
  float* out = img + (size_t)b * npix;
  if (sc.status != 0) {
    for (int p = threadIdx.x; p < npix; p += THREADS) out[p] = __int_as_float(0x7fc00000);
    return;
  }
  int c = 0;
  for (int k = 0; k < sp.nL + sp.nS; ++k)
    if (sc.light[k].Ip.x != 0.f) {
      c = k;
      break;
    }
  const bool source = c >= sp.nL;
  load_table<THREADS, SURR>(sp.table + (size_t)blockIdx.x * TABLE_ROW, sc, tab);
  if (source && table_failed<SURR>(sc, tab)) {
    for (int p = threadIdx.x; p < npix; p += THREADS) out[p] = __int_as_float(0x7fc00000);
    return;
  }
  if (SURR && sc.use_table && source)
    bin_component<THREADS, true>(sp, sc, tab, A, c, source);
  else
    bin_component<THREADS, false>(sp, sc, tab, A, c, source);
  __syncthreads();
  correlate<THREADS, true>(sp, A, [&](int i, int j, float m) { out[i * sp.nx + j] = m; });
}

// Forward + adjoint of one row (all T threads of the CTA): log p and
// d log p / d theta of theta row th into *logp_out and grad_out[0..P).
// slot_index picks the CTA's global-scratch slot, table_row the row's table;
// NPR pixel pairs per thread in flight in phase 1 (2 or 3). STAGED: the
// caller has staged the row into st, zeroed the adjoint sums and, for a row
// that uses a table, written it into tab (the fused kernel); the image
// buffers' halos are then zeroed here.
// Ends with a block barrier, so a persistent CTA can start its next row.
template <int NL, int NS, bool SURR, bool MULTI, int T, int NPR, bool STAGED = false>
__device__ __forceinline__ void grad_row(const SysParams& sp, const float* __restrict__ th,
                                         float* __restrict__ logp_out,
                                         float* __restrict__ grad_out,
                                         const float4* __restrict__ table_row, int slot_index,
                                         float* dsm, SmemStatic<T / 32>& st, float4* tab) {
  constexpr int P = 8 + 7 * (NL + NS);
  constexpr int NW = T / 32;
  SampleC& sc = st.sc;
  float *A, *Bf;
  buffers(sp, dsm, true, A, Bf, slot_index);
  if constexpr (STAGED) {
    zero_halo<T>(sp, A, 0);
    zero_halo<T>(sp, Bf, 0);
  } else {
    if (threadIdx.x < 32) {
      stage_warp(sp, th, sc, st.fin, true);
    } else {
      zero_halo<T>(sp, A, 32);
      zero_halo<T>(sp, Bf, 32);
    }
    for (int k = threadIdx.x; k < NW * MAX_P; k += T) (&st.adj.redP[0][0])[k] = 0.f;
  }
  __syncthreads();
  if (sc.status != 0) {
    const float lv = sc.status == 2 ? __int_as_float(0x7fc00000) : -__int_as_float(0x7f800000);
    const float gv = sc.status == 2 ? __int_as_float(0x7fc00000) : 0.f;
    if (threadIdx.x == 0) *logp_out = lv;
    if (threadIdx.x < P) grad_out[threadIdx.x] = gv;
    __syncthreads();
    return;
  }
  if constexpr (!STAGED) load_table<T, SURR>(table_row, sc, tab);
  if (table_failed<SURR>(sc, tab)) {
    if (threadIdx.x == 0) *logp_out = __int_as_float(0x7fc00000);
    if (threadIdx.x < P) grad_out[threadIdx.x] = __int_as_float(0x7fc00000);
    __syncthreads();
    return;
  }
  const bool use_tab = SURR && sc.use_table;
  const int Wp = sp.Wp, cy = sp.cy, cx = sp.cx, nx = sp.nx;
  // phase 1
  if (use_tab)
    bin_pixels<T, NPR, NL, NS, true>(sp, sc, tab, A);
  else
    bin_pixels<T, NPR, NL, NS, false>(sp, sc, tab, A);
  __syncthreads();
  // phase 2
  float csum = 0.f, ccomp = 0.f;
  correlate<T, true, MULTI>(sp, A, [&](int i, int j, float m) {
    const int idx = i * nx + j;
    const float r = sp.data[idx] - m;
    const float wr = sp.w[idx] * r;
    const float y = fmaf(wr, r, -ccomp);
    const float t = csum + y;
    ccomp = (t - csum) - y;
    csum = t;
    Bf[(size_t)(i + cy) * Wp + j + cx] = wr;
  });
  const double chi2 = block_sum_double<NW>((double)csum - (double)ccomp, st.red);
  // (block_sum_double synchronised the block: phase 2 is complete)
  // phase 3
  const float scale = sp.scale;
  correlate<T, false, MULTI>(sp, Bf, [&](int i, int j, float g) {
    A[(size_t)(i + cy) * Wp + j + cx] = g * scale;
  });
  __syncthreads();
  // phase 4
  if (use_tab)
    adjoint_pixels<T, NL, NS, true>(sp, sc, tab, A, st.adj.redP);
  else
    adjoint_pixels<T, NL, NS, false>(sp, sc, tab, A, st.adj.redP);
  __syncthreads();
  if (threadIdx.x < P) {
    double v = 0.0;
    for (int w = 0; w < NW; ++w) v += (double)st.adj.redP[w][threadIdx.x];
    st.adj.gsum[threadIdx.x] = v;
  }
  __syncthreads();
  // chain rule to the parameters, one lane per component
  if (threadIdx.x <= NL + NS) {
    const int c = threadIdx.x;
    float g[8];
    if (c == 0) {
      epl_finish(st.fin[0], st.adj.gsum, g, use_tab);
#pragma unroll
      for (int k = 0; k < 8; ++k) grad_out[k] = g[k] + sc.dprior[k];
    } else {
      const int o = 8 + 7 * (c - 1);
      sersic_finish(st.fin[c], st.adj.gsum + o, g, c - 1 < NL);
#pragma unroll
      for (int k = 0; k < 7; ++k) grad_out[o + k] = g[k] + sc.dprior[o + k];
    }
  }
  if (threadIdx.x == 0) *logp_out = (float)(-0.5 * chi2 + sc.logprior);
  __syncthreads();
}

// Forward + adjoint: log p and d log p / d theta per row (one CTA per row).
template <int NL, int NS, bool SURR>
__global__ void __launch_bounds__(THREADS, 2)
k_grad(const __grid_constant__ SysParams sp, const float* __restrict__ theta, int B,
       float* __restrict__ logp, float* __restrict__ grad) {
  constexpr int P = 8 + 7 * (NL + NS);
  extern __shared__ __align__(16) float dsm[];
  __shared__ SmemStatic<NWARPS> st;
  __shared__ float4 tab[SURR ? TABLE_ROW : 1];
  const int b = blockIdx.x;
  if (b >= B) return;
  grad_row<NL, NS, SURR, false, THREADS, 3>(sp, theta + (size_t)b * P, logp + b,
                                            grad + (size_t)b * P,
                                            SURR ? sp.table + (size_t)b * TABLE_ROW : nullptr, b,
                                            dsm, st, tab);
}

// Persistent forward + adjoint over uneven multi-system batches: each CTA
// takes items from a global counter, heaviest first (the host sorts them by
// cost), and uses its own global-scratch slot. counter must be 0 at launch.
// Launch shape: T threads per CTA (128 or 256; 512/T CTAs per SM at 128
// registers a thread), NPR pixel pairs per thread in phase 1 (2 or 3).
template <int NL, int NS, bool SURR, int T, int NPR>
__global__ void __launch_bounds__(T, 512 / T)
k_grad_multi(const SysParams* __restrict__ systems, const MultiItem* __restrict__ items,
             int n_items, int* __restrict__ counter) {
  extern __shared__ __align__(16) float dsm[];
  __shared__ SmemStatic<T / 32> st;
  __shared__ float4 tab[SURR ? TABLE_ROW : 1];
  __shared__ int next;
  __shared__ SysParams sps;  // the item's parameter block
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(counter, 1);
    __syncthreads();
    const int it = next;
    if (it >= n_items) break;
    const MultiItem m = items[it];
    {
      const int* src = reinterpret_cast<const int*>(systems + m.sys);
      int* dst = reinterpret_cast<int*>(&sps);
      for (int k = threadIdx.x; k < (int)(sizeof(SysParams) / sizeof(int)); k += T)
        dst[k] = src[k];
    }
    __syncthreads();
    grad_row<NL, NS, SURR, true, T, NPR>(sps, m.theta, m.logp, m.grad, m.table, blockIdx.x, dsm,
                                         st, tab);
  }
}

}  // namespace gl
