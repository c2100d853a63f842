// Nonlinear coefficient law and its learned surrogate (device side).
//
// The law (the nonlinear workload's constitutive relation; the paper's
// Section 2 allows coefficients c^Q that depend on old degrees of freedom):
//     k = 1 + 0.5 exp(-u^2) + 0.2 log(1 + k g),   g = |grad u|^2,
// solved by exactly 8 Newton steps from k0 = 1 + 0.5 exp(-u^2) on
//     F(k) = k - 1 - 0.5 exp(-u^2) - 0.2 log(1 + k g),  F'(k) = 1 - 0.2 g / (1 + k g)
// (F' >= 0.8 for k >= 1, so the root is unique).  D = k I at the point.
//
// Surrogate: a 2 -> H -> H -> 1 tanh network of (u, s = |grad u|), parameter
// layout W1[H][2], b1[H], W2[H][H], b2[H], W3[H], b3; inputs mapped onto
// [-1, 1]: x0 = a0 u + a1, x1 = c0 log s + c1 (the box [u0,u1] x [s0,s1]).
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

namespace fem {

constexpr int kMlpH = 64;
__host__ __device__ constexpr int mlp_nparams(int H) { return 2 * H + H + H * H + H + H + 1; }
constexpr int kMlpP = mlp_nparams(kMlpH);  // 4481

// iters: Newton steps (the law's 8; more only to make the law costlier when
// its cost is compared with the surrogate's)
template <class R>
__device__ __forceinline__ R law_exact(R u, R g, int iters = 8);

template <>
__device__ __forceinline__ float law_exact<float>(float u, float g, int iters) {
  const float e = 0.5f * expf(-u * u);
  float k = 1.f + e;
#pragma unroll 8
  for (int it = 0; it < iters; it++) {
    const float kg1 = 1.f + k * g;
    const float F = k - 1.f - e - 0.2f * logf(kg1);
    const float Fp = 1.f - 0.2f * g / kg1;
    k -= F / Fp;
  }
  return k;
}

template <>
__device__ __forceinline__ double law_exact<double>(double u, double g, int iters) {
  const double e = 0.5 * exp(-u * u);
  double k = 1.0 + e;
#pragma unroll 8
  for (int it = 0; it < iters; it++) {
    const double kg1 = 1.0 + k * g;
    const double F = k - 1.0 - e - 0.2 * log(kg1);
    const double Fp = 1.0 - 0.2 * g / kg1;
    k -= F / Fp;
  }
  return k;
}

// Input normalisation of the box (u0, u1, s0, s1) -> {a0, a1, c0, c1}.
__host__ __device__ inline void mlp_norm_from_box(const double *box, float *nrm) {
  const double du = box[1] - box[0];
  const double ls0 = log(box[2]), ls1 = log(box[3]);
  nrm[0] = (float)(2.0 / du);
  nrm[1] = (float)(-2.0 * box[0] / du - 1.0);
  nrm[2] = (float)(2.0 / (ls1 - ls0));
  nrm[3] = (float)(-2.0 * ls0 / (ls1 - ls0) - 1.0);
}

// Network output at (u, s); w: parameters (FP32 values, typically BF16-rounded).
__device__ __forceinline__ float mlp_eval(const float *w, const float *nrm, float u, float s) {
  constexpr int H = kMlpH;
  const float *W1 = w, *b1 = W1 + 2 * H, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H, *b3 = W3 + H;
  const float x0 = fmaf(u, nrm[0], nrm[1]), x1 = fmaf(logf(s), nrm[2], nrm[3]);
  float h1[H];
#pragma unroll
  for (int i = 0; i < H; i++) h1[i] = tanhf(fmaf(W1[2 * i], x0, fmaf(W1[2 * i + 1], x1, b1[i])));
  float y = b3[0];
#pragma unroll 2
  for (int i = 0; i < H; i++) {
    float a = b2[i];
#pragma unroll
    for (int j = 0; j < H; j++) a = fmaf(W2[i * H + j], h1[j], a);
    y = fmaf(W3[i], tanhf(a), y);
  }
  return y;
}

// tanh from the identity tanh(x) = 1 - 2 / (exp(2x) + 1), with the exponential
// as exp2 of 2 x / ln 2 (hardware ex2.approx) and the reciprocal from
// rcp.approx: absolute error about 2^-22, and exactly +-1 where exp(2x)
// overflows or underflows.
__device__ __forceinline__ float tanh_fast(float x) {
  float e, r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(x * 2.8853900817779268f));  // 2 / ln 2
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.f + e));
  return fmaf(-2.f, r, 1.f);
}

// tanh as the single hardware approximation tanh.approx.f32 (one MUFU
// operation instead of two; a larger error than tanh_fast, measured against
// the oracle's network in the tests)
__device__ __forceinline__ float tanh_hw(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// D (16x8, FP32) += A (16x16, BF16, row-major) * B (16x8, BF16, column-major),
// one warp (PTX mma.sync m16n8k16; fragment layout of the PTX ISA).
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// x = hi + lo for two values, each half a BF16 pair (first value in the low half).
__device__ __forceinline__ uint32_t bf16x2_split(float x0, float x1, uint32_t &lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  lo = *reinterpret_cast<const uint32_t *>(&l);
  return *reinterpret_cast<const uint32_t *>(&h);
}

// Network layout inside a law kernel's shared memory: FP32 W1[H][2], b1[H],
// b2[H], W3[H], b3 (kMlpSmall floats, padded), then W2 as BF16 rows of
// kW2Stride values (padded so that the B fragments of a warp hit 32 distinct banks).
constexpr int kMlpSmall = 2 * kMlpH + 3 * kMlpH + 4;  // 324
constexpr int kW2Stride = kMlpH + 8;                  // 72 BF16 values per row
constexpr int kMlpSmemBytes = kMlpSmall * 4 + kMlpH * kW2Stride * 2;

// Network output for npts points, 16 points per warp tile on the tensor
// cores: layer 1 (2 -> 64) and the tanh on CUDA cores, the 64 x 64 layer as
// BF16 MMAs with the activations split hi + lo (the weights are BF16 values,
// so hi*W + lo*W keeps about 16 bits of the activations) and FP32
// accumulation, then tanh and the 64 -> 1 layer.  xin: normalised inputs
// [npts][2]; pending(p) -> whether point p uses the network; apply(p, k)
// consumes its output.  warp / nwarp: this warp's index among the nwarp
// whole warps that share the points (negative: all whole warps of the block).
// hw: tanh from tanh_hw instead of tanh_fast.
template <class Pending, class Apply>
__device__ __forceinline__ void mlp_points_mma(const float *sp, const uint32_t *w2, const float *xin, int npts,
                                               Pending pending, Apply apply, int warp = -1, int nwarp = 0,
                                               bool hw = false) {
  auto act = [hw](float x) { return hw ? tanh_hw(x) : tanh_fast(x); };
  constexpr int H = kMlpH;
  const float *W1 = sp, *b1 = W1 + 2 * H, *b2 = b1 + H, *W3 = b2 + H;
  const float b3 = W3[H];
  const int lane = threadIdx.x & 31;
  if (warp < 0) {
    warp = threadIdx.x >> 5;
    nwarp = blockDim.x >> 5;
    if (warp >= nwarp) return;  // the trailing partial warp of a block
  }
  const int g = lane >> 2, t4 = lane & 3;
  const int nmt = (npts + 15) / 16;
  for (int mt = warp; mt < nmt; mt += nwarp) {
    const int p0 = mt * 16 + g, p1 = p0 + 8;
    if (!__any_sync(0xffffffffu, (p0 < npts && pending(p0)) || (p1 < npts && pending(p1)))) continue;
    const float x00 = p0 < npts ? xin[2 * p0] : 0.f, x01 = p0 < npts ? xin[2 * p0 + 1] : 0.f;
    const float x10 = p1 < npts ? xin[2 * p1] : 0.f, x11 = p1 < npts ? xin[2 * p1 + 1] : 0.f;
    uint32_t ah[4][4], al[4][4];
#pragma unroll
    for (int ks = 0; ks < 4; ks++)
#pragma unroll
      for (int hh = 0; hh < 2; hh++) {
        const int n = ks * 16 + hh * 8 + 2 * t4;  // neurons n, n + 1 (K columns of the A fragment)
        const float wa0 = W1[2 * n], wa1 = W1[2 * n + 1], wb0 = W1[2 * n + 2], wb1 = W1[2 * n + 3];
        const float ca = b1[n], cb = b1[n + 1];
        const float h00 = act(fmaf(wa0, x00, fmaf(wa1, x01, ca)));
        const float h01 = act(fmaf(wb0, x00, fmaf(wb1, x01, cb)));
        const float h10 = act(fmaf(wa0, x10, fmaf(wa1, x11, ca)));
        const float h11 = act(fmaf(wb0, x10, fmaf(wb1, x11, cb)));
        ah[ks][2 * hh] = bf16x2_split(h00, h01, al[ks][2 * hh]);          // row g
        ah[ks][2 * hh + 1] = bf16x2_split(h10, h11, al[ks][2 * hh + 1]);  // row g + 8
      }
    float acc[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; nt++) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ks++)
#pragma unroll
      for (int nt = 0; nt < 8; nt++) {
        // B[k][n] = W2[n][k]: two consecutive k of output neuron n = 8 nt + g
        const uint32_t *wr = w2 + (nt * 8 + g) * (kW2Stride / 2) + ks * 8 + t4;
        const uint32_t bw0 = wr[0], bw1 = wr[4];
        mma_bf16_16816(acc[nt], ah[ks], bw0, bw1);
        mma_bf16_16816(acc[nt], al[ks], bw0, bw1);
      }
    float y0 = 0.f, y1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
      const int n = nt * 8 + 2 * t4;
      y0 = fmaf(W3[n], act(acc[nt][0] + b2[n]), y0);
      y0 = fmaf(W3[n + 1], act(acc[nt][1] + b2[n + 1]), y0);
      y1 = fmaf(W3[n], act(acc[nt][2] + b2[n]), y1);
      y1 = fmaf(W3[n + 1], act(acc[nt][3] + b2[n + 1]), y1);
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    if (t4 == 0) {
      if (p0 < npts && pending(p0)) apply(p0, y0 + b3);
      if (p1 < npts && pending(p1)) apply(p1, y1 + b3);
    }
  }
}

}  // namespace fem
