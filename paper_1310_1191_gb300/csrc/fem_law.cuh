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

namespace fem {

constexpr int kMlpH = 64;
__host__ __device__ constexpr int mlp_nparams(int H) { return 2 * H + H + H * H + H + H + 1; }
constexpr int kMlpP = mlp_nparams(kMlpH);  // 4481

template <class R>
__device__ __forceinline__ R law_exact(R u, R g);

template <>
__device__ __forceinline__ float law_exact<float>(float u, float g) {
  const float e = 0.5f * expf(-u * u);
  float k = 1.f + e;
#pragma unroll
  for (int it = 0; it < 8; it++) {
    const float kg1 = 1.f + k * g;
    const float F = k - 1.f - e - 0.2f * logf(kg1);
    const float Fp = 1.f - 0.2f * g / kg1;
    k -= F / Fp;
  }
  return k;
}

template <>
__device__ __forceinline__ double law_exact<double>(double u, double g) {
  const double e = 0.5 * exp(-u * u);
  double k = 1.0 + e;
#pragma unroll
  for (int it = 0; it < 8; it++) {
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

}  // namespace fem
