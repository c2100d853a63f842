// Learned coefficient surrogate: training data from the exact law on the GPU,
// a 2 -> 64 -> 64 -> 1 tanh network trained by hand-written forward /
// backward / Adam kernels, field sampling at quadrature points for the
// training box, and the law-aware integration entry point.
//
// Precision: the network computes with BF16-rounded weights (kept as FP32
// values) and FP32 activations and accumulation; Adam updates an FP32 master
// copy and re-rounds the compute copy after every step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fem_geometry.cuh"
#include "fem_internal.h"
#include "fem_law.cuh"

struct fem_mlp_s {
  double box[4] = {0, 0, 0, 0};
  float nrm[4] = {0, 0, 0, 0};
  float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *wc = nullptr;
  float *losses = nullptr;  // per-step losses of the last training call
  uint32_t *w2img = nullptr;  // W2 of the compute weights as BF16 pairs (integration kernels)
  int64_t nlosses = 0;
  int64_t step = 0;
  bool bias_init = false;
};

namespace fem {

constexpr int kGradThreads = 64;  // samples per CTA in the gradient kernel

// SplitMix64 output function on key + (n+1) * golden (Steele, Lea, Flood 2014),
// key = seed XOR (index * golden): the same counter-based draws as the host-side
// input generators.
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t draw_u64(uint64_t seed, uint64_t index, uint64_t n) {
  const uint64_t g = 0x9E3779B97F4A7C15ull;
  return mix64((seed ^ (index * g)) + (n + 1) * g);
}
__host__ __device__ inline double draw_uniform(uint64_t seed, uint64_t index, uint64_t n) {
  return ((double)(draw_u64(seed, index, n) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---------------------------------------------------------------- kernels

__global__ void law_samples_kernel(int64_t n, double u0, double u1, double ls0, double ls1, uint64_t seed,
                                   float *us, float *k) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double u = u0 + (u1 - u0) * draw_uniform(seed, (uint64_t)i, 0);
  const double s = exp(ls0 + (ls1 - ls0) * draw_uniform(seed, (uint64_t)i, 1));
  us[2 * i] = (float)u;
  us[2 * i + 1] = (float)s;
  k[i] = (float)law_exact<double>(u, s * s);
}

__global__ void round_kernel(const float *master, float *wc, int P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) wc[i] = bf16_round(master[i]);
}

__global__ void mean_kernel(int64_t n, const float *t, float *out) {
  float s = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += t[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s / (float)n);
}

// W2 of the compute weights (BF16 values held as FP32) packed as BF16 pairs,
// row n = output neuron: the B operand of the integration kernels' network stage.
__global__ void pack_w2_kernel(const float *wc, uint32_t *img) {
  constexpr int H = kMlpH;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= H * H / 2) return;
  const float *W2 = wc + 3 * H;
  const __nv_bfloat162 v = __floats2bfloat162_rn(W2[2 * i], W2[2 * i + 1]);
  img[i] = *reinterpret_cast<const uint32_t *>(&v);
}

__global__ void set_bias_kernel(float *master, float *wc, const float *mean, int idx) {
  master[idx] = *mean;
  wc[idx] = bf16_round(*mean);
}

__global__ void mlp_forward_kernel(const float *wc, float n0, float n1, float n2, float n3, int64_t n,
                                   const float *us, float *y) {
  __shared__ float sW[kMlpP];
  for (int i = threadIdx.x; i < kMlpP; i += blockDim.x) sW[i] = wc[i];
  __syncthreads();
  const float nrm[4] = {n0, n1, n2, n3};
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = mlp_eval(sW, nrm, us[2 * i], us[2 * i + 1]);
}

// Loss and gradient of the mean squared error over a set of samples (one
// sample per thread, 64 per CTA), reduced per CTA and added to grad/loss.
// mode 0: samples 0..n-1, mean over n; mode 1: a minibatch of `batch`
// samples drawn with replacement (seed, step), mean over batch.
__global__ void __launch_bounds__(kGradThreads) mlp_grad_kernel(const float *wc, float n0, float n1, float n2,
                                                                float n3, int64_t n, const float *us,
                                                                const float *tg, int mode, int64_t batch,
                                                                uint64_t seed, int64_t step, float *grad,
                                                                float *loss) {
  constexpr int H = kMlpH, S = kGradThreads, LD = H + 1;
  extern __shared__ float sm[];
  float *sW = sm;                   // [P]
  float *sH1 = sW + kMlpP;          // [S][LD]  h1, later d1
  float *sH2 = sH1 + S * LD;        // [S][LD]  h2, later d2
  float *sX = sH2 + S * LD;         // [S][2]
  float *sDY = sX + 2 * S;          // [S]
  const float *W1 = sW, *b1 = W1 + 2 * H, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H, *b3 = W3 + H;
  float *gW1 = grad, *gb1 = gW1 + 2 * H, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H, *gb3 = gW3 + H;
  const int t = threadIdx.x;
  for (int i = t; i < kMlpP; i += S) sW[i] = wc[i];
  // this thread's sample
  const int64_t local = blockIdx.x * (int64_t)S + t;
  const int64_t total = mode == 0 ? n : batch;
  const bool live = local < total;
  int64_t si = 0;
  if (live) si = mode == 0 ? local : (int64_t)(draw_u64(seed, (uint64_t)step, (uint64_t)local) % (uint64_t)n);
  const float u = live ? us[2 * si] : 0.f, sv = live ? us[2 * si + 1] : 1.f, target = live ? tg[si] : 0.f;
  const float x0 = fmaf(u, n0, n1), x1 = fmaf(logf(sv), n2, n3);
  sX[2 * t] = x0;
  sX[2 * t + 1] = x1;
  __syncthreads();
  // forward
  float h1[H];
#pragma unroll
  for (int j = 0; j < H; j++) {
    h1[j] = tanhf(fmaf(W1[2 * j], x0, fmaf(W1[2 * j + 1], x1, b1[j])));
    sH1[t * LD + j] = h1[j];
  }
  float y = b3[0];
#pragma unroll 2
  for (int i = 0; i < H; i++) {
    float a = b2[i];
#pragma unroll
    for (int j = 0; j < H; j++) a = fmaf(W2[i * H + j], h1[j], a);
    const float h2 = tanhf(a);
    sH2[t * LD + i] = h2;
    y = fmaf(W3[i], h2, y);
  }
  const float r = live ? y - target : 0.f;
  const float dy = 2.f * r / (float)total;
  sDY[t] = dy;
  float lsum = r * r;
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((t & 31) == 0) atomicAdd(loss, lsum / (float)total);
  __syncthreads();
  // output layer: gW3[j] = sum_s dy_s h2[s][j], gb3 = sum_s dy_s
  {
    float a = 0.f;
    for (int s = 0; s < S; s++) a = fmaf(sDY[s], sH2[s * LD + t], a);
    atomicAdd(&gW3[t], a);
    if (t == 0) {
      float b = 0.f;
      for (int s = 0; s < S; s++) b += sDY[s];
      atomicAdd(gb3, b);
    }
  }
  __syncthreads();
  // d2 = dy W3 (1 - h2^2), own row
#pragma unroll 4
  for (int i = 0; i < H; i++) {
    const float h2 = sH2[t * LD + i];
    sH2[t * LD + i] = dy * W3[i] * (1.f - h2 * h2);
  }
  __syncthreads();
  // gW2[i][j] = sum_s d2[s][i] h1[s][j], gb2[i] = sum_s d2[s][i]  (thread i)
  {
    const int i = t;
    float acc[H];
#pragma unroll
    for (int j = 0; j < H; j++) acc[j] = 0.f;
    float bsum = 0.f;
    for (int s = 0; s < S; s++) {
      const float d = sH2[s * LD + i];
      bsum += d;
#pragma unroll
      for (int j = 0; j < H; j++) acc[j] = fmaf(d, sH1[s * LD + j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < H; j++) atomicAdd(&gW2[i * H + j], acc[j]);
    atomicAdd(&gb2[i], bsum);
  }
  __syncthreads();
  // d1[j] = (1 - h1[j]^2) sum_i W2[i][j] d2[i], own row (overwrites h1)
  {
    float d1[H];
#pragma unroll
    for (int j = 0; j < H; j++) d1[j] = 0.f;
    for (int i = 0; i < H; i++) {
      const float d = sH2[t * LD + i];
#pragma unroll
      for (int j = 0; j < H; j++) d1[j] = fmaf(W2[i * H + j], d, d1[j]);
    }
#pragma unroll
    for (int j = 0; j < H; j++) {
      const float h = sH1[t * LD + j];
      sH1[t * LD + j] = d1[j] * (1.f - h * h);
    }
  }
  __syncthreads();
  // gW1[j][0..1] = sum_s d1[s][j] x[s][0..1], gb1[j] = sum_s d1[s][j]  (thread j)
  {
    const int j = t;
    float a0 = 0.f, a1 = 0.f, bb = 0.f;
    for (int s = 0; s < S; s++) {
      const float d = sH1[s * LD + j];
      a0 = fmaf(d, sX[2 * s], a0);
      a1 = fmaf(d, sX[2 * s + 1], a1);
      bb += d;
    }
    atomicAdd(&gW1[2 * j], a0);
    atomicAdd(&gW1[2 * j + 1], a1);
    atomicAdd(&gb1[j], bb);
  }
}

__global__ void adam_kernel(float *master, float *m, float *v, const float *g, float *wc, int P, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float w = master[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  master[i] = w;
  wc[i] = bf16_round(w);
}

// u and |grad u| at every quadrature point of prisms of one degree (FP64
// geometry, FP32 sums), for the surrogate's training box.
__global__ void field_samples_kernel(int64_t n, int ns, int nq, const double *coords, const float *ucoef,
                                     const double *qp, const float *phi32, float *out) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n * nq) return;
  const int64_t e = idx / nq;
  const int q = (int)(idx % nq);
  double adj[3][3];
  const double det = jac_adj<FEM_PRISM6>(coords + e * 18, qp + 4 * q, adj);
  const float *U = ucoef + e * ns;
  const float *ph = phi32 + (size_t)(4 * q) * ns;
  float u = 0.f, r0 = 0.f, r1 = 0.f, r2 = 0.f;
  for (int k = 0; k < ns; k++) {
    u = fmaf(U[k], ph[k], u);
    r0 = fmaf(U[k], ph[ns + k], r0);
    r1 = fmaf(U[k], ph[2 * ns + k], r1);
    r2 = fmaf(U[k], ph[3 * ns + k], r2);
  }
  const double gx = (adj[0][0] * r0 + adj[1][0] * r1 + adj[2][0] * r2) / det;
  const double gy = (adj[0][1] * r0 + adj[1][1] * r1 + adj[2][1] * r2) / det;
  const double gz = (adj[0][2] * r0 + adj[1][2] * r1 + adj[2][2] * r2) / det;
  out[2 * idx] = u;
  out[2 * idx + 1] = (float)sqrt(gx * gx + gy * gy + gz * gz);
}

static int cuda_check(const char *what, cudaError_t e) {
  if (e == cudaSuccess) return FEM_OK;
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return FEM_ECUDA;
}

static size_t grad_smem() { return sizeof(float) * (kMlpP + 2 * kGradThreads * (kMlpH + 1) + 3 * kGradThreads); }

static int launch_grad(fem_mlp_s *m, int64_t n, const float *us, const float *t, int mode, int64_t batch,
                       uint64_t seed, int64_t step, float *loss, cudaStream_t s) {
  const int64_t total = mode == 0 ? n : batch;
  const int64_t blocks = (total + kGradThreads - 1) / kGradThreads;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
    attr = true;
  }
  mlp_grad_kernel<<<(unsigned)blocks, kGradThreads, grad_smem(), s>>>(m->wc, m->nrm[0], m->nrm[1], m->nrm[2],
                                                                       m->nrm[3], n, us, t, mode, batch, seed, step,
                                                                       m->grad, loss);
  return cuda_check("mlp_grad_kernel", cudaGetLastError());
}

}  // namespace fem

using namespace fem;

extern "C" {

int fem_law_samples(int64_t n, const double *box, uint64_t seed, float *us, float *k, void *stream) {
  if (n < 0 || !box || (n > 0 && (!us || !k)) || !(box[1] > box[0]) || !(box[2] > 0.0) || !(box[3] > box[2])) {
    set_error("fem_law_samples: bad arguments (box must have u1 > u0 and s1 > s0 > 0)");
    return FEM_EINVAL;
  }
  if (n == 0) return FEM_OK;
  const int64_t blocks = (n + 255) / 256;
  law_samples_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, box[0], box[1], std::log(box[2]),
                                                                         std::log(box[3]), seed, us, k);
  return cuda_check("law_samples_kernel", cudaGetLastError());
}

int fem_field_samples(fem_tables t, int p, int64_t n, const double *coords, const float *ucoef, float *us,
                      void *stream) {
  if (rule_check(t, "fem_field_samples") != FEM_OK) return FEM_EUNSUPPORTED;
  if (!t || t->elem != FEM_PRISM6 || p < t->p_min || p > t->p_max || n < 0 ||
      (n > 0 && (!coords || !ucoef || !us))) {
    set_error("fem_field_samples: bad arguments");
    return FEM_EINVAL;
  }
  if (n == 0) return FEM_OK;
  const DevTable &d = t->tab[p];
  const int64_t total = n * d.nq;
  field_samples_kernel<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      n, d.ns, d.nq, coords, ucoef, d.qp, d.phi32, us);
  return cuda_check("field_samples_kernel", cudaGetLastError());
}

int fem_box_from_samples(int64_t n, const float *us_host, double lo_pct, double hi_pct, double *box) {
  if (n <= 0 || !us_host || !box || !(lo_pct >= 0.0) || !(hi_pct <= 100.0) || !(lo_pct < hi_pct)) {
    set_error("fem_box_from_samples: bad arguments");
    return FEM_EINVAL;
  }
  std::vector<float> u(n), s(n);
  for (int64_t i = 0; i < n; i++) {
    u[i] = us_host[2 * i];
    s[i] = us_host[2 * i + 1];
  }
  auto pct = [&](std::vector<float> &v, double q) {
    const int64_t k = std::min<int64_t>(n - 1, std::max<int64_t>(0, (int64_t)std::llround(q / 100.0 * (n - 1))));
    std::nth_element(v.begin(), v.begin() + k, v.end());
    return (double)v[k];
  };
  box[0] = pct(u, lo_pct);
  box[1] = pct(u, hi_pct);
  box[2] = pct(s, lo_pct);
  box[3] = pct(s, hi_pct);
  if (!(box[1] > box[0]) || !(box[2] > 0.0) || !(box[3] > box[2])) {
    set_error("fem_box_from_samples: degenerate box");
    return FEM_EINVAL;
  }
  return FEM_OK;
}

int fem_mlp_create(const double *box, uint64_t seed, fem_mlp *out) {
  if (!out || !box || !(box[1] > box[0]) || !(box[2] > 0.0) || !(box[3] > box[2])) {
    set_error("fem_mlp_create: bad arguments (box must have u1 > u0 and s1 > s0 > 0)");
    return FEM_EINVAL;
  }
  *out = nullptr;
  fem_mlp m = new (std::nothrow) fem_mlp_s();
  if (!m) return FEM_ENOMEM;
  for (int i = 0; i < 4; i++) m->box[i] = box[i];
  mlp_norm_from_box(box, m->nrm);
  // Glorot-uniform weights from counter-based draws, zero biases
  constexpr int H = kMlpH;
  std::vector<float> w(kMlpP, 0.f);
  auto fill = [&](int off, int count, int fan_in, int fan_out, uint64_t stream_id) {
    const double a = std::sqrt(6.0 / (fan_in + fan_out));
    for (int i = 0; i < count; i++) w[off + i] = (float)(a * (2.0 * draw_uniform(seed, stream_id * 1000003ull + i, 0) - 1.0));
  };
  fill(0, 2 * H, 2, H, 1);
  fill(3 * H, H * H, H, H, 2);
  fill(3 * H + H * H + H, H, H, 1, 3);
  int rc = FEM_OK;
  auto alloc = [&](float **p) {
    if (rc != FEM_OK) return;
    if (cudaMalloc((void **)p, sizeof(float) * kMlpP) != cudaSuccess) {
      set_error("fem_mlp_create: cudaMalloc");
      rc = FEM_ENOMEM;
      return;
    }
    cudaMemset(*p, 0, sizeof(float) * kMlpP);
  };
  alloc(&m->master);
  alloc(&m->m);
  alloc(&m->v);
  alloc(&m->grad);
  alloc(&m->wc);
  if (rc == FEM_OK && cudaMalloc((void **)&m->w2img, sizeof(uint32_t) * H * H / 2) != cudaSuccess) {
    m->w2img = nullptr;
    set_error("fem_mlp_create: cudaMalloc");
    rc = FEM_ENOMEM;
  }
  if (rc == FEM_OK) rc = cuda_check("fem_mlp_create", cudaMemcpy(m->master, w.data(), sizeof(float) * kMlpP,
                                                                 cudaMemcpyHostToDevice));
  if (rc == FEM_OK) {
    round_kernel<<<(kMlpP + 255) / 256, 256>>>(m->master, m->wc, kMlpP);
    rc = cuda_check("round_kernel", cudaDeviceSynchronize());
  }
  if (rc != FEM_OK) {
    fem_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return FEM_OK;
}

int fem_mlp_destroy(fem_mlp m) {
  if (!m) return FEM_OK;
  for (float *p : {m->master, m->m, m->v, m->grad, m->wc, m->losses})
    if (p) cudaFree(p);
  if (m->w2img) cudaFree(m->w2img);
  delete m;
  return FEM_OK;
}

int fem_mlp_nparams(void) { return kMlpP; }

int fem_mlp_forward(fem_mlp m, int64_t n, const float *us, float *y, void *stream) {
  if (!m || n < 0 || (n > 0 && (!us || !y))) {
    set_error("fem_mlp_forward: bad arguments");
    return FEM_EINVAL;
  }
  if (n == 0) return FEM_OK;
  mlp_forward_kernel<<<(unsigned)((n + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
      m->wc, m->nrm[0], m->nrm[1], m->nrm[2], m->nrm[3], n, us, y);
  return cuda_check("mlp_forward_kernel", cudaGetLastError());
}

int fem_mlp_loss_grad(fem_mlp m, int64_t n, const float *us, const float *t, float *grad, float *loss,
                      void *stream) {
  if (!m || n <= 0 || !us || !t || !grad || !loss) {
    set_error("fem_mlp_loss_grad: bad arguments");
    return FEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int rc = cuda_check("memset", cudaMemsetAsync(m->grad, 0, sizeof(float) * kMlpP, s));
  if (rc == FEM_OK) rc = cuda_check("memset", cudaMemsetAsync(loss, 0, sizeof(float), s));
  if (rc == FEM_OK) rc = launch_grad(m, n, us, t, 0, 0, 0, 0, loss, s);
  if (rc == FEM_OK)
    rc = cuda_check("copy", cudaMemcpyAsync(grad, m->grad, sizeof(float) * kMlpP, cudaMemcpyDeviceToDevice, s));
  return rc;
}

int fem_mlp_train(fem_mlp m, int64_t n, const float *us, const float *t, int64_t steps, int batch, float lr,
                  uint64_t seed, float *loss_host, void *stream) {
  if (!m || n <= 0 || !us || !t || steps < 0 || batch <= 0 || !(lr > 0.f)) {
    set_error("fem_mlp_train: bad arguments");
    return FEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int rc = FEM_OK;
  if (steps > m->nlosses) {
    if (m->losses) cudaFree(m->losses);
    m->losses = nullptr;
    rc = cuda_check("cudaMalloc(losses)", cudaMalloc((void **)&m->losses, sizeof(float) * steps));
    if (rc != FEM_OK) return rc;
    m->nlosses = steps;
  }
  if (steps > 0) rc = cuda_check("memset", cudaMemsetAsync(m->losses, 0, sizeof(float) * steps, s));
  if (rc == FEM_OK && !m->bias_init && steps > 0) {  // output bias starts at the mean target
    float *mean = m->losses;          // scratch slot, cleared again below
    mean_kernel<<<256, 256, 0, s>>>(n, t, mean);
    set_bias_kernel<<<1, 1, 0, s>>>(m->master, m->wc, mean, kMlpP - 1);
    rc = cuda_check("bias init", cudaGetLastError());
    if (rc == FEM_OK) rc = cuda_check("memset", cudaMemsetAsync(m->losses, 0, sizeof(float), s));
    m->bias_init = true;
  }
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int64_t it = 0; it < steps && rc == FEM_OK; it++) {
    rc = cuda_check("memset", cudaMemsetAsync(m->grad, 0, sizeof(float) * kMlpP, s));
    if (rc == FEM_OK) rc = launch_grad(m, n, us, t, 1, batch, seed, m->step, m->losses + it, s);
    m->step++;
    const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
    if (rc == FEM_OK) {
      adam_kernel<<<(kMlpP + 255) / 256, 256, 0, s>>>(m->master, m->m, m->v, m->grad, m->wc, kMlpP, lr, b1, b2,
                                                      eps, c1, c2);
      rc = cuda_check("adam_kernel", cudaGetLastError());
    }
  }
  if (rc == FEM_OK && loss_host && steps > 0) {
    rc = cuda_check("losses", cudaMemcpyAsync(loss_host, m->losses, sizeof(float) * steps, cudaMemcpyDeviceToHost, s));
    if (rc == FEM_OK) rc = cuda_check("sync", cudaStreamSynchronize(s));
  }
  return rc;
}

int fem_mlp_get(fem_mlp m, float *master_host, float *compute_host, double *box) {
  if (!m) {
    set_error("fem_mlp_get: NULL network");
    return FEM_EINVAL;
  }
  int rc = cuda_check("sync", cudaDeviceSynchronize());
  if (rc == FEM_OK && master_host)
    rc = cuda_check("copy", cudaMemcpy(master_host, m->master, sizeof(float) * kMlpP, cudaMemcpyDeviceToHost));
  if (rc == FEM_OK && compute_host)
    rc = cuda_check("copy", cudaMemcpy(compute_host, m->wc, sizeof(float) * kMlpP, cudaMemcpyDeviceToHost));
  if (box)
    for (int i = 0; i < 4; i++) box[i] = m->box[i];
  return rc;
}

int fem_mlp_set(fem_mlp m, const float *master_host) {
  if (!m || !master_host) {
    set_error("fem_mlp_set: bad arguments");
    return FEM_EINVAL;
  }
  int rc = cuda_check("copy", cudaMemcpy(m->master, master_host, sizeof(float) * kMlpP, cudaMemcpyHostToDevice));
  if (rc == FEM_OK) {
    round_kernel<<<(kMlpP + 255) / 256, 256>>>(m->master, m->wc, kMlpP);
    rc = cuda_check("round_kernel", cudaDeviceSynchronize());
  }
  m->bias_init = true;
  return rc;
}

// File: "FEMMLP01", int32 H, int32 P, double box[4], int64 step, then float
// master[P], Adam m[P], v[P].
int fem_mlp_save(fem_mlp m, const char *path) {
  if (!m || !path) {
    set_error("fem_mlp_save: bad arguments");
    return FEM_EINVAL;
  }
  std::vector<float> a(kMlpP), b(kMlpP), c(kMlpP);
  int rc = cuda_check("sync", cudaDeviceSynchronize());
  if (rc == FEM_OK) rc = cuda_check("copy", cudaMemcpy(a.data(), m->master, sizeof(float) * kMlpP, cudaMemcpyDeviceToHost));
  if (rc == FEM_OK) rc = cuda_check("copy", cudaMemcpy(b.data(), m->m, sizeof(float) * kMlpP, cudaMemcpyDeviceToHost));
  if (rc == FEM_OK) rc = cuda_check("copy", cudaMemcpy(c.data(), m->v, sizeof(float) * kMlpP, cudaMemcpyDeviceToHost));
  if (rc != FEM_OK) return rc;
  FILE *f = std::fopen(path, "wb");
  if (!f) {
    set_error("fem_mlp_save: cannot open file");
    return FEM_EINVAL;
  }
  const int32_t hp[2] = {kMlpH, kMlpP};
  bool ok = std::fwrite("FEMMLP01", 1, 8, f) == 8 && std::fwrite(hp, 4, 2, f) == 2 &&
            std::fwrite(m->box, 8, 4, f) == 4 && std::fwrite(&m->step, 8, 1, f) == 1 &&
            std::fwrite(a.data(), 4, kMlpP, f) == (size_t)kMlpP && std::fwrite(b.data(), 4, kMlpP, f) == (size_t)kMlpP &&
            std::fwrite(c.data(), 4, kMlpP, f) == (size_t)kMlpP;
  std::fclose(f);
  if (!ok) {
    set_error("fem_mlp_save: write failed");
    return FEM_EINVAL;
  }
  return FEM_OK;
}

int fem_mlp_load(const char *path, fem_mlp *out) {
  if (!path || !out) {
    set_error("fem_mlp_load: bad arguments");
    return FEM_EINVAL;
  }
  *out = nullptr;
  FILE *f = std::fopen(path, "rb");
  if (!f) {
    set_error("fem_mlp_load: cannot open file");
    return FEM_EINVAL;
  }
  char magic[8];
  int32_t hp[2];
  double box[4];
  int64_t step;
  std::vector<float> a(kMlpP), b(kMlpP), c(kMlpP);
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "FEMMLP01", 8) == 0 && std::fread(hp, 4, 2, f) == 2 &&
            hp[0] == kMlpH && hp[1] == kMlpP && std::fread(box, 8, 4, f) == 4 && std::fread(&step, 8, 1, f) == 1 &&
            std::fread(a.data(), 4, kMlpP, f) == (size_t)kMlpP && std::fread(b.data(), 4, kMlpP, f) == (size_t)kMlpP &&
            std::fread(c.data(), 4, kMlpP, f) == (size_t)kMlpP;
  std::fclose(f);
  if (!ok) {
    set_error("fem_mlp_load: not a network file of this library");
    return FEM_EINVAL;
  }
  fem_mlp m = nullptr;
  int rc = fem_mlp_create(box, 0, &m);
  if (rc != FEM_OK) return rc;
  rc = fem_mlp_set(m, a.data());
  if (rc == FEM_OK) rc = cuda_check("copy", cudaMemcpy(m->m, b.data(), sizeof(float) * kMlpP, cudaMemcpyHostToDevice));
  if (rc == FEM_OK) rc = cuda_check("copy", cudaMemcpy(m->v, c.data(), sizeof(float) * kMlpP, cudaMemcpyHostToDevice));
  m->step = step;
  if (rc != FEM_OK) {
    fem_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return FEM_OK;
}

int fem_integrate_law(fem_tables t, int p, int64_t n_elem, const double *coords, const double *coeffs,
                      int64_t coeff_stride, const float *ucoef, int law, fem_mlp mlp, int prec, int layout,
                      void *A_out, void *b_out, int32_t *status, void *stream) {
  return integrate_law_opts(t, p, n_elem, coords, coeffs, coeff_stride, ucoef, law, mlp, 8, 0, prec, layout, A_out,
                            b_out, status, stream);
}

}  // extern "C"

namespace fem {

int integrate_law_opts(fem_tables t, int p, int64_t n_elem, const double *coords, const double *coeffs,
                       int64_t coeff_stride, const float *ucoef, int law, fem_mlp mlp, int newton_steps,
                       int hw_tanh, int prec, int layout, void *A_out, void *b_out, int32_t *status, void *stream) {
  if (rule_check(t, "fem_integrate_law") != FEM_OK) return FEM_EUNSUPPORTED;
  if (newton_steps < 1 || newton_steps > 1024) {
    set_error("fem_integrate_law: Newton steps must be in 1..1024");
    return FEM_EINVAL;
  }
  if (!t) {
    set_error("fem_integrate_law: tables handle is NULL");
    return FEM_EINVAL;
  }
  if (law != FEM_LAW_EXACT && law != FEM_LAW_MLP) {
    set_error("fem_integrate_law: law must be FEM_LAW_EXACT or FEM_LAW_MLP");
    return FEM_EINVAL;
  }
  if (law == FEM_LAW_MLP && !mlp) {
    set_error("fem_integrate_law: FEM_LAW_MLP needs a network");
    return FEM_EINVAL;
  }
  if (prec != FEM_F64 && prec != FEM_F32 && !(prec == FEM_BF16X3 && t->elem == FEM_PRISM6)) {
    set_error("fem_integrate_law: FP64, FP32, or BF16x3 tensor cores (prisms)");
    return FEM_EUNSUPPORTED;
  }
  if (p < t->p_min || p > t->p_max || n_elem < 0 || (layout != FEM_OUT_FULL && layout != FEM_OUT_SYMPACKED)) {
    set_error("fem_integrate_law: bad degree, n_elem or layout");
    return FEM_EINVAL;
  }
  if (n_elem == 0) return FEM_OK;
  if (!coords || !coeffs || !A_out || !ucoef || coeff_stride < n_elem) {
    set_error("fem_integrate_law: NULL buffer or coeff_stride < n_elem");
    return FEM_EINVAL;
  }
  if ((((uintptr_t)coords | (uintptr_t)coeffs) & 7) || ((uintptr_t)A_out & 15) || ((uintptr_t)ucoef & 3)) {
    set_error("fem_integrate_law: misaligned buffer");
    return FEM_EINVAL;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) {
    set_error("fem_integrate_law: tables live on another device");
    return FEM_EINVAL;
  }
  const DevTable &d = t->tab[p];
  if (law == FEM_LAW_MLP)  // the compute weights may have changed since the last call (training)
    pack_w2_kernel<<<(kMlpH * kMlpH / 2 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(mlp->wc, mlp->w2img);
  if (prec == FEM_BF16X3) {
    TcLaunch l;
    l.n = n_elem;
    l.coords = coords;
    l.coeffs = coeffs;
    l.cstride = coeff_stride;
    l.A = A_out;
    l.b = b_out;
    l.status = status;
    l.layout = layout;
    l.err = t->d_err;
    l.stall = 0;
    l.law = law;
    l.ucoef = ucoef;
    l.law_iters = newton_steps;
    l.hw_tanh = hw_tanh;
    if (law == FEM_LAW_MLP) {
      l.mlpw = mlp->wc;
      l.mlpw2 = mlp->w2img;
      for (int i = 0; i < 4; i++) {
        l.nrm[i] = mlp->nrm[i];
        l.box[i] = (float)mlp->box[i];
      }
    }
    return launch_tc(p, false, d, l, stream);
  }
  FmaArgs a;
  a.n = n_elem;
  a.coords = coords;
  a.coeffs = coeffs;
  a.cstride = coeff_stride;
  a.qp = d.qp;
  a.phi = prec == FEM_F64 ? (const void *)d.phi64 : (const void *)d.phi32;
  a.phiT = prec == FEM_F64 ? (const void *)d.phiT64 : (const void *)d.phiT32;
  a.A = A_out;
  a.b = b_out;
  a.status = status;
  a.layout = layout;
  a.err = t->d_err;
  a.ucoef = ucoef;
  a.law_iters = newton_steps;
  a.hw_tanh = hw_tanh;
  if (law == FEM_LAW_MLP) {
    a.mlpw2 = mlp->w2img;
    a.mlpw = mlp->wc;
    for (int i = 0; i < 4; i++) {
      a.nrm[i] = mlp->nrm[i];
      a.box[i] = (float)mlp->box[i];
    }
  }
  return prec == FEM_F64 ? launch_fma_law_f64(t->elem, p, law, a, stream)
                         : launch_fma_law_f32(t->elem, p, law, a, stream);
}

}  // namespace fem
