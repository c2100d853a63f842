// Internal declarations shared by the library's translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "fem.h"

namespace fem {

constexpr int kMaxP = 7;

// Checked builds (-DFEM_CHECKED, libfem_gb300_checked.so): the kernels check
// the element ids and output offsets that come from permutations and offset
// tables against the launch's bounds; a failed check skips the access and
// sets bit 2 of the device error word (fem_error_flag then returns
// FEM_ECHECKED).  In normal builds every check is compiled out.
#ifdef FEM_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
constexpr int kErrTimeout = 1, kErrCheck = 2;

#ifdef __CUDACC__
__device__ __forceinline__ bool fem_chk(bool ok, int *err) {
  if constexpr (kChecked) {
    if (!ok && err) atomicOr(err, kErrCheck);
    return ok;
  } else {
    return true;
  }
}
#endif

__host__ __device__ constexpr int ns_of(int elem, int p) {
  return elem == FEM_TET4 ? 4 : (p + 1) * (p + 1) * (p + 2) / 2;
}
// Triangle points of a prism rule: (p+1)^2 for the collapsed rule, the
// fully symmetric triangle rule's 3, 6, 12, 16, 25, 33, 42 points for the
// paper's rule (Table 1: N_Q = that times p + 1).
__host__ __device__ constexpr int ntri_of(int p, int rule = FEM_RULE_COLLAPSED) {
  return rule == FEM_RULE_TABLE1
             ? (p == 1 ? 3 : p == 2 ? 6 : p == 3 ? 12 : p == 4 ? 16 : p == 5 ? 25 : p == 6 ? 33 : 42)
             : (p + 1) * (p + 1);
}
__host__ __device__ constexpr int nq_of(int elem, int p, int rule = FEM_RULE_COLLAPSED) {
  return elem == FEM_TET4 ? 4 : (p + 1) * ntri_of(p, rule);
}
__host__ __device__ constexpr int nv_of(int elem) { return elem == FEM_TET4 ? 4 : 6; }

// Reference data of one (element, degree), built on the host in FP64.
struct HostRule {
  int nq = 0, ns = 0;
  std::vector<double> xi;   // [nq][3]
  std::vector<double> w;    // [nq]
  std::vector<double> phi;  // [nq][4][ns]
};

// Builds the quadrature rule and shape-function table; false if (elem, p,
// rule) is invalid (the paper's rule exists for prisms only).  Prism points
// are ordered q = iz * ntri_of(p, rule) + it: zeta level iz, triangle point it.
bool build_host_rule(int elem, int p, HostRule *out, int rule = FEM_RULE_COLLAPSED);

// 1D factor tables of the prism rule and basis for sum factorisation, FP64:
// Pa, Px, Pe [N][N] (point ia, index i), Bq, Bx, By [NT][N | 1] (triangle DOF
// t, point ib; rows padded to an odd length), L, dL [N][N] (zeta level iz,
// degree k); N = p + 1, NT = N (N + 1) / 2.  Definitions in fem_tables.cpp.
void build_sf_tables(int p, std::vector<double> &out);

// Device copies of one degree's tables.
struct DevTable {
  int p = 0, ns = 0, nq = 0, rule = FEM_RULE_COLLAPSED;
  double *qp = nullptr;     // [nq][4]: xi, eta, zeta, w (FP64)
  double *phi64 = nullptr;  // [4 nq][ns] row k = 4 q + d (FP64)
  float *phi32 = nullptr;   // same, FP32
  // point-major copies [ns][nq][4] (value + 3 derivatives of shape function i
  // at point q contiguous): threads that own consecutive points read
  // consecutive 4-vectors when they evaluate a field at their points
  double *phiT64 = nullptr;
  float *phiT32 = nullptr;
  // [nq][ns][4] FP32 (the 4 values of function i at point q contiguous, then
  // the next function): the tensor-core producers, whose threads own
  // consecutive functions, load one float4 per point
  float *phiq32 = nullptr;
  // tensor-core operand images of Phi^T (hi | lo per K chunk), prisms only
  uint16_t *img_bf16 = nullptr;
  uint16_t *img_f16 = nullptr;
  // sum-factorisation factors (build_sf_tables), prisms only
  double *sf64 = nullptr;
  float *sf32 = nullptr;
  float phimax = 0.f;  // max |Phi|
  int aphi_f16 = 0;    // power-of-two scale applied to the FP16 image
};

}  // namespace fem

struct fem_tables_s {
  int elem = 0, p_min = 0, p_max = 0, device = 0;
  int rule = FEM_RULE_COLLAPSED;  // quadrature rule of every degree in the tables
  int *d_err = nullptr;  // device error word (bounded waits that expired)
  unsigned long long *d_red = nullptr;  // [2] status reduction of fem_sync_status (OR of bits, count)
  int stall_next = 0;    // test hook: the next tensor-core launch withholds its operand copies
  fem::DevTable tab[fem::kMaxP + 1];
  // staging for host-buffer integration (two pipeline slots)
  unsigned char *stage[2] = {nullptr, nullptr};
  size_t stage_bytes = 0;
  cudaStream_t hs[2] = {nullptr, nullptr};
  // mixed-degree plan that fem_integrate keeps for per-element degrees (the
  // degrees, precision and layout it was made for)
  struct fem_plan_s *mixed = nullptr;
  std::vector<int8_t> mixed_p;
  int mixed_prec = -1, mixed_layout = -1;
  std::mutex mixed_mutex;
};

namespace fem {

// thread-local last-error text
void set_error(const std::string &msg);

// FEM_EUNSUPPORTED (with a message naming fn) for tables built with the
// paper's rule: the entry points other than fem_integrate / fem_integrate_uniform
// / fem_integrate_elastic / fem_integrate_host have kernels for the collapsed
// rule only.
inline int rule_check(const fem_tables_s *t, const char *fn) {
  if (t && t->rule != FEM_RULE_COLLAPSED) {
    set_error(std::string(fn) + ": tables with the paper's rule (FEM_RULE_TABLE1) serve fem_integrate only");
    return FEM_EUNSUPPORTED;
  }
  return FEM_OK;
}

// Kernel launch arguments of the FMA path.
struct FmaArgs {
  int64_t n;
  const double *coords;
  const double *coeffs;
  int64_t cstride;
  const double *qp;
  const void *phi;  // FP64 or FP32 table by precision
  void *A;
  void *b;
  int32_t *status;
  int layout;
  const int64_t *perm = nullptr;  // sorted position -> element id (batched path), or NULL
  const int64_t *offA = nullptr;  // per-element offset of A_e in A (values), or NULL
  const int64_t *offb = nullptr;  // per-element offset of b_e in b (values), or NULL
  // split geometry: [n][NQ][10] det J and J^{-1} per point, read instead of
  // computing J from coords (coords unused then), or NULL
  const double *terms = nullptr;
  // nonlinear coefficient law (law kernels only)
  const float *ucoef = nullptr;  // [n][NS] field coefficients of u per element
  const void *phiT = nullptr;    // point-major table [NS][NQ][4] in the kernel's precision
  const float *mlpw = nullptr;   // network parameters (FP32 values of BF16 weights)
  const uint32_t *mlpw2 = nullptr;  // the network's W2 as BF16 pairs, [H][H/2] words
  float nrm[4] = {0, 0, 0, 0};   // input normalisation of the network
  float box[4] = {0, 0, 0, 0};   // u0, u1, s0, s1 (network used inside)
  int law_iters = 8;             // Newton steps of the exact law
  int hw_tanh = 0;               // network activations from tanh.approx.f32
  // checked builds: device error word and the values of A and b the outputs
  // hold (negative: not checked)
  int *err = nullptr;
  int64_t limA = -1, limb = -1;
  int64_t nmesh = -1;  // checked builds: element ids from perm lie below it (negative: not checked)
};

// fem_integrate with per-element degrees: runs (and keeps in t) a per-degree
// concurrent plan for these degrees, precision and layout (fem_batch.cu).
int integrate_mixed_cached(fem_tables t, int64_t n, const int8_t *p_host, const double *coords,
                           const double *coeffs, int64_t cstride, int prec, int layout, void *A, void *b,
                           int32_t *status, void *stream);

// Launch the FP64 / FP32 FMA kernels for (elem, p); returns a fem status code.
int launch_fma_f64(int elem, int p, const FmaArgs &a, void *stream);
int launch_fma_f32(int elem, int p, const FmaArgs &a, void *stream);
// the same for prisms with the paper's rule (FEM_RULE_TABLE1), constant coefficients
int launch_fma_t1_f64(int p, const FmaArgs &a, void *stream);
int launch_fma_t1_f32(int p, const FmaArgs &a, void *stream);
int launch_fma_t1_elastic_f64(int p, const FmaArgs &a, void *stream);
int launch_fma_t1_elastic_f32(int p, const FmaArgs &a, void *stream);
// linear elastostatics: a.n real elements, 9 blocks each
int launch_fma_elastic_f64(int p, const FmaArgs &a, void *stream);
// split geometry (a.terms set, a.coords unused): scalar form and elastostatics
int launch_fma_terms(int elem, int p, int prec, const FmaArgs &a, void *stream);
int launch_fma_elastic_terms(int p, int prec, const FmaArgs &a, void *stream);
int launch_fma_elastic_f32(int p, const FmaArgs &a, void *stream);
// law = 1 exact Newton law, 2 network with exact-law fallback
int launch_fma_law_f64(int elem, int p, int law, const FmaArgs &a, void *stream);
int launch_fma_law_f32(int elem, int p, int law, const FmaArgs &a, void *stream);

// Tensor-core path (prisms).
struct TcLaunch {
  int64_t n;
  const double *coords;
  const double *coeffs;
  int64_t cstride;
  void *A;
  void *b;
  int32_t *status;
  int layout;
  int *err;
  int stall;  // withhold the operand copies (failure-detection test)
  int elastic = 0;  // linear elastostatics (coeffs E, nu, f; A [n][3][3][NS][NS], b [n][3][NS])
  // element permutation and output offsets of mixed-degree plans (or NULL)
  const int64_t *perm = nullptr;
  const int64_t *offA = nullptr;
  const int64_t *offb = nullptr;
  // nonlinear coefficient law: 1 exact, 2 network (BF16x3 scalar form)
  int law = 0;
  const float *ucoef = nullptr;
  const float *mlpw = nullptr;
  const uint32_t *mlpw2 = nullptr;
  float nrm[4] = {0, 0, 0, 0};
  float box[4] = {0, 0, 0, 0};
  int law_iters = 8;
  int hw_tanh = 0;
  int64_t limA = -1, limb = -1;  // checked builds: values of A and b (negative: not checked)
  int64_t nmesh = -1;            // checked builds: element ids from perm lie below it
};
int launch_tc(int p, bool f16, const DevTable &d, const TcLaunch &l, void *stream);

// fem_integrate_law with the law's options (Newton steps, hardware tanh)
int integrate_law_opts(fem_tables t, int p, int64_t n_elem, const double *coords, const double *coeffs,
                       int64_t coeff_stride, const float *ucoef, int law, fem_mlp mlp, int newton_steps,
                       int hw_tanh, int prec, int layout, void *A_out, void *b_out, int32_t *status, void *stream);

// Matrix-free element-operator apply y_e = A_e x_e (constant coefficients).
struct ApplyArgs {
  int64_t n;
  const double *coords;
  const double *coeffs;
  int64_t cstride;
  const double *qp;   // [NQ][4]
  const void *tab;    // prisms: sum-factorisation factors; tets: Phi [4 NQ][NS] (the precision's type)
  const void *x;      // [n][NS]
  void *y;            // [n][NS]
  int32_t *status;
};
int launch_apply(int elem, int p, bool f32, const ApplyArgs &a, void *stream);
void build_tc_image(int p, int rule, const std::vector<double> &phi, bool f16, int aphi, std::vector<uint16_t> &out);

}  // namespace fem
