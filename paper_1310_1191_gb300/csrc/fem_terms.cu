// Split geometry pass: the Jacobian terms of the paper's NOJAC kernel variants
// (Section 4: det J and the 9 entries of J^{-1} for every element and
// quadrature point, read by the integration kernel instead of computed).
// The paper prepares them on the host and copies them over; here a device
// pass writes them to HBM, so the comparison with the fused (JAC) kernels
// isolates what storing instead of recomputing costs.
//
// A CTA owns whole elements (EB per CTA, at least 512 points), so it writes
// each element's status word itself.  Prisms use the tensor-product factors
// of J (per zeta level and per (xi, eta) point) built once per element in
// shared memory; tetrahedra have one J per element.
#include "fem_internal.h"
#include "fem_geometry.cuh"

namespace fem {

struct TermsArgs {
  int64_t n;
  const double *coords;  // [n][NV][3]
  const double *qp;      // [NQ][4]
  double *terms;         // [n][NQ][10], 16-byte aligned
  int32_t *status;       // [n] or NULL
};

template <int ELEM, int P>
struct TermsCfg {
  static constexpr int NQ = nq_of(ELEM, P), NV = nv_of(ELEM);
  static constexpr int EB = NQ >= 512 ? 1 : 512 / NQ;  // elements per CTA
  static constexpr int NZ = ELEM == FEM_PRISM6 ? P + 1 : 0, NAB = NZ * NZ;
  static constexpr size_t SMEM = sizeof(double) * (size_t)EB * (kEdgeRec + NZ * kZf + NAB * kXf) +
                                 sizeof(int) * (size_t)EB;
};

constexpr int kTermsThreads = 256;

template <int ELEM, int P>
__global__ void __launch_bounds__(kTermsThreads) terms_kernel(TermsArgs a) {
  using C = TermsCfg<ELEM, P>;
  extern __shared__ __align__(16) unsigned char smem[];
  double *sEd = reinterpret_cast<double *>(smem);  // [EB][21]
  double *sZF = sEd + C::EB * kEdgeRec;            // [EB][NZ][9]
  double *sXF = sZF + C::EB * C::NZ * kZf;         // [EB][NAB][3]
  int *sSt = reinterpret_cast<int *>(sXF + C::EB * C::NAB * kXf);
  const int tid = threadIdx.x;
  const int64_t e0 = (int64_t)blockIdx.x * C::EB;
  const int nb = a.n - e0 < C::EB ? (int)(a.n - e0) : C::EB;

  for (int le = tid; le < nb; le += kTermsThreads) {
    double X[C::NV * 3];
    int st = 0;
#pragma unroll
    for (int k = 0; k < C::NV * 3; k++) {
      X[k] = a.coords[(e0 + le) * (C::NV * 3) + k];
      if (!isfinite(X[k])) st = FEM_ST_NONFINITE;
    }
    edge_record<ELEM>(X, sEd + le * kEdgeRec);
    sSt[le] = st;
  }
  __syncthreads();
  if constexpr (ELEM == FEM_PRISM6) {
    for (int idx = tid; idx < nb * (C::NZ + C::NAB); idx += kTermsThreads) {
      const int le = idx / (C::NZ + C::NAB), r = idx % (C::NZ + C::NAB);
      const double *ed = sEd + le * kEdgeRec;
      if (r < C::NZ)
        prism_zf(ed, a.qp[4 * (r * C::NAB) + 2], sZF + (le * C::NZ + r) * kZf);
      else
        prism_xf(ed, a.qp[4 * (r - C::NZ)], a.qp[4 * (r - C::NZ) + 1], sXF + (le * C::NAB + r - C::NZ) * kXf);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nb * C::NQ; idx += kTermsThreads) {
    const int le = idx / C::NQ, q = idx % C::NQ;
    double adj[3][3], det;
    if constexpr (ELEM == FEM_PRISM6) {
      const int iz = q / C::NAB, iab = q % C::NAB;
      det = jac_adj_tp(sZF + (le * C::NZ + iz) * kZf, sXF + (le * C::NAB + iab) * kXf, adj);
    } else {
      det = jac_adj_edges<ELEM>(sEd + le * kEdgeRec, a.qp + 4 * q, adj);
    }
    if (!(det > 0.0)) atomicOr(&sSt[le], FEM_ST_DET);
    const double r = 1.0 / det;
    // 80-byte record = five 16-byte stores; consecutive threads write consecutive records
    double2 *dst = reinterpret_cast<double2 *>(a.terms + ((size_t)(e0 + le) * C::NQ + q) * 10);
    dst[0] = make_double2(det, adj[0][0] * r);
    dst[1] = make_double2(adj[0][1] * r, adj[0][2] * r);
    dst[2] = make_double2(adj[1][0] * r, adj[1][1] * r);
    dst[3] = make_double2(adj[1][2] * r, adj[2][0] * r);
    dst[4] = make_double2(adj[2][1] * r, adj[2][2] * r);
  }
  __syncthreads();
  if (a.status)
    for (int le = tid; le < nb; le += kTermsThreads) a.status[e0 + le] = sSt[le];
}

template <int ELEM, int P>
static int launch_terms_cfg(const TermsArgs &a, cudaStream_t s) {
  using C = TermsCfg<ELEM, P>;
  const int64_t grid = (a.n + C::EB - 1) / C::EB;
  if (grid > 0x7fffffffLL) {
    set_error("fem_jacobian_terms: too many elements for one launch");
    return FEM_EINVAL;
  }
  terms_kernel<ELEM, P><<<(unsigned)grid, kTermsThreads, C::SMEM, s>>>(a);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) {
    set_error(std::string("terms_kernel launch: ") + cudaGetErrorString(err));
    return FEM_ECUDA;
  }
  return FEM_OK;
}

}  // namespace fem

using namespace fem;

extern "C" int fem_jacobian_terms(fem_tables t, int p, int64_t n_elem, const double *coords, double *terms,
                                  int32_t *status, void *stream) {
  if (rule_check(t, "fem_jacobian_terms") != FEM_OK) return FEM_EUNSUPPORTED;
  if (!t) {
    set_error("fem_jacobian_terms: tables handle is NULL");
    return FEM_EINVAL;
  }
  if (p < t->p_min || p > t->p_max || n_elem < 0) {
    set_error("fem_jacobian_terms: degree not in the tables or n_elem < 0");
    return FEM_EINVAL;
  }
  if (n_elem == 0) return FEM_OK;
  if (!coords || !terms) {
    set_error("fem_jacobian_terms: NULL coords or terms");
    return FEM_EINVAL;
  }
  if (((uintptr_t)coords & 7) || ((uintptr_t)terms & 15) || ((uintptr_t)status & 3)) {
    set_error("fem_jacobian_terms: coords not 8-byte, terms not 16-byte or status not 4-byte aligned");
    return FEM_EINVAL;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) {
    set_error("fem_jacobian_terms: tables live on another device");
    return FEM_EINVAL;
  }
  TermsArgs a{n_elem, coords, t->tab[p].qp, terms, status};
  const cudaStream_t s = (cudaStream_t)stream;
  if (t->elem == FEM_TET4) return launch_terms_cfg<FEM_TET4, 1>(a, s);
  switch (p) {
    case 1: return launch_terms_cfg<FEM_PRISM6, 1>(a, s);
    case 2: return launch_terms_cfg<FEM_PRISM6, 2>(a, s);
    case 3: return launch_terms_cfg<FEM_PRISM6, 3>(a, s);
    case 4: return launch_terms_cfg<FEM_PRISM6, 4>(a, s);
    case 5: return launch_terms_cfg<FEM_PRISM6, 5>(a, s);
    case 6: return launch_terms_cfg<FEM_PRISM6, 6>(a, s);
    case 7: return launch_terms_cfg<FEM_PRISM6, 7>(a, s);
  }
  set_error("fem_jacobian_terms: degree out of range");
  return FEM_EINVAL;
}
