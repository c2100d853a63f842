// C ABI entry points: argument validation, table management and dispatch.
//
// Host-side responsibilities follow the paper's host code (Section 4.2): the
// element data stay in caller-owned device memory, the reference tables are
// built once per degree and kept resident, the launch shape is derived from
// the degree, and the output is left on the device for the caller (the
// "second alternative" of Section 4.2).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "fem_internal.h"

namespace fem {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

static int cuda_fail(const char *what, cudaError_t e) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return FEM_ECUDA;
}

static int invalid(const char *what) {
  set_error(what);
  return FEM_EINVAL;
}

static void free_table(DevTable &d) {
  if (d.qp) cudaFree(d.qp);
  if (d.phi64) cudaFree(d.phi64);
  if (d.phi32) cudaFree(d.phi32);
  if (d.phiT64) cudaFree(d.phiT64);
  if (d.phiT32) cudaFree(d.phiT32);
  if (d.phiq32) cudaFree(d.phiq32);
  if (d.sf64) cudaFree(d.sf64);
  if (d.sf32) cudaFree(d.sf32);
  if (d.img_bf16) cudaFree(d.img_bf16);
  if (d.img_f16) cudaFree(d.img_f16);
  d = DevTable();
}

static void free_tables(fem_tables t) {
  if (t->mixed) fem_plan_destroy(t->mixed);
  t->mixed = nullptr;
  for (int p = 0; p <= kMaxP; p++) free_table(t->tab[p]);
  if (t->d_err) cudaFree(t->d_err);
  t->d_err = nullptr;
  if (t->d_red) cudaFree(t->d_red);
  t->d_red = nullptr;
  for (int i = 0; i < 2; i++) {
    if (t->stage[i]) cudaFree(t->stage[i]);
    if (t->hs[i]) cudaStreamDestroy(t->hs[i]);
    t->stage[i] = nullptr;
    t->hs[i] = nullptr;
  }
}

// OR of the status words and number of elements with an error bit (every
// bit but the informational FEM_ST_FALLBACK); red[0] = OR, red[1] = count.
__global__ void status_reduce_kernel(const int32_t *__restrict__ st, int64_t n, unsigned long long *red) {
  unsigned bits = 0, cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned v = (unsigned)st[i];
    bits |= v;
    cnt += (v & ~(unsigned)FEM_ST_FALLBACK) != 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    bits |= __shfl_xor_sync(0xffffffffu, bits, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (bits) atomicOr(&red[0], (unsigned long long)bits);
    if (cnt) atomicAdd(&red[1], (unsigned long long)cnt);
  }
}

template <class T>
static int upload(T **dst, const T *src, size_t n) {
  cudaError_t e = cudaMalloc((void **)dst, n * sizeof(T));
  if (e != cudaSuccess) {
    *dst = nullptr;
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return FEM_ENOMEM;
  }
  e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail("cudaMemcpy", e);
  return FEM_OK;
}

}  // namespace fem

using namespace fem;

extern "C" {

const char *fem_status_str(int s) {
  switch (s) {
    case FEM_OK: return "ok";
    case FEM_EINVAL: return "invalid argument";
    case FEM_ENOMEM: return "out of memory";
    case FEM_ECUDA: return "CUDA error";
    case FEM_EUNSUPPORTED: return "unsupported combination";
    case FEM_EELEMENT: return "element flagged";
    case FEM_ETIMEOUT: return "device wait timed out";
    case FEM_ECHECKED: return "kernel index check failed (checked build)";
  }
  return "unknown status";
}

const char *fem_last_error(void) { return g_last_error.c_str(); }

int64_t fem_matrix_size(int elem, int p, int layout) {
  if (elem == FEM_TET4 ? p != 1 : (elem != FEM_PRISM6 || p < 1 || p > kMaxP)) return -1;
  const int64_t ns = ns_of(elem, p);
  if (layout == FEM_OUT_FULL) return ns * ns;
  if (layout == FEM_OUT_SYMPACKED) return ns * (ns + 1) / 2;
  return -1;
}

int fem_reference_rule(int elem, int p, int *nq, int *ns, double *xi, double *w, double *phi) {
  return fem_reference_rule_ex(elem, FEM_RULE_COLLAPSED, p, nq, ns, xi, w, phi);
}

int fem_reference_rule_ex(int elem, int rule, int p, int *nq, int *ns, double *xi, double *w, double *phi) {
  HostRule r;
  if (!build_host_rule(elem, p, &r, rule))
    return invalid("fem_reference_rule: unknown element, rule or degree");
  if (nq) *nq = r.nq;
  if (ns) *ns = r.ns;
  if (xi) std::memcpy(xi, r.xi.data(), r.xi.size() * sizeof(double));
  if (w) std::memcpy(w, r.w.data(), r.w.size() * sizeof(double));
  if (phi) std::memcpy(phi, r.phi.data(), r.phi.size() * sizeof(double));
  return FEM_OK;
}

int fem_tables_build(int elem, int p_min, int p_max, fem_tables *out) {
  return fem_tables_build_ex(elem, FEM_RULE_COLLAPSED, p_min, p_max, out);
}

int fem_tables_build_ex(int elem, int rule, int p_min, int p_max, fem_tables *out) {
  if (!out) return invalid("fem_tables_build: out is NULL");
  *out = nullptr;
  if (elem == FEM_TET4) {
    if (p_min != 1 || p_max != 1) return invalid("fem_tables_build: tetrahedra have p = 1 only");
    if (rule != FEM_RULE_COLLAPSED) return invalid("fem_tables_build: tetrahedra have the 4-point rule only");
  } else if (elem != FEM_PRISM6 || p_min < 1 || p_max > kMaxP || p_min > p_max) {
    return invalid("fem_tables_build: bad element type or degree range");
  }
  if (rule != FEM_RULE_COLLAPSED && rule != FEM_RULE_TABLE1) return invalid("fem_tables_build: unknown rule");
  fem_tables t = new (std::nothrow) fem_tables_s();
  if (!t) return FEM_ENOMEM;
  t->elem = elem;
  t->rule = rule;
  t->p_min = p_min;
  t->p_max = p_max;
  cudaGetDevice(&t->device);
  int rc = FEM_OK;
  for (int p = p_min; p <= p_max && rc == FEM_OK; p++) {
    HostRule r;
    if (!build_host_rule(elem, p, &r, rule)) {
      rc = invalid("fem_tables_build: the rule's reference data failed its exactness check");
      break;
    }
    DevTable &d = t->tab[p];
    d.p = p;
    d.ns = r.ns;
    d.nq = r.nq;
    d.rule = rule;
    std::vector<double> qp(4 * (size_t)r.nq);
    for (int q = 0; q < r.nq; q++) {
      qp[4 * q + 0] = r.xi[3 * q + 0];
      qp[4 * q + 1] = r.xi[3 * q + 1];
      qp[4 * q + 2] = r.xi[3 * q + 2];
      qp[4 * q + 3] = r.w[q];
    }
    std::vector<float> phi32(r.phi.size());
    for (size_t i = 0; i < r.phi.size(); i++) phi32[i] = (float)r.phi[i];
    std::vector<double> phiT64(r.phi.size());
    std::vector<float> phiT32(r.phi.size()), phiq32(r.phi.size());
    for (int q = 0; q < r.nq; q++)
      for (int dd = 0; dd < 4; dd++)
        for (int i = 0; i < r.ns; i++) {
          const size_t src = ((size_t)(4 * q + dd)) * r.ns + i, dst = ((size_t)i * r.nq + q) * 4 + dd;
          phiT64[dst] = r.phi[src];
          phiT32[dst] = phi32[src];
          phiq32[((size_t)q * r.ns + i) * 4 + dd] = phi32[src];
        }
    rc = upload(&d.qp, qp.data(), qp.size());
    if (rc == FEM_OK) rc = upload(&d.phi64, r.phi.data(), r.phi.size());
    if (rc == FEM_OK) rc = upload(&d.phi32, phi32.data(), phi32.size());
    if (rc == FEM_OK) rc = upload(&d.phiT64, phiT64.data(), phiT64.size());
    if (rc == FEM_OK) rc = upload(&d.phiT32, phiT32.data(), phiT32.size());
    if (rc == FEM_OK) rc = upload(&d.phiq32, phiq32.data(), phiq32.size());
    if (rc == FEM_OK && elem == FEM_PRISM6) {
      double mx = 0.0;
      for (double v : r.phi) mx = std::fmax(mx, std::fabs(v));
      int ex = 0;
      std::frexp(mx, &ex);  // mx < 2^ex
      if (rule == FEM_RULE_COLLAPSED) {  // 1D factors of the collapsed rule (operator apply)
        std::vector<double> sf;
        build_sf_tables(p, sf);
        std::vector<float> sf32(sf.begin(), sf.end());
        rc = upload(&d.sf64, sf.data(), sf.size());
        if (rc == FEM_OK) rc = upload(&d.sf32, sf32.data(), sf32.size());
      }
      d.phimax = (float)mx;
      d.aphi_f16 = 14 - ex;  // scaled magnitudes below 2^14
      std::vector<uint16_t> img;
      build_tc_image(p, rule, r.phi, false, 0, img);
      if (rc == FEM_OK) rc = upload(&d.img_bf16, img.data(), img.size());
      if (rc == FEM_OK) {
        build_tc_image(p, rule, r.phi, true, d.aphi_f16, img);
        rc = upload(&d.img_f16, img.data(), img.size());
      }
    }
  }
  if (rc == FEM_OK) {
    cudaError_t e = cudaMalloc((void **)&t->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(t->d_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&t->d_red, 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) rc = cuda_fail("cudaMalloc(error word)", e);
  }
  if (rc != FEM_OK) {
    free_tables(t);
    delete t;
    return rc;
  }
  *out = t;
  return FEM_OK;
}

int fem_tables_destroy(fem_tables t) {
  if (!t) return FEM_OK;
  free_tables(t);
  delete t;
  return FEM_OK;
}

int fem_debug_stall_next(fem_tables t) {
  if (!t) return invalid("fem_debug_stall_next: tables handle is NULL");
  t->stall_next = 1;
  return FEM_OK;
}

int fem_error_flag(fem_tables t, int clear) {
  if (!t || !t->d_err) return invalid("fem_error_flag: tables handle is NULL");
  int h = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, t->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && clear) e = cudaMemset(t->d_err, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail("fem_error_flag", e);
  if (h & kErrTimeout) return FEM_ETIMEOUT;
  if (h & kErrCheck) {
    set_error("fem_error_flag: a kernel index check of the checked build failed");
    return FEM_ECHECKED;
  }
  return FEM_OK;
}

int fem_integrate(fem_tables t, int64_t n_elem, const double *coords, const int8_t *p_per_elem,
                  int p_uniform, const double *coeffs, int64_t coeff_stride, const fem_coef_law *law,
                  int prec, int layout, void *A_out, void *b_out, int32_t *status, void *stream) {
  if (!t) return invalid("fem_integrate: tables handle is NULL");
  const int lw = law ? law->law : 0;
  if (lw != 0 && lw != FEM_LAW_EXACT && lw != FEM_LAW_MLP) return invalid("fem_integrate: unknown coefficient law");
  if (!p_per_elem) {
    if (lw == 0)
      return fem_integrate_uniform(t, p_uniform, n_elem, coords, coeffs, coeff_stride, prec, layout, A_out, b_out,
                                   status, stream);
    return integrate_law_opts(t, p_uniform, n_elem, coords, coeffs, coeff_stride, law->ucoef, lw, law->mlp,
                              law->newton_steps > 0 ? law->newton_steps : 8, law->hw_tanh, prec, layout, A_out,
                              b_out, status, stream);
  }
  if (lw != 0) {
    set_error("fem_integrate: a coefficient law needs a uniform degree (p_per_elem = NULL)");
    return FEM_EUNSUPPORTED;
  }
  return integrate_mixed_cached(t, n_elem, p_per_elem, coords, coeffs, coeff_stride, prec, layout, A_out, b_out,
                                status, stream);
}

int fem_integrate_uniform(fem_tables t, int p, int64_t n_elem, const double *coords, const double *coeffs,
                          int64_t coeff_stride, int prec, int layout, void *A_out, void *b_out,
                          int32_t *status, void *stream) {
  if (!t) return invalid("fem_integrate: tables handle is NULL");
  if (p < t->p_min || p > t->p_max) return invalid("fem_integrate: degree not in the tables");
  if (n_elem < 0) return invalid("fem_integrate: n_elem < 0");
  if (prec < FEM_F64 || prec > FEM_F16X3) return invalid("fem_integrate: unknown precision");
  if (layout != FEM_OUT_FULL && layout != FEM_OUT_SYMPACKED) return invalid("fem_integrate: unknown layout");
  if (n_elem == 0) return FEM_OK;
  if (!coords || !coeffs || !A_out) return invalid("fem_integrate: NULL coords, coeffs or A_out");
  if (coeff_stride < n_elem) return invalid("fem_integrate: coeff_stride < n_elem");
  if (((uintptr_t)coords | (uintptr_t)coeffs) & 7) return invalid("fem_integrate: coords/coeffs not 8-byte aligned");
  if ((uintptr_t)A_out & 15) return invalid("fem_integrate: A_out not 16-byte aligned");
  const size_t osz = prec == FEM_F64 ? 8 : 4;
  if (b_out && ((uintptr_t)b_out & (osz - 1))) return invalid("fem_integrate: b_out misaligned");
  if (status && ((uintptr_t)status & 3)) return invalid("fem_integrate: status misaligned");
  const DevTable &d = t->tab[p];
  FmaArgs a;
  a.n = n_elem;
  a.coords = coords;
  a.coeffs = coeffs;
  a.cstride = coeff_stride;
  a.qp = d.qp;
  a.A = A_out;
  a.b = b_out;
  a.status = status;
  a.layout = layout;
  a.err = t->d_err;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) return invalid("fem_integrate: tables live on another device");
  const bool t1 = t->rule == FEM_RULE_TABLE1;
  switch (prec) {
    case FEM_F64:
      a.phi = d.phi64;
      return t1 ? launch_fma_t1_f64(p, a, stream) : launch_fma_f64(t->elem, p, a, stream);
    case FEM_F32:
      a.phi = d.phi32;
      return t1 ? launch_fma_t1_f32(p, a, stream) : launch_fma_f32(t->elem, p, a, stream);
    default: {
      if (t->elem != FEM_PRISM6) {
        set_error("fem_integrate: tensor-core precisions are provided for prisms only");
        return FEM_EUNSUPPORTED;
      }
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
      l.stall = t->stall_next;
      t->stall_next = 0;
      return launch_tc(p, prec == FEM_F16X3, d, l, stream);
    }
  }
}

int fem_sync_status(fem_tables t, const int32_t *status, int64_t n_elem, int32_t *bits, int64_t *nflag,
                    void *stream) {
  if (!t || !t->d_red) return invalid("fem_sync_status: tables handle is NULL");
  if (n_elem < 0 || (n_elem > 0 && !status)) return invalid("fem_sync_status: bad n_elem or NULL status");
  if ((uintptr_t)status & 3) return invalid("fem_sync_status: status misaligned");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) return invalid("fem_sync_status: tables live on another device");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long h[2] = {0, 0};
  int herr = 0;
  cudaError_t e = cudaMemsetAsync(t->d_red, 0, 2 * sizeof(unsigned long long), s);
  if (e == cudaSuccess && n_elem > 0) {
    const int grid = (int)std::min<int64_t>((n_elem + 255) / 256, 4 * 152);
    status_reduce_kernel<<<grid, 256, 0, s>>>(status, n_elem, t->d_red);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, t->d_red, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, t->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail("fem_sync_status", e);
  if (bits) *bits = (int32_t)h[0];
  if (nflag) *nflag = (int64_t)h[1];
  if (herr) {
    set_error("fem_sync_status: a bounded device wait expired");
    return FEM_ETIMEOUT;
  }
  if (h[1]) {
    set_error("fem_sync_status: " + std::to_string(h[1]) + " element(s) flagged in status[]");
    return FEM_EELEMENT;
  }
  return FEM_OK;
}

int fem_apply(fem_tables t, int p, int64_t n_elem, const double *coords, const double *coeffs,
              int64_t coeff_stride, int prec, const void *x, void *y, int32_t *status, void *stream) {
  if (rule_check(t, "fem_apply") != FEM_OK) return FEM_EUNSUPPORTED;
  if (!t) return invalid("fem_apply: tables handle is NULL");
  if (p < t->p_min || p > t->p_max) return invalid("fem_apply: degree not in the tables");
  if (n_elem < 0) return invalid("fem_apply: n_elem < 0");
  if (prec < FEM_F64 || prec > FEM_F16X3) return invalid("fem_apply: unknown precision");
  if (prec != FEM_F64 && prec != FEM_F32) {
    set_error("fem_apply: FEM_F64 and FEM_F32 only");
    return FEM_EUNSUPPORTED;
  }
  if (n_elem == 0) return FEM_OK;
  if (!coords || !coeffs || !x || !y) return invalid("fem_apply: NULL coords, coeffs, x or y");
  if (coeff_stride < n_elem) return invalid("fem_apply: coeff_stride < n_elem");
  if (((uintptr_t)coords | (uintptr_t)coeffs) & 7) return invalid("fem_apply: coords/coeffs not 8-byte aligned");
  const uintptr_t osz = prec == FEM_F64 ? 8 : 4;
  if (((uintptr_t)x | (uintptr_t)y) & (osz - 1)) return invalid("fem_apply: x or y misaligned");
  if (status && ((uintptr_t)status & 3)) return invalid("fem_apply: status misaligned");
  const DevTable &d = t->tab[p];
  const size_t bytes = (size_t)n_elem * d.ns * osz;
  const uintptr_t xa = (uintptr_t)x, ya = (uintptr_t)y;
  if (xa < ya + bytes && ya < xa + bytes) return invalid("fem_apply: x and y overlap");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) return invalid("fem_apply: tables live on another device");
  ApplyArgs a;
  a.n = n_elem;
  a.coords = coords;
  a.coeffs = coeffs;
  a.cstride = coeff_stride;
  a.qp = d.qp;
  if (t->elem == FEM_PRISM6)
    a.tab = prec == FEM_F64 ? (const void *)d.sf64 : (const void *)d.sf32;
  else
    a.tab = prec == FEM_F64 ? (const void *)d.phi64 : (const void *)d.phi32;
  a.x = x;
  a.y = y;
  a.status = status;
  return launch_apply(t->elem, p, prec == FEM_F32, a, stream);
}

int fem_integrate_elastic(fem_tables t, int p, int64_t n_elem, const double *coords, const double *coeffs,
                          int64_t coeff_stride, int prec, void *A_out, void *b_out, int32_t *status,
                          void *stream) {
  if (!t || t->elem != FEM_PRISM6) return invalid("fem_integrate_elastic: needs prism tables");
  if (p < t->p_min || p > t->p_max || n_elem < 0) return invalid("fem_integrate_elastic: bad degree or n_elem");
  if (prec != FEM_F64 && prec != FEM_F32 && prec != FEM_BF16X3 && prec != FEM_F16X3) {
    set_error("fem_integrate_elastic: unknown precision");
    return FEM_EUNSUPPORTED;
  }
  if (n_elem == 0) return FEM_OK;
  if (!coords || !coeffs || !A_out || coeff_stride < n_elem)
    return invalid("fem_integrate_elastic: NULL buffer or coeff_stride < n_elem");
  if ((((uintptr_t)coords | (uintptr_t)coeffs) & 7) || ((uintptr_t)A_out & 15))
    return invalid("fem_integrate_elastic: misaligned buffer");
  if (9 * n_elem > 0x7fffffffLL * 4) return invalid("fem_integrate_elastic: too many elements");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) return invalid("fem_integrate_elastic: tables live on another device");
  const DevTable &d = t->tab[p];
  if (prec == FEM_BF16X3 || prec == FEM_F16X3) {
    TcLaunch l;
    l.n = n_elem;
    l.coords = coords;
    l.coeffs = coeffs;
    l.cstride = coeff_stride;
    l.A = A_out;
    l.b = b_out;
    l.status = status;
    l.layout = FEM_OUT_FULL;
    l.err = t->d_err;
    l.stall = t->stall_next;
    l.elastic = 1;
    t->stall_next = 0;
    return launch_tc(p, prec == FEM_F16X3, d, l, stream);
  }
  FmaArgs a;
  a.n = n_elem;
  a.coords = coords;
  a.coeffs = coeffs;
  a.cstride = coeff_stride;
  a.qp = d.qp;
  a.phi = prec == FEM_F64 ? (const void *)d.phi64 : (const void *)d.phi32;
  a.A = A_out;
  a.b = b_out;
  a.status = status;
  a.layout = FEM_OUT_FULL;
  a.err = t->d_err;
  if (t->rule == FEM_RULE_TABLE1)
    return prec == FEM_F64 ? launch_fma_t1_elastic_f64(p, a, stream) : launch_fma_t1_elastic_f32(p, a, stream);
  return prec == FEM_F64 ? launch_fma_elastic_f64(p, a, stream) : launch_fma_elastic_f32(p, a, stream);
}

int fem_integrate_terms(fem_tables t, int p, int64_t n_elem, const double *terms, const double *coeffs,
                        int64_t coeff_stride, int prec, int layout, void *A_out, void *b_out,
                        int32_t *status, void *stream) {
  if (rule_check(t, "fem_integrate_terms") != FEM_OK) return FEM_EUNSUPPORTED;
  if (!t) return invalid("fem_integrate_terms: tables handle is NULL");
  if (p < t->p_min || p > t->p_max || n_elem < 0) return invalid("fem_integrate_terms: bad degree or n_elem");
  if (prec != FEM_F64 && prec != FEM_F32) {
    set_error("fem_integrate_terms: FEM_F64 or FEM_F32 only");
    return FEM_EUNSUPPORTED;
  }
  if (layout != FEM_OUT_FULL && layout != FEM_OUT_SYMPACKED) return invalid("fem_integrate_terms: unknown layout");
  if (n_elem == 0) return FEM_OK;
  if (!terms || !coeffs || !A_out) return invalid("fem_integrate_terms: NULL terms, coeffs or A_out");
  if (coeff_stride < n_elem) return invalid("fem_integrate_terms: coeff_stride < n_elem");
  if (((uintptr_t)terms | (uintptr_t)coeffs) & 7) return invalid("fem_integrate_terms: terms/coeffs not 8-byte aligned");
  if ((uintptr_t)A_out & 15) return invalid("fem_integrate_terms: A_out not 16-byte aligned");
  const size_t osz = prec == FEM_F64 ? 8 : 4;
  if (b_out && ((uintptr_t)b_out & (osz - 1))) return invalid("fem_integrate_terms: b_out misaligned");
  if (status && ((uintptr_t)status & 3)) return invalid("fem_integrate_terms: status misaligned");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) return invalid("fem_integrate_terms: tables live on another device");
  const DevTable &d = t->tab[p];
  FmaArgs a;
  a.n = n_elem;
  a.coords = nullptr;
  a.terms = terms;
  a.coeffs = coeffs;
  a.cstride = coeff_stride;
  a.qp = d.qp;
  a.A = A_out;
  a.b = b_out;
  a.status = status;
  a.layout = layout;
  a.err = t->d_err;
  a.phi = prec == FEM_F64 ? (const void *)d.phi64 : (const void *)d.phi32;
  return launch_fma_terms(t->elem, p, prec, a, stream);
}

int fem_integrate_elastic_terms(fem_tables t, int p, int64_t n_elem, const double *terms, const double *coeffs,
                                int64_t coeff_stride, int prec, void *A_out, void *b_out, int32_t *status,
                                void *stream) {
  if (rule_check(t, "fem_integrate_elastic_terms") != FEM_OK) return FEM_EUNSUPPORTED;
  if (!t || t->elem != FEM_PRISM6) return invalid("fem_integrate_elastic_terms: needs prism tables");
  if (p < t->p_min || p > t->p_max || n_elem < 0) return invalid("fem_integrate_elastic_terms: bad degree or n_elem");
  if (prec != FEM_F64 && prec != FEM_F32) {
    set_error("fem_integrate_elastic_terms: FP64 or FP32 only");
    return FEM_EUNSUPPORTED;
  }
  if (n_elem == 0) return FEM_OK;
  if (!terms || !coeffs || !A_out || coeff_stride < n_elem)
    return invalid("fem_integrate_elastic_terms: NULL buffer or coeff_stride < n_elem");
  if ((((uintptr_t)terms | (uintptr_t)coeffs) & 7) || ((uintptr_t)A_out & 15))
    return invalid("fem_integrate_elastic_terms: misaligned buffer");
  if (9 * n_elem > 0x7fffffffLL * 4) return invalid("fem_integrate_elastic_terms: too many elements");
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) return invalid("fem_integrate_elastic_terms: tables live on another device");
  const DevTable &d = t->tab[p];
  FmaArgs a;
  a.n = n_elem;
  a.coords = nullptr;
  a.terms = terms;
  a.coeffs = coeffs;
  a.cstride = coeff_stride;
  a.qp = d.qp;
  a.phi = prec == FEM_F64 ? (const void *)d.phi64 : (const void *)d.phi32;
  a.A = A_out;
  a.b = b_out;
  a.status = status;
  a.layout = FEM_OUT_FULL;
  a.err = t->d_err;
  return launch_fma_elastic_terms(p, prec, a, stream);
}

int fem_integrate_host(fem_tables t, int p, int64_t n_elem, const double *coords, const double *coeffs,
                       int64_t coeff_stride, int prec, int layout, void *A_out, void *b_out, int32_t *status,
                       int64_t chunk) {
  if (!t) return invalid("fem_integrate_host: tables handle is NULL");
  if (p < t->p_min || p > t->p_max || n_elem < 0) return invalid("fem_integrate_host: bad degree or n_elem");
  if (n_elem == 0) return FEM_OK;
  if (!coords || !coeffs || !A_out || coeff_stride < n_elem)
    return invalid("fem_integrate_host: NULL buffer or coeff_stride < n_elem");
  const int64_t m = fem_matrix_size(t->elem, p, layout);
  if (m < 0) return invalid("fem_integrate_host: unknown layout");
  const int nv = nv_of(t->elem), ns = ns_of(t->elem, p);
  const size_t osz = prec == FEM_F64 ? 8 : 4;
  // per element: coords, 11 coefficients, A, b, status; staging rounded to 256 B per array
  const size_t per = (size_t)nv * 3 * 8 + 11 * 8 + (size_t)m * osz + (size_t)ns * osz + 4;
  if (chunk <= 0) chunk = std::max<int64_t>(1, (int64_t)((size_t)256 << 20) / (int64_t)per);
  if (chunk > n_elem) chunk = n_elem;
  const size_t need = (size_t)chunk * per + 5 * 256;
  if (t->stage_bytes < need) {
    // at least the default chunk's 256 MB, so that calls of other degrees
    // (other per-element sizes) reuse the slots: a reallocation frees the
    // old slots, which synchronises the device
    const size_t alloc = std::max(need, ((size_t)256 << 20) + 5 * 256);
    for (int i = 0; i < 2; i++) {
      if (t->stage[i]) cudaFree(t->stage[i]);
      t->stage[i] = nullptr;
      cudaError_t e = cudaMalloc((void **)&t->stage[i], alloc);
      if (e != cudaSuccess) {
        t->stage_bytes = 0;
        return cuda_fail("fem_integrate_host: staging allocation", e);
      }
    }
    t->stage_bytes = alloc;
  }
  for (int i = 0; i < 2; i++)
    if (!t->hs[i]) {
      cudaError_t e = cudaStreamCreateWithFlags(&t->hs[i], cudaStreamNonBlocking);
      if (e != cudaSuccess) return cuda_fail("fem_integrate_host: stream", e);
    }
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t oX = 0, oC = al(oX + (size_t)chunk * nv * 3 * 8), oA = al(oC + (size_t)chunk * 11 * 8),
               oB = al(oA + (size_t)chunk * m * osz), oS = al(oB + (size_t)chunk * ns * osz);
  int rc = FEM_OK;
  int64_t k = 0;
  for (int64_t e0 = 0; e0 < n_elem && rc == FEM_OK; e0 += chunk, k++) {
    const int64_t c = std::min<int64_t>(chunk, n_elem - e0);
    const int slot = (int)(k & 1);
    cudaStream_t s = t->hs[slot];
    unsigned char *st = t->stage[slot];
    double *dX = reinterpret_cast<double *>(st + oX);
    double *dC = reinterpret_cast<double *>(st + oC);
    // the slot's previous chunk finished its copies before these are queued (same stream)
    cudaError_t e = cudaMemcpyAsync(dX, coords + e0 * nv * 3, (size_t)c * nv * 3 * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(dC, (size_t)c * 8, coeffs + e0, (size_t)coeff_stride * 8, (size_t)c * 8, 11,
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      rc = cuda_fail("fem_integrate_host: copy in", e);
      break;
    }
    rc = fem_integrate_uniform(t, p, c, dX, dC, c, prec, layout, st + oA, b_out ? st + oB : nullptr,
                               status ? reinterpret_cast<int32_t *>(st + oS) : nullptr, s);
    if (rc != FEM_OK) break;
    e = cudaMemcpyAsync(static_cast<unsigned char *>(A_out) + (size_t)e0 * m * osz, st + oA, (size_t)c * m * osz,
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && b_out)
      e = cudaMemcpyAsync(static_cast<unsigned char *>(b_out) + (size_t)e0 * ns * osz, st + oB, (size_t)c * ns * osz,
                          cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && status)
      e = cudaMemcpyAsync(status + e0, st + oS, (size_t)c * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) rc = cuda_fail("fem_integrate_host: copy out", e);
  }
  for (int i = 0; i < 2; i++) {
    cudaError_t e = cudaStreamSynchronize(t->hs[i]);
    if (e != cudaSuccess && rc == FEM_OK) rc = cuda_fail("fem_integrate_host: synchronize", e);
  }
  return rc;
}

}  // extern "C"
