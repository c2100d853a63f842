// Matrix-free application of the element operators, y_e = A_e x_e, without
// forming A_e.
//
// The element matrix of the weak form is a sum over quadrature points of
// Phi^T G_Q Phi (the G-form of the integration kernels: Phi the 4 NQ x NS
// table of values and reference derivatives, G_Q the 4x4 point matrix that
// folds geometry, weight and coefficients), so
//     y = sum_Q Phi_Q^T (G_Q (Phi_Q x)):
// evaluate the field and its reference gradient at the points, apply G_Q per
// point, and test against the basis.  This is the element-level product that
// an iterative solver of the assembled system performs with the element
// matrices kept in device memory (Section 4), and the high-order alternative
// to forming them that Section 3 points to: 16 NQ NS flops per element
// instead of 8 NQ NS^2 for A_e.
//
// Prisms use sum factorisation in all three directions.  The basis function
// of DOF t + NT k is psi_t(a, b) L_k(zeta) with the Dubiner function
// psi_(i,j) = P_i(a) h(b)^i Q_j(b) in collapsed coordinates, and the rule is a
// tensor product of Gauss rules in a, b and zeta (point iz NAB + ia N + ib),
// so every table entry is a product of 1D factors (build_sf_tables) and the
// field at the points follows from three small contractions per direction:
//   zeta:  W[iz][t] = sum_k L[iz][k] x[k][t]   (and Wd with L'),
//   b:     G[i] = sum_j B[t(i,j)][ib] W[iz][t(i,j)]   per (iz, ib), for the
//          factors Bq, Bx, By of the value and the two triangle derivatives,
//   a:     u = sum_i P[ia][i] G[i]   per point (Pa, Px, Pe),
// then the point stage v = G_Q u (FP64 adj J and det J from the element's
// tensor-product geometry factors), and the transposed contractions in
// reverse order give y.  Per element that is 4 N NS + 2 N (4 N NT + 5 N^3)
// multiply-adds plus about 60 FP64 operations per point: at p = 7 about 100k
// FP64 operations against 170M multiply-adds to form A_e.  The kernel moves
// 2 NS values, 18 coordinates and 11 coefficients per element, so even then
// the FP64 path is bound by GB300's FP64 pipe, not by HBM, at every degree;
// the FP32 path is bound by latency (barriers and shared-memory loads).
//
// Work decomposition: a CTA owns groups of EB elements (grid-stride over the
// groups), keeps the factor tables in shared memory for the whole launch, and
// pipelines the groups: the next group's x, coordinates and coefficients are
// fetched with cp.async while the current one is computed.  Per group five
// phases separated by barriers:
//   A.  element status, geometry factors, zeta contraction;
//   B.  per column (element, iz, ib): b-direction contraction, then for each of
//       the column's N points the a-direction contraction and the point stage;
//   C1. per column: transposed a-direction contraction, in place over v;
//   C2. transposed b-direction contraction;
//   D.  transposed zeta contraction, y written to global memory.
// The FP64 path does everything in FP64.  The FP32 path computes the
// element's geometry factors and det J at every point in FP64 and the rest
// (adj J from the rounded factors, point stage, contractions) in FP32.
//
// P1 tetrahedra (NS = NQ = 4, J constant) use one thread per element.
#include "fem_geometry.cuh"

namespace fem {
namespace {

// Point stage v = G_Q u for the scalar form, without forming G_Q:
// with t = adj^T grad_ref u (= det J times the physical gradient),
//   v[1 + k] = (w / det) (adj D t)[k],   v[0] = w (det c u0 + b . t).
__device__ __forceinline__ void apply_point(const double (&adj)[3][3], double det, double w, const double *cf,
                                            double u0, double u1, double u2, double u3, double (&v)[4]) {
  const double t0 = adj[0][0] * u1 + adj[1][0] * u2 + adj[2][0] * u3;
  const double t1 = adj[0][1] * u1 + adj[1][1] * u2 + adj[2][1] * u3;
  const double t2 = adj[0][2] * u1 + adj[1][2] * u2 + adj[2][2] * u3;
  // cf: Dxx Dyy Dzz Dxy Dxz Dyz bx by bz c
  const double s0 = cf[0] * t0 + cf[3] * t1 + cf[4] * t2;
  const double s1 = cf[3] * t0 + cf[1] * t1 + cf[5] * t2;
  const double s2 = cf[4] * t0 + cf[5] * t1 + cf[2] * t2;
  const double sc = w / det;
  v[1] = sc * (adj[0][0] * s0 + adj[0][1] * s1 + adj[0][2] * s2);
  v[2] = sc * (adj[1][0] * s0 + adj[1][1] * s1 + adj[1][2] * s2);
  v[3] = sc * (adj[2][0] * s0 + adj[2][1] * s1 + adj[2][2] * s2);
  v[0] = w * (det * cf[9] * u0 + cf[6] * t0 + cf[7] * t1 + cf[8] * t2);
}

template <int B>
__device__ __forceinline__ void cp_async(void *sdst, const void *gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gsrc), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

template <int P, class T>
struct ApCfg {
  static constexpr int N = P + 1, NT = N * (N + 1) / 2, NS = NT * N, NAB = N * N, NQ = N * NAB, NP = N | 1;
  static constexpr int NTH = 256;
  static constexpr int EB = NTH / NAB > 1 ? NTH / NAB : 1;  // elements per group: one (level, ib) column per thread
  static constexpr int NGC = 18 + 11;                       // coordinates + coefficients per element
  // factor tables (type T): Pa, Px, Pe [N][N]; Bq, Bx, By [NT][NP]; L, dL [N][N]
  static constexpr int OPA = 0, OPX = N * N, OPE = 2 * N * N, OBQ = 3 * N * N, OBX = OBQ + NT * NP,
                       OBY = OBX + NT * NP, OL = OBY + NT * NP, OD = OL + N * N, NTAB = OD + N * N;
  // shared memory (bytes)
  static constexpr size_t O_TAB = 0;                                          // T [NTAB]
  static constexpr size_t O_WQ = al16(O_TAB + sizeof(T) * NTAB);              // double [NQ] weights (FP64 path)
  static constexpr size_t O_TI = al16(O_WQ + (sizeof(T) == 8 ? sizeof(double) * NQ : 0));  // int [NT]: i of DOF t
  static constexpr size_t O_X = al16(O_TI + sizeof(int) * NT);                // T [2][EB][NS]
  static constexpr size_t O_W = al16(O_X + sizeof(T) * 2 * EB * NS);          // T [EB][2][N][NT]
  static constexpr size_t O_V = al16(O_W + sizeof(T) * EB * 2 * NS);          // T [EB][4][NQ]
  static constexpr size_t O_GC = al16(O_V + sizeof(T) * EB * 4 * NQ);         // double [2][EB][NGC]
  static constexpr size_t O_ZF = al16(O_GC + sizeof(double) * 2 * EB * NGC);  // double [EB][N][9]
  static constexpr size_t O_XF = al16(O_ZF + sizeof(double) * EB * N * kZf);  // double [EB][NAB][3]
  // FP32 path: float copies of the geometry factors, coefficients, weights
  static constexpr size_t O_ZR = al16(O_XF + sizeof(double) * EB * NAB * kXf);// float [EB][N][9]
  static constexpr size_t O_XR = al16(O_ZR + sizeof(float) * EB * N * kZf);   // float [EB][NAB][3]
  static constexpr size_t O_WF = al16(O_XR + sizeof(float) * EB * NAB * kXf); // float [NQ]
  static constexpr size_t O_CF = al16(O_WF + sizeof(float) * NQ);             // float [EB][10]
  static constexpr size_t O_ST = al16(O_CF + sizeof(float) * EB * 10);
  static constexpr size_t SMEM = al16(O_ST + sizeof(int) * EB);
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// Start the asynchronous copies of group g (its x, coordinates, coefficients).
template <class C, class T>
__device__ __forceinline__ void prefetch_group(const ApplyArgs &a, int64_t g, T *sX, double *sGC) {
  const int64_t e0 = g * C::EB;
  const int ne = (int)min((int64_t)C::EB, a.n - e0);
  const T *xg = static_cast<const T *>(a.x) + e0 * C::NS;
  for (int i = threadIdx.x; i < ne * C::NS; i += C::NTH) cp_async<sizeof(T)>(sX + i, xg + i);
  const double *cg = a.coords + e0 * 18;
  for (int i = threadIdx.x; i < ne * 18; i += C::NTH) cp_async<8>(sGC + (i / 18) * C::NGC + i % 18, cg + i);
  for (int i = threadIdx.x; i < ne * 11; i += C::NTH) {
    const int k = i / ne, e = i - k * ne;
    cp_async<8>(sGC + e * C::NGC + 18 + k, a.coeffs + k * a.cstride + e0 + e);
  }
}

// Point stage in the FP32 path: adj J from FP32 copies of the element's
// tensor-product factors (zr: J[:,0], J[:,1] and adj row 2 of the point's
// zeta level; xr: J[:,2] of its triangle point), det J computed in FP64 by the
// caller (its sign sets the status flag), the rest in FP32.
__device__ __forceinline__ void apply_point_f32(const float *zr, const float *xr, float d, float w, const float *cf,
                                                float u0, float u1, float u2, float u3, float (&v)[4]) {
  const float c0x = zr[0], c0y = zr[1], c0z = zr[2], c1x = zr[3], c1y = zr[4], c1z = zr[5];
  const float c2x = xr[0], c2y = xr[1], c2z = xr[2];
  const float a[3][3] = {{c1y * c2z - c1z * c2y, c1z * c2x - c1x * c2z, c1x * c2y - c1y * c2x},
                         {c2y * c0z - c2z * c0y, c2z * c0x - c2x * c0z, c2x * c0y - c2y * c0x},
                         {zr[6], zr[7], zr[8]}};
  const float t0 = a[0][0] * u1 + a[1][0] * u2 + a[2][0] * u3;
  const float t1 = a[0][1] * u1 + a[1][1] * u2 + a[2][1] * u3;
  const float t2 = a[0][2] * u1 + a[1][2] * u2 + a[2][2] * u3;
  const float s0 = cf[0] * t0 + cf[3] * t1 + cf[4] * t2;
  const float s1 = cf[3] * t0 + cf[1] * t1 + cf[5] * t2;
  const float s2 = cf[4] * t0 + cf[5] * t1 + cf[2] * t2;
  const float sc = w / d;
  v[1] = sc * (a[0][0] * s0 + a[0][1] * s1 + a[0][2] * s2);
  v[2] = sc * (a[1][0] * s0 + a[1][1] * s1 + a[1][2] * s2);
  v[3] = sc * (a[2][0] * s0 + a[2][1] * s1 + a[2][2] * s2);
  v[0] = w * (d * cf[9] * u0 + cf[6] * t0 + cf[7] * t1 + cf[8] * t2);
}

template <int P, class T>
__global__ void __launch_bounds__(256) apply_prism_kernel(const ApplyArgs a) {
  using C = ApCfg<P, T>;
  constexpr int N = C::N, NT = C::NT, NS = C::NS, NAB = C::NAB, NQ = C::NQ, NP = C::NP, EB = C::EB;
  constexpr bool F32 = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char smem[];
  T *sTab = reinterpret_cast<T *>(smem + C::O_TAB);
  double *sWq = reinterpret_cast<double *>(smem + C::O_WQ);
  int *sTi = reinterpret_cast<int *>(smem + C::O_TI);
  T *sX = reinterpret_cast<T *>(smem + C::O_X);
  T *sW = reinterpret_cast<T *>(smem + C::O_W);
  T *sV = reinterpret_cast<T *>(smem + C::O_V);
  double *sGC = reinterpret_cast<double *>(smem + C::O_GC);
  double *sZF = reinterpret_cast<double *>(smem + C::O_ZF);
  double *sXF = reinterpret_cast<double *>(smem + C::O_XF);
  float *sZR = reinterpret_cast<float *>(smem + C::O_ZR);
  float *sXR = reinterpret_cast<float *>(smem + C::O_XR);
  float *sWf = reinterpret_cast<float *>(smem + C::O_WF);
  float *sCF = reinterpret_cast<float *>(smem + C::O_CF);
  int *sSt = reinterpret_cast<int *>(smem + C::O_ST);
  const int tid = threadIdx.x;
  const int64_t ngroups = (a.n + EB - 1) / EB;
  int64_t g = blockIdx.x;
  if (g >= ngroups) return;

  const T *tab = static_cast<const T *>(a.tab);
  for (int i = tid; i < C::NTAB; i += C::NTH) sTab[i] = tab[i];
  for (int q = tid; q < NQ; q += C::NTH) {
    if (F32)
      sWf[q] = (float)a.qp[4 * q + 3];
    else
      sWq[q] = a.qp[4 * q + 3];
  }
  if (tid == 0)
    for (int m = 0, t = 0; m < N; m++)
      for (int i = m; i >= 0; i--, t++) sTi[t] = i;
  prefetch_group<C>(a, g, sX, sGC);
  cp_commit();
  const T *sPa = sTab + C::OPA, *sPx = sTab + C::OPX, *sPe = sTab + C::OPE;
  const T *sBq = sTab + C::OBQ, *sBx = sTab + C::OBX, *sBy = sTab + C::OBY;
  const T *sL = sTab + C::OL, *sD = sTab + C::OD;

  for (int it = 0; g < ngroups; g += gridDim.x, it++) {
    const int cur = it & 1;
    cp_wait_all();
    if (g + gridDim.x < ngroups)
      prefetch_group<C>(a, g + gridDim.x, sX + (cur ^ 1) * EB * NS, sGC + (cur ^ 1) * EB * C::NGC);
    cp_commit();
    __syncthreads();
    const int64_t e0 = g * EB;
    const int ne = (int)min((int64_t)EB, a.n - e0);
    const T *X = sX + cur * EB * NS;
    const double *GC = sGC + cur * EB * C::NGC;

    // A. status, geometry factors, zeta contraction W = L x, Wd = L' x
    for (int e = tid; e < ne; e += C::NTH) {
      int st = 0;
      for (int k = 0; k < C::NGC; k++)
        if (!isfinite(GC[e * C::NGC + k])) st = FEM_ST_NONFINITE;
      sSt[e] = st;
      if (F32)
        for (int k = 0; k < 10; k++) sCF[e * 10 + k] = (float)GC[e * C::NGC + 18 + k];
    }
    for (int i = tid; i < ne * N; i += C::NTH) {
      const int e = i / N, iz = i - e * N;
      double ed[kEdgeRec];
      edge_record<FEM_PRISM6>(GC + e * C::NGC, ed);
      double *zf = sZF + i * kZf;
      prism_zf(ed, a.qp[4 * (iz * NAB) + 2], zf);
      if (F32)
        for (int k = 0; k < kZf; k++) sZR[i * kZf + k] = (float)zf[k];
    }
    for (int i = tid; i < ne * NAB; i += C::NTH) {
      const int e = i / NAB, iab = i - e * NAB;
      double ed[kEdgeRec];
      edge_record<FEM_PRISM6>(GC + e * C::NGC, ed);
      double *xf = sXF + i * kXf;
      prism_xf(ed, a.qp[4 * iab], a.qp[4 * iab + 1], xf);
      if (F32)
        for (int k = 0; k < kXf; k++) sXR[i * kXf + k] = (float)xf[k];
    }
    for (int i = tid; i < ne * NS; i += C::NTH) {
      const int e = i / NS, r = i - e * NS, iz = r / NT, t = r - iz * NT;
      const T *xe = X + e * NS + t;
      T w = 0, wd = 0;
#pragma unroll
      for (int k = 0; k < N; k++) {
        const T xv = xe[k * NT];
        w = fma(sL[iz * N + k], xv, w);
        wd = fma(sD[iz * N + k], xv, wd);
      }
      sW[e * 2 * NS + r] = w;
      sW[e * 2 * NS + NS + r] = wd;
    }
    __syncthreads();

    // B. per column (element, level iz, point ib): the b-direction factors
    // G[i] = sum_j B[t(i,j)][ib] W[t(i,j)], then for each of the column's N
    // points (ia, ib) the a-direction sums and the point stage
    for (int i = tid; i < ne * NAB; i += C::NTH) {
      const int e = i / NAB, r = i - e * NAB, iz = r / N, ib = r - iz * N;
      const T *w = sW + e * 2 * NS + iz * NT, *wd = w + NS;
      T g0[N], gx[N], gy[N], gd[N];
#pragma unroll
      for (int ii = 0; ii < N; ii++) {
        T s0 = 0, sx = 0, sy = 0, sd = 0;
#pragma unroll 2
        for (int j = 0; j < N - ii; j++) {
          const int t = (ii + j) * (ii + j + 1) / 2 + j;  // DOF (ii, j)
          const T wv = w[t], bq = sBq[t * NP + ib];
          s0 = fma(bq, wv, s0);
          sd = fma(bq, wd[t], sd);
          sy = fma(sBy[t * NP + ib], wv, sy);
          if (ii > 0) sx = fma(sBx[t * NP + ib], wv, sx);
        }
        g0[ii] = s0;
        gx[ii] = sx;
        gy[ii] = sy;
        gd[ii] = sd;
      }
      const int e_ = e;
      const double *zf = sZF + (e_ * N + iz) * kZf;
#pragma unroll 1
      for (int ia = 0; ia < N; ia++) {
        T u0 = 0, u1 = 0, u2 = 0, u3 = 0;
#pragma unroll
        for (int ii = 0; ii < N; ii++) {
          const T pa = sPa[ia * N + ii];
          u0 = fma(pa, g0[ii], u0);
          u2 = fma(pa, gy[ii], u2);
          u3 = fma(pa, gd[ii], u3);
          if (ii > 0) {
            u1 = fma(sPx[ia * N + ii], gx[ii], u1);
            u2 = fma(sPe[ia * N + ii], gx[ii], u2);
          }
        }
        const int iab = ia * N + ib, q = iz * NAB + iab;
        const double *xf = sXF + (e_ * NAB + iab) * kXf;
        T *vo = sV + e_ * 4 * NQ + q;
        double det;
        if constexpr (F32) {
          float v[4];
          det = xf[0] * zf[6] + xf[1] * zf[7] + xf[2] * zf[8];
          apply_point_f32(sZR + (e_ * N + iz) * kZf, sXR + (e_ * NAB + iab) * kXf, (float)det, sWf[q],
                          sCF + e_ * 10, u0, u1, u2, u3, v);
          vo[0] = v[0];
          vo[NQ] = v[1];
          vo[2 * NQ] = v[2];
          vo[3 * NQ] = v[3];
        } else {
          double adj[3][3];
          det = jac_adj_tp(zf, xf, adj);
          double v[4];
          apply_point(adj, det, sWq[q], GC + e_ * C::NGC + 18, u0, u1, u2, u3, v);
          vo[0] = v[0];
          vo[NQ] = v[1];
          vo[2 * NQ] = v[2];
          vo[3 * NQ] = v[3];
        }
        if (!(det > 0.0)) atomicOr(&sSt[e_], FEM_ST_DET);
      }
    }
    __syncthreads();

    // C1. per column (element, level, ib): the transposed a-direction sums
    // H[i] over the column's points, written over the column's v values
    for (int i = tid; i < ne * NAB; i += C::NTH) {
      const int e = i / NAB, r = i - e * NAB, iz = r / N, ib = r - iz * N;
      T *col = sV + e * 4 * NQ + iz * NAB + ib;  // [c][ia] at col[c NQ + ia N]
      T h0[N], hx[N], hy[N], hd[N];
#pragma unroll
      for (int c = 0; c < N; c++) h0[c] = hx[c] = hy[c] = hd[c] = 0;
#pragma unroll 1
      for (int ia = 0; ia < N; ia++) {
        const T v0 = col[ia * N], v1 = col[NQ + ia * N], v2 = col[2 * NQ + ia * N], v3 = col[3 * NQ + ia * N];
#pragma unroll
        for (int ii = 0; ii < N; ii++) {
          const T pa = sPa[ia * N + ii];
          h0[ii] = fma(pa, v0, h0[ii]);
          hy[ii] = fma(pa, v2, hy[ii]);
          hd[ii] = fma(pa, v3, hd[ii]);
          if (ii > 0) hx[ii] = fma(sPx[ia * N + ii], v1, fma(sPe[ia * N + ii], v2, hx[ii]));
        }
      }
#pragma unroll
      for (int ii = 0; ii < N; ii++) {
        col[ii * N] = h0[ii];
        col[NQ + ii * N] = hx[ii];
        col[2 * NQ + ii * N] = hy[ii];
        col[3 * NQ + ii * N] = hd[ii];
      }
    }
    __syncthreads();

    // C2. transposed b-direction sums -> R, Rd (in place of W, Wd)
    for (int i = tid; i < ne * NS; i += C::NTH) {
      const int e = i / NS, r = i - e * NS, iz = r / NT, t = r - iz * NT;
      const T *h = sV + e * 4 * NQ + iz * NAB + sTi[t] * N;  // [c][ib] at h[c NQ + ib]
      const T *bq = sBq + t * NP, *bx = sBx + t * NP, *by = sBy + t * NP;
      T ra = 0, rb = 0, rd = 0;
#pragma unroll
      for (int ib = 0; ib < N; ib++) {
        ra = fma(bq[ib], h[ib], ra);
        rb = fma(bx[ib], h[NQ + ib], rb);
        ra = fma(by[ib], h[2 * NQ + ib], ra);
        rd = fma(bq[ib], h[3 * NQ + ib], rd);
      }
      sW[e * 2 * NS + r] = ra + rb;
      sW[e * 2 * NS + NS + r] = rd;
    }
    __syncthreads();

    // D. transposed zeta contraction -> y
    T *yg = static_cast<T *>(a.y) + e0 * NS;
    for (int i = tid; i < ne * NS; i += C::NTH) {
      const int e = i / NS, r = i - e * NS, k = r / NT, t = r - k * NT;
      const T *R = sW + e * 2 * NS + t, *Rd = R + NS;
      T y = 0;
#pragma unroll
      for (int iz = 0; iz < N; iz++) {
        y = fma(sL[iz * N + k], R[iz * NT], y);
        y = fma(sD[iz * N + k], Rd[iz * NT], y);
      }
      yg[i] = y;
    }
    if (a.status != nullptr)
      for (int e = tid; e < ne; e += C::NTH) a.status[e0 + e] = sSt[e];
    // the next iteration's barrier (after its wait) orders these reads of
    // sW and sSt before that iteration's phase A overwrites them
  }
}

// P1 tetrahedra: one thread per element, J constant over the element.
template <class T>
__global__ void __launch_bounds__(256) apply_tet_kernel(const ApplyArgs a) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= a.n) return;
  double X[12], cf[10];
  int st = 0;
#pragma unroll
  for (int k = 0; k < 12; k++) {
    X[k] = a.coords[e * 12 + k];
    if (!isfinite(X[k])) st = FEM_ST_NONFINITE;
  }
#pragma unroll
  for (int k = 0; k < 11; k++) {
    const double c = a.coeffs[k * a.cstride + e];
    if (k < 10) cf[k] = c;
    if (!isfinite(c)) st = FEM_ST_NONFINITE;
  }
  const T *xe = static_cast<const T *>(a.x) + e * 4;
  const double x0 = (double)xe[0], x1 = (double)xe[1], x2 = (double)xe[2], x3 = (double)xe[3];
  double adj[3][3];
  const double det = jac_adj<FEM_TET4>(X, a.qp, adj);
  if (!(det > 0.0)) st |= FEM_ST_DET;
  const T *phi = static_cast<const T *>(a.tab);  // [4 NQ][4], row 4 q + d
  double y[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int q = 0; q < 4; q++) {
    double u[4];
#pragma unroll
    for (int d = 0; d < 4; d++) {
      const T *r = phi + (4 * q + d) * 4;
      u[d] = (double)r[0] * x0 + (double)r[1] * x1 + (double)r[2] * x2 + (double)r[3] * x3;
    }
    double v[4];
    apply_point(adj, det, a.qp[4 * q + 3], cf, u[0], u[1], u[2], u[3], v);
#pragma unroll
    for (int d = 0; d < 4; d++) {
      const T *r = phi + (4 * q + d) * 4;
#pragma unroll
      for (int i = 0; i < 4; i++) y[i] += (double)r[i] * v[d];
    }
  }
  T *ye = static_cast<T *>(a.y) + e * 4;
#pragma unroll
  for (int i = 0; i < 4; i++) ye[i] = (T)y[i];
  if (a.status != nullptr) a.status[e] = st;
}

template <int P, class T>
int launch_prism(const ApplyArgs &a, void *stream) {
  using C = ApCfg<P, T>;
  cudaError_t err =
      cudaFuncSetAttribute(apply_prism_kernel<P, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (err != cudaSuccess) {
    set_error(std::string("cudaFuncSetAttribute(apply_prism_kernel): ") + cudaGetErrorString(err));
    return FEM_ECUDA;
  }
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, apply_prism_kernel<P, T>, C::NTH, C::SMEM);
  if (per_sm < 1) per_sm = 1;
  const int64_t groups = (a.n + C::EB - 1) / C::EB;
  const int64_t grid = groups < (int64_t)nsm * per_sm ? groups : (int64_t)nsm * per_sm;
  apply_prism_kernel<P, T><<<(unsigned)grid, C::NTH, C::SMEM, (cudaStream_t)stream>>>(a);
  err = cudaGetLastError();
  if (err != cudaSuccess) {
    set_error(std::string("apply_prism_kernel launch: ") + cudaGetErrorString(err));
    return FEM_ECUDA;
  }
  return FEM_OK;
}

template <class T>
int launch_typed(int elem, int p, const ApplyArgs &a, void *stream) {
  if (elem == FEM_TET4) {
    const int64_t grid = (a.n + 255) / 256;
    if (grid > 0x7fffffffLL) {
      set_error("fem_apply: too many elements for one launch");
      return FEM_EINVAL;
    }
    apply_tet_kernel<T><<<(unsigned)grid, 256, 0, (cudaStream_t)stream>>>(a);
    const cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) {
      set_error(std::string("apply_tet_kernel launch: ") + cudaGetErrorString(err));
      return FEM_ECUDA;
    }
    return FEM_OK;
  }
  switch (p) {
    case 1: return launch_prism<1, T>(a, stream);
    case 2: return launch_prism<2, T>(a, stream);
    case 3: return launch_prism<3, T>(a, stream);
    case 4: return launch_prism<4, T>(a, stream);
    case 5: return launch_prism<5, T>(a, stream);
    case 6: return launch_prism<6, T>(a, stream);
    case 7: return launch_prism<7, T>(a, stream);
  }
  set_error("fem_apply: degree out of range");
  return FEM_EINVAL;
}

}  // namespace

int launch_apply(int elem, int p, bool f32, const ApplyArgs &a, void *stream) {
  if (a.n == 0) return FEM_OK;
  return f32 ? launch_typed<float>(elem, p, a, stream) : launch_typed<double>(elem, p, a, stream);
}

}  // namespace fem
