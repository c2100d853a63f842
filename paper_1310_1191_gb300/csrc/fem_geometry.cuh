// Geometry stage (always FP64): Jacobian of the reference->real map at one
// quadrature point, its determinant and adjugate, folded with the element's
// coefficients into the 4x4 point matrix G_Q of the weak form.
//
// Section 2 / eq. sum_int: physical derivatives are psi = J^{-T} grad_ref phi,
// so with c[iD][jD] as in fem.h the contribution of one point is
//     sum_{d,d'} phi[d][i] G[d][d'] phi[d'][j]   (d = 0 value, 1..3 ref. derivs)
// with
//     G[1+k][1+l] = w det  (J^{-1} D J^{-T})[k][l] = (w / det) (adj D adj^T)[k][l]
//     G[0][1+l]   = w det  (J^{-1} b)[l]           = w (adj b)[l]
//     G[0][0]     = w det c,      G[1+k][0] = 0,
// and the load vector weight S = w det f.  Using the adjugate leaves a single
// division per point.
#pragma once

#include "fem_internal.h"

namespace fem {

// Slots of the packed point record (11 used, padded to 12).
enum GSlot { G00 = 0, G01, G02, G03, G11, G12, G13, G22, G23, G33, GS, GPAD };
constexpr int kGStride = 12;

// J (reference -> real map), adj J and det J at one point, FP64.
// X: vertex coordinates [nv][3]; q4: xi, eta, zeta, w.
template <int ELEM>
__device__ __forceinline__ double jac_adj(const double *X, const double *q4, double (&adj)[3][3]) {
  double J[3][3];
  if (ELEM == FEM_PRISM6) {
    // x(xi,eta,zeta) = sum_a lam_a(xi,eta) [ (1-zeta)/2 x_a + (1+zeta)/2 x_{a+3} ]
    const double xi = q4[0], eta = q4[1], ze = q4[2];
    const double lo = 0.5 * (1.0 - ze), hi = 0.5 * (1.0 + ze), l0 = 1.0 - xi - eta;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const double b0 = X[0 + i], b1 = X[3 + i], b2 = X[6 + i];
      const double t0 = X[9 + i], t1 = X[12 + i], t2 = X[15 + i];
      J[i][0] = lo * (b1 - b0) + hi * (t1 - t0);
      J[i][1] = lo * (b2 - b0) + hi * (t2 - t0);
      J[i][2] = 0.5 * (l0 * (t0 - b0) + xi * (t1 - b1) + eta * (t2 - b2));
    }
  } else {
#pragma unroll
    for (int i = 0; i < 3; i++) {
      J[i][0] = X[3 + i] - X[i];
      J[i][1] = X[6 + i] - X[i];
      J[i][2] = X[9 + i] - X[i];
    }
  }
  adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
}

// Element edge record (FP64, computed once per element): for a prism the
// vectors x1-x0, x4-x3, x2-x0, x5-x3, x3-x0, x4-x1, x5-x2 (21 values), for a
// tetrahedron x1-x0, x2-x0, x3-x0 (9 values).  J at a point is then
//   prism: J[:,0] = lo (x1-x0) + hi (x4-x3),  J[:,1] = lo (x2-x0) + hi (x5-x3),
//          J[:,2] = ((1-xi-eta) (x3-x0) + xi (x4-x1) + eta (x5-x2)) / 2,
//   lo = (1-zeta)/2, hi = (1+zeta)/2 (the map is bilinear in zeta).
constexpr int kEdgeRec = 21;

template <int ELEM>
__device__ __forceinline__ void edge_record(const double *X, double *ed) {
  if (ELEM == FEM_PRISM6) {
#pragma unroll
    for (int i = 0; i < 3; i++) {
      ed[0 + i] = X[3 + i] - X[0 + i];
      ed[3 + i] = X[12 + i] - X[9 + i];
      ed[6 + i] = X[6 + i] - X[0 + i];
      ed[9 + i] = X[15 + i] - X[9 + i];
      ed[12 + i] = X[9 + i] - X[0 + i];
      ed[15 + i] = X[12 + i] - X[3 + i];
      ed[18 + i] = X[15 + i] - X[6 + i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < 3; i++) {
      ed[0 + i] = X[3 + i] - X[i];
      ed[3 + i] = X[6 + i] - X[i];
      ed[6 + i] = X[9 + i] - X[i];
    }
  }
}

// adj J and det J at a point from the element's edge record (FP64).
template <int ELEM>
__device__ __forceinline__ double jac_adj_edges(const double *ed, const double *q4, double (&adj)[3][3]) {
  double J[3][3];
  if (ELEM == FEM_PRISM6) {
    const double xi = q4[0], eta = q4[1], ze = q4[2];
    const double lo = 0.5 * (1.0 - ze), hi = 0.5 * (1.0 + ze);
    const double h0 = 0.5 * (1.0 - xi - eta), h1 = 0.5 * xi, h2 = 0.5 * eta;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      J[i][0] = fma(lo, ed[0 + i], hi * ed[3 + i]);
      J[i][1] = fma(lo, ed[6 + i], hi * ed[9 + i]);
      J[i][2] = fma(h0, ed[12 + i], fma(h1, ed[15 + i], h2 * ed[18 + i]));
    }
  } else {
#pragma unroll
    for (int i = 0; i < 3; i++) {
      J[i][0] = ed[0 + i];
      J[i][1] = ed[3 + i];
      J[i][2] = ed[6 + i];
    }
  }
  adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
}

// Tensor-product geometry factors of a prism (FP64).  The rule's points are
// q = iz n^2 + iab (iab = ia n + ib), with zeta depending on iz only and
// (xi, eta) on iab only, so
//   J[:,0], J[:,1] and adj row 2 = J[:,0] x J[:,1] depend on iz only  (zf[iz][9]),
//   J[:,2]                                       depends on iab only (xf[iab][3]),
// and per point only adj rows 0, 1 (J[:,1] x J[:,2], J[:,2] x J[:,0]) and
// det = J[:,2] . adj row 2 remain: 15 FP64 operations instead of about 45.
constexpr int kZf = 9, kXf = 3;

__device__ __forceinline__ void prism_zf(const double *ed, double zeta, double *zf) {
  const double lo = 0.5 * (1.0 - zeta), hi = 0.5 * (1.0 + zeta);
  double c0[3], c1[3];
#pragma unroll
  for (int i = 0; i < 3; i++) {
    c0[i] = fma(lo, ed[0 + i], hi * ed[3 + i]);
    c1[i] = fma(lo, ed[6 + i], hi * ed[9 + i]);
  }
  zf[0] = c0[0], zf[1] = c0[1], zf[2] = c0[2];
  zf[3] = c1[0], zf[4] = c1[1], zf[5] = c1[2];
  zf[6] = c0[1] * c1[2] - c0[2] * c1[1];
  zf[7] = c0[2] * c1[0] - c0[0] * c1[2];
  zf[8] = c0[0] * c1[1] - c0[1] * c1[0];
}

// The same two factors from the level's (lo, hi) and the triangle point's
// (h0, h1, h2), computed once per rule.
__device__ __forceinline__ void prism_zf_lh(const double *ed, double lo, double hi, double *zf) {
  double c0[3], c1[3];
#pragma unroll
  for (int i = 0; i < 3; i++) {
    c0[i] = fma(lo, ed[0 + i], hi * ed[3 + i]);
    c1[i] = fma(lo, ed[6 + i], hi * ed[9 + i]);
  }
  zf[0] = c0[0], zf[1] = c0[1], zf[2] = c0[2];
  zf[3] = c1[0], zf[4] = c1[1], zf[5] = c1[2];
  zf[6] = c0[1] * c1[2] - c0[2] * c1[1];
  zf[7] = c0[2] * c1[0] - c0[0] * c1[2];
  zf[8] = c0[0] * c1[1] - c0[1] * c1[0];
}

__device__ __forceinline__ void prism_xf_h(const double *ed, double h0, double h1, double h2, double *xf) {
#pragma unroll
  for (int i = 0; i < 3; i++) xf[i] = fma(h0, ed[12 + i], fma(h1, ed[15 + i], h2 * ed[18 + i]));
}

__device__ __forceinline__ void prism_xf(const double *ed, double xi, double eta, double *xf) {
  const double h0 = 0.5 * (1.0 - xi - eta), h1 = 0.5 * xi, h2 = 0.5 * eta;
#pragma unroll
  for (int i = 0; i < 3; i++) xf[i] = fma(h0, ed[12 + i], fma(h1, ed[15 + i], h2 * ed[18 + i]));
}

// adj J and det J at point (iz, iab) from the element's factors.
__device__ __forceinline__ double jac_adj_tp(const double *zf, const double *xf, double (&adj)[3][3]) {
  const double c0x = zf[0], c0y = zf[1], c0z = zf[2], c1x = zf[3], c1y = zf[4], c1z = zf[5];
  const double c2x = xf[0], c2y = xf[1], c2z = xf[2];
  adj[0][0] = c1y * c2z - c1z * c2y;
  adj[0][1] = c1z * c2x - c1x * c2z;
  adj[0][2] = c1x * c2y - c1y * c2x;
  adj[1][0] = c2y * c0z - c2z * c0y;
  adj[1][1] = c2z * c0x - c2x * c0z;
  adj[1][2] = c2x * c0y - c2y * c0x;
  adj[2][0] = zf[6];
  adj[2][1] = zf[7];
  adj[2][2] = zf[8];
  return c2x * zf[6] + c2y * zf[7] + c2z * zf[8];
}

// adj J and det J at a prism point from the element's tensor-product
// factors: adj rows 0, 1 and det J in FP64 (two cross products and a dot
// product), rounded to FP32 (a); zr: adj row 2 of the point's zeta level
// already in FP32.  Returns det J (FP64).
__device__ __forceinline__ double adj_tp_f32(const double *zf, const float *zr, const double *xf, float (&a)[3][3]) {
  const double c0x = zf[0], c0y = zf[1], c0z = zf[2], c1x = zf[3], c1y = zf[4], c1z = zf[5];
  const double c2x = xf[0], c2y = xf[1], c2z = xf[2];
  a[0][0] = (float)(c1y * c2z - c1z * c2y);
  a[0][1] = (float)(c1z * c2x - c1x * c2z);
  a[0][2] = (float)(c1x * c2y - c1y * c2x);
  a[1][0] = (float)(c2y * c0z - c2z * c0y);
  a[1][1] = (float)(c2z * c0x - c2x * c0z);
  a[1][2] = (float)(c2x * c0y - c2y * c0x);
  a[2][0] = zr[0];
  a[2][1] = zr[1];
  a[2][2] = zr[2];
  return c2x * zf[6] + c2y * zf[7] + c2z * zf[8];
}

// FP32 point record from FP32 adj J, det J (FP32), weight and coefficients
// cf: D00 D11 D22 D01 D02 D12 b0 b1 b2 c f.
__device__ __forceinline__ void record_f32(const float (&a)[3][3], float detf, float w, const float *cf, float *g) {
  const float D[3][3] = {{cf[0], cf[3], cf[4]}, {cf[3], cf[1], cf[5]}, {cf[4], cf[5], cf[2]}};
  float M[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int n = 0; n < 3; n++) M[k][n] = a[k][0] * D[0][n] + a[k][1] * D[1][n] + a[k][2] * D[2][n];
  const float s = w / detf;
  auto Gd = [&](int k, int l) { return s * (M[k][0] * a[l][0] + M[k][1] * a[l][1] + M[k][2] * a[l][2]); };
  g[G11] = Gd(0, 0);
  g[G12] = Gd(0, 1);
  g[G13] = Gd(0, 2);
  g[G22] = Gd(1, 1);
  g[G23] = Gd(1, 2);
  g[G33] = Gd(2, 2);
#pragma unroll
  for (int l = 0; l < 3; l++) g[G01 + l] = w * (a[l][0] * cf[6] + a[l][1] * cf[7] + a[l][2] * cf[8]);
  const float wd = w * detf;
  g[G00] = wd * cf[9];
  g[GS] = wd * cf[10];
}

// Point record of the FP32 prism paths from the element's tensor-product
// factors (adj_tp_f32, then record_f32).  Returns det J (FP64).
__device__ __forceinline__ double point_tc(const double *zf, const float *zr, const double *xf, float w,
                                           const float *cf, float *g) {
  float a[3][3];
  const double det = adj_tp_f32(zf, zr, xf, a);
  record_f32(a, (float)det, w, cf, g);
  return det;
}

// Point record from FP64 adj J and det J with the 3x3 products in FP32 (for
// the FP32 and tensor-core contractions, whose point records are FP32).
__device__ __forceinline__ void point_from_adj_f32(const double (&adj)[3][3], double det, double w,
                                                   const double *cf, float *g) {
  float a[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int m = 0; m < 3; m++) a[k][m] = (float)adj[k][m];
  const float D[3][3] = {{(float)cf[0], (float)cf[3], (float)cf[4]},
                         {(float)cf[3], (float)cf[1], (float)cf[5]},
                         {(float)cf[4], (float)cf[5], (float)cf[2]}};
  float M[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int n = 0; n < 3; n++) M[k][n] = a[k][0] * D[0][n] + a[k][1] * D[1][n] + a[k][2] * D[2][n];
  const float s = (float)w / (float)det;
  auto Gd = [&](int k, int l) { return s * (M[k][0] * a[l][0] + M[k][1] * a[l][1] + M[k][2] * a[l][2]); };
  g[G11] = Gd(0, 0);
  g[G12] = Gd(0, 1);
  g[G13] = Gd(0, 2);
  g[G22] = Gd(1, 1);
  g[G23] = Gd(1, 2);
  g[G33] = Gd(2, 2);
  const float wf = (float)w, b0 = (float)cf[6], b1 = (float)cf[7], b2 = (float)cf[8];
#pragma unroll
  for (int l = 0; l < 3; l++) g[G01 + l] = wf * (a[l][0] * b0 + a[l][1] * b1 + a[l][2] * b2);
  const float wd = (float)(w * det);
  g[G00] = wd * (float)cf[9];
  g[GS] = wd * (float)cf[10];
}

// Point record from adj J, det J and the weight (FP64); cf: 11 coefficients.
__device__ __forceinline__ void point_from_adj(const double (&adj)[3][3], double det, double w,
                                               const double *cf, double *g) {
  const double D[3][3] = {{cf[0], cf[3], cf[4]}, {cf[3], cf[1], cf[5]}, {cf[4], cf[5], cf[2]}};
  double M[3][3];  // adj D
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int n = 0; n < 3; n++) M[k][n] = adj[k][0] * D[0][n] + adj[k][1] * D[1][n] + adj[k][2] * D[2][n];
  const double s = w / det;
  auto Gd = [&](int k, int l) {
    return s * (M[k][0] * adj[l][0] + M[k][1] * adj[l][1] + M[k][2] * adj[l][2]);
  };
  g[G11] = Gd(0, 0);
  g[G12] = Gd(0, 1);
  g[G13] = Gd(0, 2);
  g[G22] = Gd(1, 1);
  g[G23] = Gd(1, 2);
  g[G33] = Gd(2, 2);
#pragma unroll
  for (int l = 0; l < 3; l++) g[G01 + l] = w * (adj[l][0] * cf[6] + adj[l][1] * cf[7] + adj[l][2] * cf[8]);
  const double wd = w * det;
  g[G00] = wd * cf[9];
  g[GS] = wd * cf[10];
}

// X: vertex coordinates [nv][3]; cf: 11 coefficients (COEF order);
// q4: xi, eta, zeta, w.  Writes 11 values to g; returns FEM_ST_DET if det <= 0.
template <int ELEM>
__device__ __forceinline__ int point_matrix(const double *X, const double *cf, const double *q4,
                                            double *g) {
  double adj[3][3];
  const double det = jac_adj<ELEM>(X, q4, adj);
  point_from_adj(adj, det, q4[3], cf, g);
  return det > 0.0 ? 0 : FEM_ST_DET;
}

}  // namespace fem

namespace fem {

// Same point record with J, adj J and det J in FP64 and the 3x3 products that
// form G in FP32 (for the reduced-precision contractions, whose G is rounded
// to FP32 anyway).  Returns FEM_ST_DET if det <= 0.
template <int ELEM>
__device__ __forceinline__ int point_matrix_f32(const double *X, const double *cf, const double *q4,
                                                float *g) {
  double J[3][3];
  if (ELEM == FEM_PRISM6) {
    const double xi = q4[0], eta = q4[1], ze = q4[2];
    const double lo = 0.5 * (1.0 - ze), hi = 0.5 * (1.0 + ze), l0 = 1.0 - xi - eta;
#pragma unroll
    for (int i = 0; i < 3; i++) {
      const double b0 = X[0 + i], b1 = X[3 + i], b2 = X[6 + i];
      const double t0 = X[9 + i], t1 = X[12 + i], t2 = X[15 + i];
      J[i][0] = lo * (b1 - b0) + hi * (t1 - t0);
      J[i][1] = lo * (b2 - b0) + hi * (t2 - t0);
      J[i][2] = 0.5 * (l0 * (t0 - b0) + xi * (t1 - b1) + eta * (t2 - b2));
    }
  } else {
#pragma unroll
    for (int i = 0; i < 3; i++) {
      J[i][0] = X[3 + i] - X[i];
      J[i][1] = X[6 + i] - X[i];
      J[i][2] = X[9 + i] - X[i];
    }
  }
  double adj[3][3];
  adj[0][0] = J[1][1] * J[2][2] - J[1][2] * J[2][1];
  adj[0][1] = J[0][2] * J[2][1] - J[0][1] * J[2][2];
  adj[0][2] = J[0][1] * J[1][2] - J[0][2] * J[1][1];
  adj[1][0] = J[1][2] * J[2][0] - J[1][0] * J[2][2];
  adj[1][1] = J[0][0] * J[2][2] - J[0][2] * J[2][0];
  adj[1][2] = J[0][2] * J[1][0] - J[0][0] * J[1][2];
  adj[2][0] = J[1][0] * J[2][1] - J[1][1] * J[2][0];
  adj[2][1] = J[0][1] * J[2][0] - J[0][0] * J[2][1];
  adj[2][2] = J[0][0] * J[1][1] - J[0][1] * J[1][0];
  const double det = J[0][0] * adj[0][0] + J[0][1] * adj[1][0] + J[0][2] * adj[2][0];
  float a[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int m = 0; m < 3; m++) a[k][m] = (float)adj[k][m];
  const float w = (float)q4[3];
  const float D[3][3] = {{(float)cf[0], (float)cf[3], (float)cf[4]},
                         {(float)cf[3], (float)cf[1], (float)cf[5]},
                         {(float)cf[4], (float)cf[5], (float)cf[2]}};
  float M[3][3];
#pragma unroll
  for (int k = 0; k < 3; k++)
#pragma unroll
    for (int n = 0; n < 3; n++) M[k][n] = a[k][0] * D[0][n] + a[k][1] * D[1][n] + a[k][2] * D[2][n];
  const float s = w / (float)det;
  auto Gd = [&](int k, int l) { return s * (M[k][0] * a[l][0] + M[k][1] * a[l][1] + M[k][2] * a[l][2]); };
  g[G11] = Gd(0, 0);
  g[G12] = Gd(0, 1);
  g[G13] = Gd(0, 2);
  g[G22] = Gd(1, 1);
  g[G23] = Gd(1, 2);
  g[G33] = Gd(2, 2);
  const float b0 = (float)cf[6], b1 = (float)cf[7], b2 = (float)cf[8];
#pragma unroll
  for (int l = 0; l < 3; l++) g[G01 + l] = w * (a[l][0] * b0 + a[l][1] * b1 + a[l][2] * b2);
  const float wd = (float)(q4[3] * det);
  g[G00] = wd * (float)cf[9];
  g[GS] = wd * (float)cf[10];
  return det > 0.0 ? 0 : FEM_ST_DET;
}

}  // namespace fem
