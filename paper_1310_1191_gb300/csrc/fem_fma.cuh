// CUDA-core contraction kernels (FP64 and FP32 FMA) for the element matrices.
//
// Per element the weak form reduces to (Algorithm 2 with the sparse c):
//     A[i][j] = sum_Q sum_{d,d'} phi[Q][d][i] G_Q[d][d'] phi[Q][d'][j]
//             = sum_k Phi[k][i] T[k][j],   k = 4 Q + d,  K = 4 NQ,
// with the weighted tile T[4Q+d][j] = sum_{d'} G_Q[d][d'] phi[Q][d'][j]
// (13 FMAs per (Q, j) thanks to the zero block G[1..3][0] and the symmetric
// diffusion block).  Phi (the reference table, the same for every element) is
// the left operand, so one CTA can share it between several elements.
//
// Work decomposition (the paper's two-level parallelism, Section 4): a CTA
// owns a group of EPB elements and one BM x BM output tile of each (the
// "part" of A^e of Algorithms 3/4 when NS > BM); every thread owns a TM x TN
// register micro-tile of one element ("owner computes").  Per CTA:
//   0. stage coordinates and coefficients of its elements in shared memory;
//   1. geometry of every (element, point) in FP64 -> G records in shared memory;
//   2. per chunk of QC points: stage the Phi rows of the tile and build the
//      weighted T columns of the tile for each element, then accumulate the
//      outer products in registers;
//   3. the column-0 tiles also form the load vector b = sum_Q S_Q phi[Q][0];
//   4. write the unpadded micro-tiles (full or upper-packed rows);
//   5. mirrored pairs (see fma_mirror): the tile or micro-tile below the
//      diagonal from the one above it and the convection part, written
//      transposed.
#pragma once

#include <cuda_runtime.h>

#include "fem_geometry.cuh"
#include "fem_law.cuh"

namespace fem {

// ND_ = rows of K per point: 4 (value + 3 derivatives, scalar form) or 3
// (derivatives only, one 3x3 block of linear elastostatics per virtual element).
// RULE_: the prism rule (FEM_RULE_COLLAPSED or FEM_RULE_TABLE1); both are
// (p+1) zeta levels x NAB triangle points, point q = iz NAB + iab.
// MM_: mirrored micro-tiles (one output tile per element, square micro-tiles):
// a thread per micro-tile on or above the diagonal, see fma_mirror.
template <int ELEM_, int P_, int BM_, int TM_, int TN_, int EPB_, int QC_, int ND_ = 4, int RULE_ = FEM_RULE_COLLAPSED,
          bool MM_ = false>
struct FmaCfg {
  static constexpr int ELEM = ELEM_, P = P_, ND = ND_, RULE = RULE_;
  static constexpr bool MM = MM_;
  static constexpr int NS = ns_of(ELEM_, P_), NQ = nq_of(ELEM_, P_, RULE_), NV = nv_of(ELEM_);
  static constexpr int BM = BM_, BN = BM_, TM = TM_, TN = TN_;
  static constexpr int TY = BM / TM, TX = BN / TN, TPE = MM_ ? TY * (TY + 1) / 2 : TX * TY;
  // the same shape with a thread per micro-tile (paths that do not mirror)
  using Plain = FmaCfg<ELEM_, P_, BM_, TM_, TN_, EPB_, QC_, ND_, RULE_, false>;
  static constexpr int EPB = EPB_, NT = EPB * TPE;
  static constexpr int TILES = (NS + BM - 1) / BM;
  static constexpr int QC = QC_, KC = ND * QC, NCH = (NQ + QC - 1) / QC;
  static constexpr int NREC = NV * 3 + 11;  // coords + coefficients per element
  static constexpr int NEDGE = kEdgeRec;    // FP64 edge record per element
  static constexpr int NZ = ELEM_ == FEM_PRISM6 ? P_ + 1 : 0;                 // zeta levels of the rule
  static constexpr int NAB = ELEM_ == FEM_PRISM6 ? ntri_of(P_, RULE_) : 0;     // (xi, eta) points per level
  static_assert(BM % TM == 0 && BN % TN == 0, "tile must split into micro-tiles");
  static_assert(NT <= 1024, "too many threads");
  static_assert(!MM_ || (TM_ == TN_ && BM_ >= ns_of(ELEM_, P_)), "mirrored micro-tiles: square, one tile");

  template <class T>
  static constexpr size_t smem_bytes() {
    return sizeof(T) * ((size_t)KC * BM + (size_t)EPB * KC * BN + (size_t)EPB * NQ * kGStride) + 16 +
           sizeof(double) * (size_t)EPB * (NREC + NEDGE + NZ * kZf + NAB * kXf) + sizeof(int) * (size_t)(EPB + 1) +
           sizeof(int64_t) * (size_t)EPB + 64 + sizeof(float) * ((size_t)EPB * (12 + 4 * NZ) + NQ) + 16;
  }
};

// One work item: the group of EPB elements at sorted positions k0..k_end-1
// (at most EPB; element id = perm[k] if a.perm, else k) and output tile (ti, tj).  Cooperative loops
// stride over the whole block, so the body also runs inside kernels whose
// block is larger than C::NT (the batched kernel); the register micro-tiles
// belong to the first C::NT threads.
constexpr int cgcd(int a, int b) { return b == 0 ? a : cgcd(b, a % b); }

// N consecutive values (shared or global memory); ALIGN = a number of elements that
// divides the offset of p from a 16-byte aligned base.  Uses 16- or 8-byte
// loads when the alignment allows.
template <class T, int N, int ALIGN>
__device__ __forceinline__ void lds_vec(const T *p, T (&v)[N]) {
  if constexpr (sizeof(T) == 4 && N % 4 == 0 && ALIGN % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N / 4; i++) {
      const float4 x = reinterpret_cast<const float4 *>(p)[i];
      v[4 * i] = x.x;
      v[4 * i + 1] = x.y;
      v[4 * i + 2] = x.z;
      v[4 * i + 3] = x.w;
    }
  } else if constexpr (sizeof(T) == 4 && N % 2 == 0 && ALIGN % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; i++) {
      const float2 x = reinterpret_cast<const float2 *>(p)[i];
      v[2 * i] = x.x;
      v[2 * i + 1] = x.y;
    }
  } else if constexpr (sizeof(T) == 8 && N % 2 == 0 && ALIGN % 2 == 0) {
#pragma unroll
    for (int i = 0; i < N / 2; i++) {
      const double2 x = reinterpret_cast<const double2 *>(p)[i];
      v[2 * i] = x.x;
      v[2 * i + 1] = x.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; i++) v[i] = p[i];
  }
}

// Extra shared memory of the law variants: field coefficients per element
// and, for the network, its parameters.
template <class C>
constexpr size_t law_smem_bytes(int law) {
  return law == 0 ? 0 : (size_t)C::EPB * C::NS * 4 + 16 + (law == 2 ? (size_t)kMlpSmemBytes + 16 : 0);
}

// Mirrored tile pairs.  Diffusion and reaction make a symmetric part S of
// A_e (G[1..3][1..3] is symmetric, G[1..3][0] = 0); only the convection part
// Cv[i][j] = sum_Q phi_0[Q][i] V[Q][j], V[Q][j] = sum_{d=1..3} G[0][d]
// phi_d[Q][j], is not.  So the tile below the diagonal follows from the one
// above it: A[j][i] = A[i][j] + sum_Q (phi_0[Q][j] V[Q][i] - phi_0[Q][i]
// V[Q][j]), a contraction over 2 NQ instead of 4 NQ.  With several output
// tiles per element (TILES >= 2) a CTA takes the tile pair (ti, tj), ti <= tj:
// the upper tile as before, then, for ti < tj, the correction into the same
// registers and the transposed write.  Work per element: TILES (TILES + 1) / 2
// full tiles and TILES (TILES - 1) / 2 half tiles instead of TILES^2 full ones
// (p = 7, three tiles: 0.83; two tiles: 0.875).  With one tile per element
// the same holds for micro-tiles (C::MM): a thread per micro-tile (ty, tx),
// ty <= tx, the diagonal ones last (whole warps of them skip the correction);
// with 21 x 21 micro-tiles (p = 5) 0.76 of the dense work.  Scalar form with
// constant coefficients only.
template <class C, int LAW, bool SPLIT>
constexpr bool fma_mirror() {
  return (C::TILES >= 2 || C::MM) && C::ND == 4 && LAW == 0 && !SPLIT;
}

// tile pair pr (0 .. TILES (TILES + 1) / 2 - 1) -> (ti, tj), ti <= tj, row by row
template <int TILES>
__device__ __forceinline__ void pair_tiles(int pr, int &ti, int &tj) {
  ti = 0;
  while (pr >= TILES - ti) {
    pr -= TILES - ti;
    ti++;
  }
  tj = ti + pr;
}

// SPLIT: the Jacobian terms (det J, J^{-1} per point) are read from a.terms
// instead of computed from a.coords (the paper's NOJAC variants).
// MIRROR (fma_mirror): (ti, tj) is a tile pair, see above.
template <class T, class C, int LAW = 0, bool SPLIT = false, bool MIRROR = false>
__device__ __forceinline__ void fma_body(const FmaArgs &a, const double *qp, const T *phi, int64_t k0,
                                         int64_t k_end, int ti, int tj, unsigned char *smem) {
  T *sPA = reinterpret_cast<T *>(smem);                 // [KC][BM]
  T *sT = sPA + C::KC * C::BM;                          // [EPB][KC][BN]
  T *sG = sT + C::EPB * C::KC * C::BN;                  // [EPB][NQ][kGStride]
  // the FP64 records start on a 16-byte boundary whatever the FP32 arrays' sizes
  double *sX = reinterpret_cast<double *>(
      (reinterpret_cast<uintptr_t>(sG + C::EPB * C::NQ * kGStride) + 15) & ~(uintptr_t)15);  // [EPB][NREC]
  double *sEd = sX + C::EPB * C::NREC;                                     // [EPB][NEDGE]
  double *sZF = sEd + C::EPB * C::NEDGE;                                   // [EPB][NZ][9]  (prisms)
  double *sXF = sZF + C::EPB * C::NZ * kZf;                                // [EPB][NAB][3] (prisms)
  int *sSt = reinterpret_cast<int *>(sXF + C::EPB * C::NAB * kXf);         // [EPB]
  int64_t *sE = reinterpret_cast<int64_t *>(sSt + C::EPB + (C::EPB & 1));   // [EPB] element ids
  // FP32 copies for the FP32 point records of prisms: coefficients, adj row 2
  // per zeta level, quadrature weights
  float *sCF = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(sE + C::EPB) + 15) & ~(uintptr_t)15);      // [EPB][12]
  float *sZR = sCF + C::EPB * 12;                                               // [EPB][NZ][4]
  float *sWq = sZR + C::EPB * C::NZ * 4;                                        // [NQ]
  float *sU = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(sWq + C::NQ) + 15) & ~(uintptr_t)15);      // [EPB][NS] (LAW)
  float *sW = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(sU + C::EPB * C::NS) + 15) & ~(uintptr_t)15);  // network (LAW 2)
  uint32_t *sW2 = reinterpret_cast<uint32_t *>(sW + kMlpSmall);                   // W2, BF16 pairs
  // network inputs of the points (LAW 2), in the contraction's staging area,
  // which is idle during the geometry stage
  float *sNet = reinterpret_cast<float *>(sPA);
  static_assert(LAW != 2 || (size_t)(C::KC * C::BM + C::EPB * C::KC * C::BN) * sizeof(T) >=
                                (size_t)2 * C::EPB * C::NQ * sizeof(float),
                "staging area too small for the network inputs");

  const int tid = threadIdx.x, nthr = blockDim.x;
  constexpr int NSZ = C::NS * C::NS, NPK = C::NS * (C::NS + 1) / 2;
  constexpr bool split = SPLIT;  // Jacobian terms read, not computed
  // FP32 records of prisms from the tensor-product factors with FP32 coefficients
  constexpr bool fp32rec = sizeof(T) == 4 && C::ELEM == FEM_PRISM6 && !SPLIT && C::ND == 4;
  constexpr bool fastf32 = fp32rec && LAW == 0;

  for (int le = tid; le < C::EPB; le += nthr) {
    const int64_t k = k0 + le;
    int64_t v = k < k_end ? (a.perm ? a.perm[k] : k) : -1;
    if (v >= 0 && a.perm && a.nmesh >= 0 && !fem_chk(v < a.nmesh, a.err)) v = -1;  // checked builds
    sE[le] = v;
    sSt[le] = 0;
  }
  __syncthreads();
  // 0. element records (elasticity: the real element e = v / 9 of virtual element v,
  //    coefficients E, nu, fx, fy, fz)
  constexpr bool ELAST = C::ND == 3;
  constexpr int NCF = ELAST ? 5 : 11;
  for (int idx = tid; idx < C::EPB * C::NREC; idx += nthr) {
    const int le = idx / C::NREC, k = idx % C::NREC;
    const int64_t e = ELAST ? (sE[le] >= 0 ? sE[le] / 9 : -1) : sE[le];
    double v = 0.0;
    if (e >= 0 && k < C::NV * 3 + NCF) {
      if (k >= C::NV * 3)
        v = a.coeffs[(k - C::NV * 3) * a.cstride + e];
      else if (!split)
        v = a.coords[e * (C::NV * 3) + k];
    }
    sX[idx] = v;
  }
  if (LAW != 0) {
    for (int idx = tid; idx < C::EPB * C::NS; idx += nthr) {
      const int64_t e = sE[idx / C::NS];
      sU[idx] = e >= 0 ? a.ucoef[e * C::NS + idx % C::NS] : 0.f;
    }
    if (LAW == 2) {
      // FP32 W1, b1, b2, W3, b3 and the BF16 image of W2 (rows padded to kW2Stride)
      constexpr int H = kMlpH;
      for (int idx = tid; idx < kMlpSmall; idx += nthr) {
        float v = 0.f;
        if (idx < 3 * H) v = a.mlpw[idx];                          // W1, b1
        else if (idx < 5 * H + 1) v = a.mlpw[3 * H + H * H + (idx - 3 * H)];  // b2, W3, b3
        sW[idx] = v;
      }
      for (int idx = tid; idx < H * (H / 2); idx += nthr)
        sW2[(idx / (H / 2)) * (kW2Stride / 2) + idx % (H / 2)] = a.mlpw2[idx];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < C::EPB * C::NREC; idx += nthr)
    if (!isfinite(sX[idx])) atomicOr(&sSt[idx / C::NREC], FEM_ST_NONFINITE);
  if (!split)
    for (int le = tid; le < C::EPB; le += nthr) edge_record<C::ELEM>(sX + le * C::NREC, sEd + le * C::NEDGE);
  if constexpr (fp32rec) {
    for (int idx = tid; idx < C::EPB * 11; idx += nthr)
      sCF[(idx / 11) * 12 + idx % 11] = (float)sX[(idx / 11) * C::NREC + C::NV * 3 + idx % 11];
    for (int q = tid; q < C::NQ; q += nthr) sWq[q] = (float)qp[4 * q + 3];
  }
  __syncthreads();
  if constexpr (C::ELEM == FEM_PRISM6) {
    if (!split) {  // tensor-product factors of J (per zeta level and per (xi, eta))
      for (int idx = tid; idx < C::EPB * (C::NZ + C::NAB); idx += nthr) {
        const int le = idx / (C::NZ + C::NAB), r = idx % (C::NZ + C::NAB);
        const double *ed = sEd + le * C::NEDGE;
        if (r < C::NZ) {
          double *zf = sZF + (le * C::NZ + r) * kZf;
          prism_zf(ed, qp[4 * (r * C::NAB) + 2], zf);
          if (fp32rec) {
            float *zr = sZR + (le * C::NZ + r) * 4;
            zr[0] = (float)zf[6];
            zr[1] = (float)zf[7];
            zr[2] = (float)zf[8];
          }
        } else
          prism_xf(ed, qp[4 * (r - C::NZ)], qp[4 * (r - C::NZ) + 1], sXF + (le * C::NAB + r - C::NZ) * kXf);
      }
      __syncthreads();
    }
  }
  // adj J and det J at point q of local element le; split geometry: adj J =
  // det J * J^{-1} from the stored terms (non-finite terms flag the element)
  auto geo = [&](int le, int q, double (&adj)[3][3]) -> double {
    if constexpr (split) {
      const int64_t e = ELAST ? (sE[le] >= 0 ? sE[le] / 9 : -1) : sE[le];
      if (e < 0) {
#pragma unroll
        for (int k = 0; k < 3; k++)
#pragma unroll
          for (int m = 0; m < 3; m++) adj[k][m] = k == m ? 1.0 : 0.0;
        return 1.0;
      }
      const double *tr = a.terms + ((size_t)e * C::NQ + q) * 10;
      const double det = tr[0];
      bool fin = isfinite(det);
#pragma unroll
      for (int k = 0; k < 3; k++)
#pragma unroll
        for (int m = 0; m < 3; m++) {
          const double v = tr[1 + 3 * k + m];
          fin = fin && isfinite(v);
          adj[k][m] = det * v;
        }
      if (!fin) atomicOr(&sSt[le], FEM_ST_NONFINITE);
      return det;
    }
    if constexpr (C::ELEM == FEM_PRISM6) {
      const int iz = q / C::NAB, iab = q % C::NAB;
      return jac_adj_tp(sZF + (le * C::NZ + iz) * kZf, sXF + (le * C::NAB + iab) * kXf, adj);
    } else {
      return jac_adj_edges<C::ELEM>(sEd + le * C::NEDGE, qp + 4 * q, adj);
    }
  };
  if (!ELAST && a.layout == FEM_OUT_SYMPACKED) {
    for (int le = tid; le < C::EPB; le += nthr) {
      const double *cf = sX + le * C::NREC + C::NV * 3;
      if (cf[6] != 0.0 || cf[7] != 0.0 || cf[8] != 0.0) atomicOr(&sSt[le], FEM_ST_NONSYM);
    }
  }

  // 1. geometry (FP64) -> point records
  for (int idx = tid; idx < C::EPB * C::NQ; idx += nthr) {
    const int le = idx / C::NQ, q = idx % C::NQ;
    double g[11];
    bool pend = false;  // LAW 2: k from the network, applied after this loop
    const double *rec = sX + le * C::NREC;
    int st;
    if (ELAST) {
      // block (i, k) of isotropic elasticity: G[a][b] = (w / det) (lam adj_ai adj_bk
      //   + mu d_ik (adj adj^T)_ab + mu adj_ak adj_bi),  G[3][3] slot 9 = w det f_i (k = 0)
      double adj[3][3];
      const double det = geo(le, q, adj);
      st = det > 0.0 ? 0 : FEM_ST_DET;
      const double *cf = rec + C::NV * 3;
      const double Ey = cf[0], nu = cf[1];
      const double lam = Ey * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)), mu = Ey / (2.0 * (1.0 + nu));
      const int blk = sE[le] >= 0 ? (int)(sE[le] % 9) : 0, bi = blk / 3, bk = blk % 3;
      const double w = qp[4 * q + 3], sw = w / det;
      double ci[3], ck[3];  // columns bi and bk of adj J (selected without dynamic indexing)
#pragma unroll
      for (int m = 0; m < 3; m++) {
        ci[m] = bi == 0 ? adj[m][0] : (bi == 1 ? adj[m][1] : adj[m][2]);
        ck[m] = bk == 0 ? adj[m][0] : (bk == 1 ? adj[m][1] : adj[m][2]);
      }
      const double dik = bi == bk ? mu : 0.0;
#pragma unroll
      for (int aa = 0; aa < 3; aa++)
#pragma unroll
        for (int bb = 0; bb < 3; bb++) {
          const double v = lam * ci[aa] * ck[bb] + mu * ck[aa] * ci[bb] +
                           dik * (adj[aa][0] * adj[bb][0] + adj[aa][1] * adj[bb][1] + adj[aa][2] * adj[bb][2]);
          g[3 * aa + bb] = sw * v;
        }
      const double fi = bi == 0 ? cf[2] : (bi == 1 ? cf[3] : cf[4]);
      g[9] = bk == 0 ? w * det * fi : 0.0;
      g[10] = 0.0;
    } else if constexpr (fastf32) {
      // FP64 adj rows 0, 1 and det J, the rest in FP32 (7 FP64 -> FP32 conversions per point)
      float gf[11];
      const int iz = q / C::NAB, iab = q % C::NAB;
      const double det = point_tc(sZF + (le * C::NZ + iz) * kZf, sZR + (le * C::NZ + iz) * 4,
                                  sXF + (le * C::NAB + iab) * kXf, sWq[q], sCF + le * 12, gf);
      st = det > 0.0 ? 0 : FEM_ST_DET;
#pragma unroll
      for (int k = 0; k < 11; k++) g[k] = gf[k];
    } else if (LAW == 0) {
      double adj[3][3];
      const double det = geo(le, q, adj);
      st = det > 0.0 ? 0 : FEM_ST_DET;
      if (sizeof(T) == 4) {  // FP32 contraction: G products in FP32
        float gf[11];
        point_from_adj_f32(adj, det, qp[4 * q + 3], rec + C::NV * 3, gf);
#pragma unroll
        for (int k = 0; k < 11; k++) g[k] = gf[k];
      } else {
        point_from_adj(adj, det, qp[4 * q + 3], rec + C::NV * 3, g);
      }
    } else if constexpr (fp32rec) {
      // coefficient stage (Algorithm 1, coefficients at the point), FP32 kernel:
      // adj J and det J from FP64 factors, u, grad u, k and the record in FP32
      float a32[3][3];
      const int iz = q / C::NAB, iab = q % C::NAB;
      const double det = adj_tp_f32(sZF + (le * C::NZ + iz) * kZf, sZR + (le * C::NZ + iz) * 4,
                                    sXF + (le * C::NAB + iab) * kXf, a32);
      st = det > 0.0 ? 0 : FEM_ST_DET;
      const float *ph = static_cast<const float *>(a.phiT) + (size_t)q * 4;
      const float *U = sU + le * C::NS;
      float u = 0.f, r0 = 0.f, r1 = 0.f, r2 = 0.f;
      for (int k = 0; k < C::NS; k++) {
        const float uk = U[k];
        float f[4];
        lds_vec<float, 4, 4>(ph + (size_t)k * C::NQ * 4, f);
        u = fmaf(uk, f[0], u);
        r0 = fmaf(uk, f[1], r0);
        r1 = fmaf(uk, f[2], r1);
        r2 = fmaf(uk, f[3], r2);
      }
      const float detf = (float)det, idet = 1.f / detf;
      const float gx = (a32[0][0] * r0 + a32[1][0] * r1 + a32[2][0] * r2) * idet;
      const float gy = (a32[0][1] * r0 + a32[1][1] * r1 + a32[2][1] * r2) * idet;
      const float gz = (a32[0][2] * r0 + a32[1][2] * r1 + a32[2][2] * r2) * idet;
      const float gg = gx * gx + gy * gy + gz * gz;
      float kq = 1.f;
      if (LAW == 1) {
        kq = law_exact<float>(u, gg, a.law_iters);
      } else {
        const float sf = sqrtf(gg);
        if (u >= a.box[0] && u <= a.box[1] && sf >= a.box[2] && sf <= a.box[3]) {
          pend = true;
          sNet[2 * idx] = fmaf(u, a.nrm[0], a.nrm[1]);
          sNet[2 * idx + 1] = fmaf(logf(sf), a.nrm[2], a.nrm[3]);
        } else {
          kq = law_exact<float>(u, gg, a.law_iters);
          st |= FEM_ST_FALLBACK;
        }
      }
      const float *cf = sCF + le * 12;
      const float cfl[11] = {kq, kq, kq, 0.f, 0.f, 0.f, cf[6], cf[7], cf[8], cf[9], cf[10]};
      float gf[11];
      record_f32(a32, detf, sWq[q], cfl, gf);
#pragma unroll
      for (int k = 0; k < 11; k++) g[k] = gf[k];
    } else {
      // coefficient stage (Algorithm 1, coefficients at the point): u and grad u from
      // the element's old degrees of freedom, then k(u, |grad u|), D = k I
      double adj[3][3];
      const double det = geo(le, q, adj);
      st = det > 0.0 ? 0 : FEM_ST_DET;
      // point-major table: the 4 values of shape function k at point q are
      // contiguous, so the threads of a warp (consecutive q) read one
      // contiguous run per k
      const T *ph = static_cast<const T *>(a.phiT) + (size_t)q * 4;
      const float *U = sU + le * C::NS;
      T u = 0, r0 = 0, r1 = 0, r2 = 0;
      for (int k = 0; k < C::NS; k++) {
        const T uk = (T)U[k];
        T f[4];
        lds_vec<T, 4, 4>(ph + (size_t)k * C::NQ * 4, f);
        u = fma(uk, f[0], u);
        r0 = fma(uk, f[1], r0);
        r1 = fma(uk, f[2], r1);
        r2 = fma(uk, f[3], r2);
      }
      const double gx = (adj[0][0] * r0 + adj[1][0] * r1 + adj[2][0] * r2) / det;
      const double gy = (adj[0][1] * r0 + adj[1][1] * r1 + adj[2][1] * r2) / det;
      const double gz = (adj[0][2] * r0 + adj[1][2] * r1 + adj[2][2] * r2) / det;
      const T gg = (T)(gx * gx + gy * gy + gz * gz);
      T kq = (T)1;
      if (LAW == 1) {
        kq = law_exact<T>(u, gg, a.law_iters);
      } else {
        // inside the box the network gives k after this stage (the record is
        // built with k = 1 and its diffusion block scaled then); outside, the
        // exact law
        const float uf = (float)u, sf = sqrtf((float)gg);
        if (uf >= a.box[0] && uf <= a.box[1] && sf >= a.box[2] && sf <= a.box[3]) {
          pend = true;
          sNet[2 * idx] = fmaf(uf, a.nrm[0], a.nrm[1]);
          sNet[2 * idx + 1] = fmaf(logf(sf), a.nrm[2], a.nrm[3]);
        } else {
          kq = law_exact<T>(u, gg, a.law_iters);
          st |= FEM_ST_FALLBACK;
        }
      }
      const double *cf = rec + C::NV * 3;
      const double cfl[11] = {(double)kq, (double)kq, (double)kq, 0.0, 0.0, 0.0, cf[6], cf[7], cf[8], cf[9], cf[10]};
      point_from_adj(adj, det, qp[4 * q + 3], cfl, g);
    }
    T *dst = sG + (size_t)idx * kGStride;
    if (sE[le] >= 0) {
#pragma unroll
      for (int k = 0; k < 11; k++) dst[k] = (T)g[k];
      if (st) atomicOr(&sSt[le], st);
    } else {
#pragma unroll
      for (int k = 0; k < 11; k++) dst[k] = (T)0;
      pend = false;
    }
    if (LAW == 2) dst[GPAD] = pend ? (T)1 : (T)0;  // the network still owes this point its k
  }
  __syncthreads();
  if constexpr (LAW == 2) {
    // network coefficient of the pending points (tensor cores), then D = k I:
    // the diffusion block G11..G33 of the record is linear in k
    mlp_points_mma(
        sW, sW2, sNet, C::EPB * C::NQ, [&](int pt) { return sG[(size_t)pt * kGStride + GPAD] != (T)0; },
        [&](int pt, float k) {
          T *r = sG + (size_t)pt * kGStride;
#pragma unroll
          for (int m = G11; m <= G33; m++) r[m] *= (T)k;
        },
        -1, 0, a.hw_tanh != 0);
    __syncthreads();
  }

  // 2. contraction over chunks of points
  const bool owner = tid < C::NT;
  const int le = owner ? tid / C::TPE : 0, r = tid % C::TPE;
  int tx = r % C::TX, ty = r / C::TX;
  if constexpr (C::MM) {
    // micro-tile pairs: first the TY (TY - 1) / 2 above the diagonal, row by
    // row, then the TY diagonal ones
    constexpr int NOFF = C::TY * (C::TY - 1) / 2;
    if (r >= NOFF) {
      ty = tx = r - NOFF;
    } else {
      int rr = r;
      ty = 0;
      while (rr >= C::TY - 1 - ty) {
        rr -= C::TY - 1 - ty;
        ty++;
      }
      tx = ty + 1 + rr;
    }
  }
  T acc[C::TM][C::TN];
#pragma unroll
  for (int i = 0; i < C::TM; i++)
#pragma unroll
    for (int j = 0; j < C::TN; j++) acc[i][j] = (T)0;

  for (int ch = 0; ch < C::NCH; ch++) {
    const int q0 = ch * C::QC;
    for (int idx = tid; idx < C::KC * C::BM; idx += nthr) {
      const int k = idx / C::BM, i = idx % C::BM;
      const int row = ti * C::BM + i;
      const int qk = q0 + k / C::ND;
      const int kg = ELAST ? 4 * qk + 1 + k % 3 : 4 * q0 + k;  // elasticity: derivative rows only
      sPA[idx] = (row < C::NS && qk < C::NQ) ? phi[(size_t)kg * C::NS + row] : (T)0;
    }
    for (int idx = tid; idx < C::EPB * C::QC * C::BN; idx += nthr) {
      const int l2 = idx / (C::QC * C::BN), rem = idx % (C::QC * C::BN);
      const int qq = rem / C::BN, j = rem % C::BN;
      const int q = q0 + qq, col = tj * C::BN + j;
      T t0 = 0, t1 = 0, t2 = 0, t3 = 0;
      if (q < C::NQ && col < C::NS) {
        const T *ph = phi + (size_t)(4 * q) * C::NS + col;
        const T f0 = ph[0], f1 = ph[C::NS], f2 = ph[2 * C::NS], f3 = ph[3 * C::NS];
        const T *g = sG + ((size_t)l2 * C::NQ + q) * kGStride;
        if (ELAST) {  // general 3x3 block on the derivative rows
          t0 = g[0] * f1 + g[1] * f2 + g[2] * f3;
          t1 = g[3] * f1 + g[4] * f2 + g[5] * f3;
          t2 = g[6] * f1 + g[7] * f2 + g[8] * f3;
        } else {
          t0 = g[G00] * f0 + g[G01] * f1 + g[G02] * f2 + g[G03] * f3;
          t1 = g[G11] * f1 + g[G12] * f2 + g[G13] * f3;
          t2 = g[G12] * f1 + g[G22] * f2 + g[G23] * f3;
          t3 = g[G13] * f1 + g[G23] * f2 + g[G33] * f3;
        }
      }
      T *tt = sT + ((size_t)l2 * C::KC + C::ND * qq) * C::BN + j;
      tt[0] = t0;
      tt[C::BN] = t1;
      tt[2 * C::BN] = t2;
      if (!ELAST) tt[3 * C::BN] = t3;
    }
    __syncthreads();
    if (owner) {
      const T *pa = sPA + ty * C::TM;
      const T *pb = sT + (size_t)le * C::KC * C::BN + tx * C::TN;
      // element offsets of the operands from the 16-byte aligned shared base
      constexpr int ALA = cgcd(C::BM, C::TM);
      constexpr int ALB = cgcd(cgcd(C::KC * C::BM, C::KC * C::BN), cgcd(C::BN, C::TN));
#pragma unroll 4
      for (int k = 0; k < C::KC; k++) {
        T av[C::TM], bv[C::TN];
        lds_vec<T, C::TM, ALA>(pa + k * C::BM, av);
        lds_vec<T, C::TN, ALB>(pb + k * C::BN, bv);
        if constexpr (sizeof(T) == 4 && C::NT <= 512) {
          // FP32: two multiply-adds per instruction (fma.rn.f32x2; the same
          // round-to-nearest fused multiply-add on each lane as fmaf, so the
          // results are unchanged).  The kernel is issue-bound, and this
          // halves the issue slots of the multiply-adds.  Not in the one-tile
          // p = 6 shapes (625 threads, 96 registers): there the register
          // pairs spill (elasticity p = 6 measured 12 % slower).
#pragma unroll
          for (int i = 0; i < C::TM; i++) {
            const float2 a2 = make_float2(av[i], av[i]);
#pragma unroll
            for (int j = 0; j + 1 < C::TN; j += 2) {
              const float2 c = __ffma2_rn(a2, make_float2(bv[j], bv[j + 1]), make_float2(acc[i][j], acc[i][j + 1]));
              acc[i][j] = c.x;
              acc[i][j + 1] = c.y;
            }
            if (C::TN & 1) acc[i][C::TN - 1] = fma(av[i], bv[C::TN - 1], acc[i][C::TN - 1]);
          }
        } else {
#pragma unroll
          for (int i = 0; i < C::TM; i++)
#pragma unroll
            for (int j = 0; j < C::TN; j++) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
      }
    }
    __syncthreads();
  }

  // 3. load vector rows of this tile (mirrored pairs: by the diagonal tile)
  if ((MIRROR ? ti == tj : tj == 0) && a.b != nullptr) {
    T *bo = static_cast<T *>(a.b);
    constexpr int SLOT = ELAST ? 9 : GS;
    for (int idx = tid; idx < C::EPB * C::BM; idx += nthr) {
      const int l2 = idx / C::BM, i = idx % C::BM, row = ti * C::BM + i;
      const int64_t e = sE[l2];
      // elasticity: the (i, 0) block of element e writes component i of b_e
      if (row < C::NS && e >= 0 && (!ELAST || e % 3 == 0)) {
        T s = 0;
        const T *g = sG + (size_t)l2 * C::NQ * kGStride + SLOT;
        for (int q = 0; q < C::NQ; q++) s = fma(g[q * kGStride], phi[(size_t)(4 * q) * C::NS + row], s);
        const int64_t boff = ELAST ? (e / 3) * (int64_t)C::NS : (a.offb ? a.offb[e] : e * (int64_t)C::NS);
        if (fem_chk(a.limb < 0 || (boff >= 0 && boff + C::NS <= a.limb), a.err)) bo[boff + row] = s;
      }
    }
  }

  // 4. write the micro-tile
  const int64_t e = owner ? sE[le] : -1;
  if (e >= 0) {
    T *Ao = static_cast<T *>(a.A);
    const int64_t oA = a.offA ? a.offA[e] : e * (int64_t)(a.layout == FEM_OUT_FULL ? NSZ : NPK);
    const bool okA = fem_chk(a.limA < 0 || (oA >= 0 && oA + (a.layout == FEM_OUT_FULL ? NSZ : NPK) <= a.limA), a.err);
    if (okA && a.layout == FEM_OUT_FULL) {
      T *Ae = Ao + oA;
#pragma unroll
      for (int i = 0; i < C::TM; i++) {
        const int row = ti * C::BM + ty * C::TM + i;
        if (row >= C::NS) continue;
#pragma unroll
        for (int j = 0; j < C::TN; j++) {
          const int col = tj * C::BN + tx * C::TN + j;
          if (col < C::NS) Ae[row * C::NS + col] = acc[i][j];
        }
      }
    } else if (okA) {
      T *Ae = Ao + oA;
#pragma unroll
      for (int i = 0; i < C::TM; i++) {
        const int row = ti * C::BM + ty * C::TM + i;
        if (row >= C::NS) continue;
        const int base = row * C::NS - row * (row - 1) / 2 - row;
#pragma unroll
        for (int j = 0; j < C::TN; j++) {
          const int col = tj * C::BN + tx * C::TN + j;
          if (col < C::NS && col >= row) Ae[base + col] = acc[i][j];
        }
      }
    }
  }
  // 5. mirrored pair: the tile (tj, ti) below the diagonal from the upper one
  //    (full layout; the upper-packed layout keeps only the upper tiles)
  if constexpr (MIRROR) {
    // pairs of tiles (ti < tj), or, with one tile, of micro-tiles (ty < tx)
    const bool mine = !C::MM || ty < tx;
    if ((C::MM || ti < tj) && a.layout == FEM_OUT_FULL) {
      static_assert(2 * C::QC * C::BM <= C::KC * C::BM && 2 * C::QC * C::BN <= C::KC * C::BN, "staging");
      T *sP0i = sPA, *sP0j = sPA + C::QC * C::BM;            // phi_0 rows of tiles ti, tj: [QC][BM]
      T *sVi = sT, *sVj = sT + C::EPB * C::QC * C::BM;       // V of tiles ti, tj: [EPB][QC][BM]
      for (int ch = 0; ch < C::NCH; ch++) {
        const int q0 = ch * C::QC;
        for (int idx = tid; idx < 2 * C::QC * C::BM; idx += nthr) {
          const int h = idx / (C::QC * C::BM), r2 = idx % (C::QC * C::BM);
          const int qq = r2 / C::BM, i = r2 % C::BM, q = q0 + qq;
          const int row = (h ? tj : ti) * C::BM + i;
          sPA[idx] = (row < C::NS && q < C::NQ) ? phi[(size_t)(4 * q) * C::NS + row] : (T)0;
        }
        for (int idx = tid; idx < 2 * C::EPB * C::QC * C::BM; idx += nthr) {
          const int h = idx / (C::EPB * C::QC * C::BM), r2 = idx % (C::EPB * C::QC * C::BM);
          const int l2 = r2 / (C::QC * C::BM), r3 = r2 % (C::QC * C::BM);
          const int qq = r3 / C::BM, i = r3 % C::BM, q = q0 + qq;
          const int col = (h ? tj : ti) * C::BM + i;
          T v = 0;
          if (q < C::NQ && col < C::NS) {
            const T *ph = phi + (size_t)(4 * q) * C::NS + col;
            const T *g = sG + ((size_t)l2 * C::NQ + q) * kGStride;
            v = g[G01] * ph[C::NS] + g[G02] * ph[2 * C::NS] + g[G03] * ph[3 * C::NS];
          }
          sT[idx] = v;
        }
        __syncthreads();
        if (owner && mine) {
          const T *pi = sP0i + ty * C::TM, *pj = sP0j + tx * C::TN;
          const T *vi = sVi + (size_t)le * C::QC * C::BM + ty * C::TM;
          const T *vj = sVj + (size_t)le * C::QC * C::BN + tx * C::TN;
          // element offsets of the four operands from the 16-byte aligned shared base
          constexpr int ALPI = cgcd(C::BM, C::TM);
          constexpr int ALPJ = cgcd(cgcd(C::QC * C::BM, C::BN), C::TN);
          constexpr int ALVI = cgcd(cgcd(C::KC * C::BM, C::QC * C::BM), ALPI);
          constexpr int ALVJ = cgcd(cgcd(C::KC * C::BM + C::EPB * C::QC * C::BM, C::QC * C::BN), cgcd(C::BN, C::TN));
#pragma unroll 2
          for (int k = 0; k < C::QC; k++) {
            T api[C::TM], avi[C::TM], bpj[C::TN], bvj[C::TN];
            lds_vec<T, C::TM, ALPI>(pi + k * C::BM, api);
            lds_vec<T, C::TM, ALVI>(vi + k * C::BM, avi);
            lds_vec<T, C::TN, ALPJ>(pj + k * C::BN, bpj);
            lds_vec<T, C::TN, ALVJ>(vj + k * C::BN, bvj);
#pragma unroll
            for (int i = 0; i < C::TM; i++)
#pragma unroll
              for (int j = 0; j < C::TN; j++) acc[i][j] = fma(bpj[j], avi[i], fma(-api[i], bvj[j], acc[i][j]));
          }
        }
        __syncthreads();
      }
      if (e >= 0 && mine) {
        const int64_t oA = a.offA ? a.offA[e] : e * (int64_t)NSZ;
        if (fem_chk(a.limA < 0 || (oA >= 0 && oA + NSZ <= a.limA), a.err)) {
          T *Ae = static_cast<T *>(a.A) + oA;
#pragma unroll
          for (int i = 0; i < C::TM; i++) {
            const int row = ti * C::BM + ty * C::TM + i;
            if (row >= C::NS) continue;
#pragma unroll
            for (int j = 0; j < C::TN; j++) {
              const int col = tj * C::BN + tx * C::TN + j;
              if (col < C::NS) Ae[col * C::NS + row] = acc[i][j];
            }
          }
        }
      }
    }
  }
  if (a.status != nullptr && ti == 0 && tj == 0)
    for (int l2 = tid; l2 < C::EPB; l2 += nthr) {
      const int64_t v = sE[l2];
      if (v >= 0 && (!ELAST || v % 9 == 0)) a.status[ELAST ? v / 9 : v] = sSt[l2];
    }
  __syncthreads();  // shared memory is reused by the next work item
}

// the block's element group and output tile (or tile pair)
template <class T, class C, int LAW, bool SPLIT>
__device__ __forceinline__ void fma_block(const FmaArgs &a, unsigned char *smem) {
  long long blk = blockIdx.x;
  constexpr bool mirror = fma_mirror<C, LAW, SPLIT>();
  int ti, tj;
  if constexpr (mirror) {
    constexpr int NPAIR = C::TILES * (C::TILES + 1) / 2;
    pair_tiles<C::TILES>((int)(blk % NPAIR), ti, tj);
    blk /= NPAIR;
  } else {
    tj = (int)(blk % C::TILES);
    blk /= C::TILES;
    ti = (int)(blk % C::TILES);
    blk /= C::TILES;
  }
  fma_body<T, C, LAW, SPLIT, mirror>(a, a.qp, static_cast<const T *>(a.phi), blk * (int64_t)C::EPB, a.n, ti, tj,
                                     smem);
}

template <class T, class C, int LAW = 0, bool SPLIT = false>
__global__ void __launch_bounds__(C::NT) fma_kernel(const FmaArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  fma_block<T, C, LAW, SPLIT>(a, smem);
}

// FP64 mirrored tile pairs on CTAs of at most 256 threads, held to two CTAs
// per SM: at p = 7 the correction pass took the kernel to 138 registers and
// one CTA per SM (722 ms per 3,004 prisms); at 128 registers two CTAs run
// (710 ms).
template <class T, class C>
__global__ void __launch_bounds__(C::NT, 2) fma_kernel_pair2(const FmaArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  fma_block<T, C, 0, false>(a, smem);
}

// FP32 kernels with the network stage: the MMA fragments and activations keep
// many registers live, and with small CTAs the compiler then takes so many
// that only one to three CTAs fit per SM; capping them at about 72 registers
// (four CTAs of up to 227 threads) keeps the contraction's latency hidden
// (measured 1.3x on the p = 3 workload).  Shapes too large for two CTAs at
// that cap keep the plain kernel.
template <class C>
constexpr int net_min_blocks() {
  return 65536 / (C::NT * 72) > 4 ? 4 : 65536 / (C::NT * 72);
}
template <class T, class C, bool SPLIT = false>
__global__ void __launch_bounds__(C::NT, (net_min_blocks<C>() >= 2 ? net_min_blocks<C>() : 2))
    fma_kernel_net(const FmaArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  long long blk = blockIdx.x;
  const int tj = (int)(blk % C::TILES);
  blk /= C::TILES;
  const int ti = (int)(blk % C::TILES);
  blk /= C::TILES;
  fma_body<T, C, 2, SPLIT>(a, a.qp, static_cast<const T *>(a.phi), blk * (int64_t)C::EPB, a.n, ti, tj, smem);
}

template <class T, class C, int LAW = 0, bool SPLIT = false>
int launch_fma_cfg(const FmaArgs &a, void *stream) {
  if constexpr (C::MM && !(LAW == 0 && !SPLIT)) return launch_fma_cfg<T, typename C::Plain, LAW, SPLIT>(a, stream);
  if (a.n == 0) return FEM_OK;
  const size_t smem = C::template smem_bytes<T>() + law_smem_bytes<C>(LAW);
  constexpr bool net = LAW == 2 && sizeof(T) == 4 && net_min_blocks<C>() >= 2;
  constexpr bool pair2 = !net && sizeof(T) == 8 && fma_mirror<C, LAW, SPLIT>() && C::NT <= 256;
  void (*kern)(const FmaArgs);
  if constexpr (net)
    kern = fma_kernel_net<T, C, SPLIT>;
  else if constexpr (pair2)
    kern = fma_kernel_pair2<T, C>;
  else
    kern = fma_kernel<T, C, LAW, SPLIT>;
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) {
    set_error(std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(err));
    return FEM_ECUDA;
  }
  const int64_t groups = (a.n + C::EPB - 1) / C::EPB;
  const int64_t grid = groups * (fma_mirror<C, LAW, SPLIT>() && !net ? C::TILES * (C::TILES + 1) / 2 : C::TILES * C::TILES);
  if (grid > 0x7fffffffLL) {
    set_error("too many elements for one launch");
    return FEM_EINVAL;
  }
  kern<<<(unsigned)grid, C::NT, smem, (cudaStream_t)stream>>>(a);
  err = cudaGetLastError();
  if (err != cudaSuccess) {
    set_error(std::string("fma_kernel launch: ") + cudaGetErrorString(err));
    return FEM_ECUDA;
  }
  return FEM_OK;
}

// Tile shapes per precision and degree (ELEM, P, BM, TM, TN, EPB, QC).  FP64
// is bound by the FP64 pipe, which spends the same cycles on a warp
// instruction whatever its active lanes, so its shapes fill whole warps
// (threads per CTA at or just below a multiple of 32) and need only enough
// independent FMAs;
// FP32 is bound by instruction issue, so its micro-tiles are larger and their
// rows 16-byte aligned for vector shared loads; at p = 6 one 200 x 200 tile
// per element (625 threads, 16 points per chunk) beat 2 x 2 tiles of 98 by
// 1.4x (the weighted tile and the geometry are built once, not per tile).
template <class T, int ELEM, int P> struct FmaShape;
template <> struct FmaShape<double, FEM_TET4, 1> { using type = FmaCfg<FEM_TET4, 1, 4, 1, 4, 64, 4>; };
template <> struct FmaShape<double, FEM_PRISM6, 1> { using type = FmaCfg<FEM_PRISM6, 1, 6, 1, 6, 42, 4>; };
template <> struct FmaShape<double, FEM_PRISM6, 2> { using type = FmaCfg<FEM_PRISM6, 2, 18, 3, 6, 14, 3>; };
template <> struct FmaShape<double, FEM_PRISM6, 3> { using type = FmaCfg<FEM_PRISM6, 3, 40, 5, 8, 4, 8>; };
template <> struct FmaShape<double, FEM_PRISM6, 4> {
  using type = FmaCfg<FEM_PRISM6, 4, 75, 3, 3, 1, 5, 4, FEM_RULE_COLLAPSED, true>;
};
template <> struct FmaShape<double, FEM_PRISM6, 5> {
  using type = FmaCfg<FEM_PRISM6, 5, 126, 6, 6, 1, 6, 4, FEM_RULE_COLLAPSED, true>;
};
template <> struct FmaShape<double, FEM_PRISM6, 6> { using type = FmaCfg<FEM_PRISM6, 6, 98, 2, 7, 1, 7>; };
template <> struct FmaShape<double, FEM_PRISM6, 7> { using type = FmaCfg<FEM_PRISM6, 7, 96, 6, 6, 1, 8>; };
template <> struct FmaShape<float, FEM_TET4, 1> { using type = FmaCfg<FEM_TET4, 1, 4, 1, 4, 64, 4>; };
template <> struct FmaShape<float, FEM_PRISM6, 1> { using type = FmaCfg<FEM_PRISM6, 1, 6, 1, 6, 42, 4>; };
template <> struct FmaShape<float, FEM_PRISM6, 2> { using type = FmaCfg<FEM_PRISM6, 2, 18, 3, 6, 28, 3>; };
template <> struct FmaShape<float, FEM_PRISM6, 3> { using type = FmaCfg<FEM_PRISM6, 3, 40, 8, 4, 4, 8>; };
template <> struct FmaShape<float, FEM_PRISM6, 4> { using type = FmaCfg<FEM_PRISM6, 4, 75, 5, 5, 2, 5>; };
template <> struct FmaShape<float, FEM_PRISM6, 5> { using type = FmaCfg<FEM_PRISM6, 5, 128, 8, 8, 1, 8>; };
template <> struct FmaShape<float, FEM_PRISM6, 6> { using type = FmaCfg<FEM_PRISM6, 6, 200, 8, 8, 1, 16>; };
template <> struct FmaShape<float, FEM_PRISM6, 7> { using type = FmaCfg<FEM_PRISM6, 7, 96, 6, 6, 1, 8>; };

// Elasticity: the scalar shapes with K rows of derivatives only (ND = 3); EPB
// counts virtual elements (one 3x3 block of one element each).
template <class T, int P>
struct FmaShapeE {
  using S = typename FmaShape<T, FEM_PRISM6, P>::type;
  using type = FmaCfg<FEM_PRISM6, P, S::BM, S::TM, S::TN, S::EPB, S::QC, 3>;
};
// FP32 at p = 2 and 4: the scalar shapes' larger element groups measured
// slower for the nine-block elasticity (5.5 -> 8.4 ms and 8.3 -> 9.6 ms)
template <> struct FmaShapeE<float, 2> { using type = FmaCfg<FEM_PRISM6, 2, 18, 6, 6, 28, 3, 3>; };
template <> struct FmaShapeE<float, 4> { using type = FmaCfg<FEM_PRISM6, 4, 75, 5, 5, 1, 5, 3>; };
// FP64 p = 4: the 3 x 5 micro-tiles of the scalar form before its mirrored
// 3 x 3 micro-tiles (elasticity does not mirror)
template <> struct FmaShapeE<double, 4> { using type = FmaCfg<FEM_PRISM6, 4, 75, 3, 5, 1, 5, 3>; };

template <class T, bool SPLIT = false>
int launch_fma_elastic(int p, const FmaArgs &a, void *stream) {
  FmaArgs v = a;
  v.n = 9 * a.n;  // virtual elements
  switch (p) {
    case 1: return launch_fma_cfg<T, typename FmaShapeE<T, 1>::type, 0, SPLIT>(v, stream);
    case 2: return launch_fma_cfg<T, typename FmaShapeE<T, 2>::type, 0, SPLIT>(v, stream);
    case 3: return launch_fma_cfg<T, typename FmaShapeE<T, 3>::type, 0, SPLIT>(v, stream);
    case 4: return launch_fma_cfg<T, typename FmaShapeE<T, 4>::type, 0, SPLIT>(v, stream);
    case 5: return launch_fma_cfg<T, typename FmaShapeE<T, 5>::type, 0, SPLIT>(v, stream);
    case 6: return launch_fma_cfg<T, typename FmaShapeE<T, 6>::type, 0, SPLIT>(v, stream);
    case 7: return launch_fma_cfg<T, typename FmaShapeE<T, 7>::type, 0, SPLIT>(v, stream);
  }
  return FEM_EINVAL;
}

// The paper's prism rule (Table 1's point counts): the collapsed rule's
// shapes with its points (constant coefficients).
template <class S>
using Table1Cfg = FmaCfg<S::ELEM, S::P, S::BM, S::TM, S::TN, S::EPB, S::QC, S::ND, FEM_RULE_TABLE1, S::MM>;

template <class T>
int launch_fma_table1(int p, const FmaArgs &a, void *stream) {
  switch (p) {
    case 1: return launch_fma_cfg<T, Table1Cfg<typename FmaShape<T, FEM_PRISM6, 1>::type>>(a, stream);
    case 2: return launch_fma_cfg<T, Table1Cfg<typename FmaShape<T, FEM_PRISM6, 2>::type>>(a, stream);
    case 3: return launch_fma_cfg<T, Table1Cfg<typename FmaShape<T, FEM_PRISM6, 3>::type>>(a, stream);
    case 4: return launch_fma_cfg<T, Table1Cfg<typename FmaShape<T, FEM_PRISM6, 4>::type>>(a, stream);
    case 5: return launch_fma_cfg<T, Table1Cfg<typename FmaShape<T, FEM_PRISM6, 5>::type>>(a, stream);
    case 6: return launch_fma_cfg<T, Table1Cfg<typename FmaShape<T, FEM_PRISM6, 6>::type>>(a, stream);
    case 7: return launch_fma_cfg<T, Table1Cfg<typename FmaShape<T, FEM_PRISM6, 7>::type>>(a, stream);
  }
  return FEM_EINVAL;
}

// linear elastostatics with the paper's rule (a.n real elements, 9 blocks each)
template <class T>
int launch_fma_elastic_table1(int p, const FmaArgs &a, void *stream) {
  FmaArgs v = a;
  v.n = 9 * a.n;  // virtual elements
  switch (p) {
    case 1: return launch_fma_cfg<T, Table1Cfg<typename FmaShapeE<T, 1>::type>>(v, stream);
    case 2: return launch_fma_cfg<T, Table1Cfg<typename FmaShapeE<T, 2>::type>>(v, stream);
    case 3: return launch_fma_cfg<T, Table1Cfg<typename FmaShapeE<T, 3>::type>>(v, stream);
    case 4: return launch_fma_cfg<T, Table1Cfg<typename FmaShapeE<T, 4>::type>>(v, stream);
    case 5: return launch_fma_cfg<T, Table1Cfg<typename FmaShapeE<T, 5>::type>>(v, stream);
    case 6: return launch_fma_cfg<T, Table1Cfg<typename FmaShapeE<T, 6>::type>>(v, stream);
    case 7: return launch_fma_cfg<T, Table1Cfg<typename FmaShapeE<T, 7>::type>>(v, stream);
  }
  return FEM_EINVAL;
}

template <class T, int LAW = 0, bool SPLIT = false>
int launch_fma_any(int elem, int p, const FmaArgs &a, void *stream) {
  if (elem == FEM_TET4) return launch_fma_cfg<T, typename FmaShape<T, FEM_TET4, 1>::type, LAW, SPLIT>(a, stream);
  switch (p) {
    case 1: return launch_fma_cfg<T, typename FmaShape<T, FEM_PRISM6, 1>::type, LAW, SPLIT>(a, stream);
    case 2: return launch_fma_cfg<T, typename FmaShape<T, FEM_PRISM6, 2>::type, LAW, SPLIT>(a, stream);
    case 3: return launch_fma_cfg<T, typename FmaShape<T, FEM_PRISM6, 3>::type, LAW, SPLIT>(a, stream);
    case 4: return launch_fma_cfg<T, typename FmaShape<T, FEM_PRISM6, 4>::type, LAW, SPLIT>(a, stream);
    case 5: return launch_fma_cfg<T, typename FmaShape<T, FEM_PRISM6, 5>::type, LAW, SPLIT>(a, stream);
    case 6: return launch_fma_cfg<T, typename FmaShape<T, FEM_PRISM6, 6>::type, LAW, SPLIT>(a, stream);
    case 7: return launch_fma_cfg<T, typename FmaShape<T, FEM_PRISM6, 7>::type, LAW, SPLIT>(a, stream);
  }
  return FEM_EINVAL;
}

}  // namespace fem
