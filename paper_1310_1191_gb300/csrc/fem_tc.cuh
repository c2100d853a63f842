// Tensor-core contraction of the element matrices on sm_103a (tcgen05, TMEM,
// bulk TMA copies, mbarrier pipeline), BF16 or FP16 operands split hi + lo,
// FP32 accumulation.
//
// Per element the weak form is A_e = Phi^T T_e (K = 4 NQ; Algorithm 2 with the
// sparse c, see fem_fma.cuh).  Transposed, A_e^T[j][i] = sum_k T_e[k][j] Phi[k][i],
// so the MMA rows are (element, j) pairs and the columns i:
//     D[(e,j)][i] = sum_k A[(e,j)][k] B[i][k],  A = T_e^T (per element), B = Phi^T.
// Rows of all elements are stacked densely, NS+1 rows per element: rows
// j < NS give column j of A_e, and an extra row whose weighted tile is
// (S_Q, 0, 0, 0) per point (S_Q = w det f) gives the load vector
// b_e[i] = sum_Q S_Q phi[Q][0][i] from the same MMAs.  An M tile of 128 rows
// therefore has no padding whatever NS is; N is NS rounded up to 16 (split in
// two MMAs of N = 144 at p = 7).
//
// hi + lo split: x = hi(x) + lo(x) with hi, lo 16-bit; the product uses
// hi*hi + hi*lo + lo*hi (three MMAs into one FP32 accumulator), dropping
// lo*lo.  For FP16 both operands are scaled by powers of two (Phi per degree,
// T per element from a bound on |G| |Phi|) so the largest magnitude sits near
// 2^14; the epilogue removes the scale exactly.
//
// Linear elastostatics (ELAS) reuses the whole pipeline: each
// element's 3x3 blocks are nine row blocks ("virtual elements", NS+1 rows
// each), the value row of T is zero, and the blocks (i, 0) carry the load
// vector b^e[i] in their extra row (see the producers).
//
// CTA roles (one CTA per SM, each CTA owns a contiguous range of M tiles;
// 512 threads, or 768 where TcCfg gives 16 producer warps):
//   warp 0, lane 0   : bulk-copies the Phi^T hi/lo image of each K chunk (TMA);
//   warp 1, lane 0   : issues tcgen05.mma and commits (warp 1 owns TMEM);
//   warps 6..        : the producers, PRODW warps: build the A tiles (T^T hi/lo)
//                      of each K chunk from the point records, 2 or 4 threads
//                      per row;
//   warps 2..5 and the last two : FP64 geometry of the elements each tile
//                      brings in -> point records in a ring of element slots
//                      (consecutive tiles share elements, so each element is
//                      computed once); warps 2..5 then drain TMEM and write
//                      A_e / b_e of the previous tile (warp w reads TMEM lanes
//                      32 (w % 4) ..).
// Every mbarrier wait is bounded (about a second); a CTA whose wait expires
// sets the library's device error word, marks its elements FEM_ST_TIMEOUT,
// waits for its own copies and MMAs, frees TMEM and returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "fem_geometry.cuh"
#include "fem_internal.h"
#include "fem_law.cuh"
#include "fem_tc_ptx.cuh"

namespace fem {

template <int P, bool ELAS = false, int LAW = 0, int RULE = FEM_RULE_COLLAPSED>
struct TcCfg {
  static constexpr int NS = ns_of(FEM_PRISM6, P), NQ = nq_of(FEM_PRISM6, P, RULE);
  static constexpr int L = NS + 1;  // MMA rows per element
  static constexpr int BM = 128;
  static constexpr int KC = 32;     // K per stage: 8 points x 4 derivatives
  static constexpr int QC = KC / 4;
  static constexpr int KP = (4 * NQ + KC - 1) / KC * KC;
  static constexpr int NCH = KP / KC;
  static constexpr int NQP = KP / 4;
  static constexpr int NP = (NS + 15) / 16 * 16;
  static constexpr int NSPLIT = NP > 256 ? 2 : 1;
  static constexpr int NH = NP / NSPLIT;
  static constexpr int MAXEL = (BM - 1 + L - 1) / L + 1;
  // accumulators per tile: with KACC = 2 the two K steps of each chunk go to
  // two accumulators whose MMAs alternate (no MMA waits for the one before
  // it on the same accumulator), summed in FP32 by the epilogue; where TMEM
  // holds four (p <= 5), else one (p = 7 alternates its two N halves)
  static constexpr int KACC = 4 * NP <= 512 ? 2 : 1;
  static constexpr int NACC = 2 * KACC * NP <= 512 ? 2 : 1;  // TMEM accumulator buffers (tiles in flight)
  static constexpr int TCOLS_NEED = NACC * KACC * NP;
  static constexpr int TMEM_COLS = TCOLS_NEED <= 32 ? 32 : TCOLS_NEED <= 64 ? 64 : TCOLS_NEED <= 128 ? 128
                                   : TCOLS_NEED <= 256 ? 256 : 512;
  // operand stages: as many as shared memory holds (the Phi^T copies come
  // from L2, partly across the die boundary, so deep rings hide their latency)
  static constexpr int STAGES = (P == 7 ? 3 : P == 6 ? 4 : P == 5 ? 5 : P == 4 ? 7 : 8) - (LAW != 0 && P >= 4 ? 1 : 0);
  // producer warps: 8 (two threads per tile row, 4 points of each chunk
  // each) or 16 (four threads per row, 2 points each; measured 1.2x at p = 5
  // and 1.1x at p = 6, the same at p = 4, 7 % slower at p = 7); the CTA is
  // 6 + PRODW + 2 warps (loader, MMA, 4 epilogue/geometry, producers,
  // 2 geometry), so 16 producer warps make a 768-thread CTA with a budget of
  // 85 registers per thread
  static constexpr int PRODW = (P >= 3 && P <= 6 && LAW == 0) ? 16 : 8;
  static constexpr int THREADS = (8 + PRODW) * 32;
  static constexpr int NPROD = PRODW * 32, PPR = NPROD / BM, QH = QC / PPR;
  static constexpr int GEOW0 = 6 + PRODW;  // first geometry-only warp
  // p <= 4: the geometry pass bounds the kernel (tiles have few K chunks), so
  // the inputs of its next pass are fetched ahead (cp.async), its J factors
  // go one value per thread and its point records are spread evenly over the
  // SM sub-partitions; above, the plain forms measured faster
  static constexpr bool GEO_FINE = P <= 4;
  // chunks of Phi values the producers keep in flight (registers)
  static constexpr int PD = PRODW == 16 ? 2 : 3;
  static constexpr int A_BYTES = BM * KC * 2;  // one half (hi or lo)
  static constexpr int B_BYTES = NP * KC * 2;
  static constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int SBO = (KC / 8) * 128;   // 8-row group stride in a stage tile
  static constexpr int NREC = 18 + (ELAS ? 5 : 11);  // coordinates + coefficients
  static constexpr int NZ = P + 1, NAB = ntri_of(P, RULE);  // zeta levels x triangle points (J factors)
  // Each CTA owns a contiguous range of tiles, so consecutive tiles share
  // elements; point records live in a ring of RING element slots (slot =
  // element mod RING) and every element's geometry is computed once per CTA.
  // RING covers the elements of two consecutive tiles (the tile being built
  // and the next one), MAXEL those of one tile (new elements per pass).
  static constexpr int RING = (2 * BM - 1 + L - 1) / L + 1;
  static constexpr int GSLOT = NQP * 12;  // floats of point records per element
  // shared layout (bytes from a 1024-aligned base)
  static constexpr size_t OFF_G = (size_t)STAGES * STAGE_BYTES;                // float [RING][NQP][12]
  static constexpr size_t OFF_X = OFF_G + (size_t)RING * GSLOT * 4;            // double [2][MAXEL][NREC]
  static constexpr size_t OFF_ED = OFF_X + (size_t)2 * MAXEL * NREC * 8;       // double [MAXEL][21]
  static constexpr size_t OFF_ZF = OFF_ED + (size_t)MAXEL * kEdgeRec * 8;      // double [MAXEL][NZ][9]
  static constexpr size_t OFF_XF = OFF_ZF + (size_t)MAXEL * NZ * kZf * 8;      // double [MAXEL][NAB][3]
  static constexpr size_t OFF_ZR = OFF_XF + (size_t)MAXEL * NAB * kXf * 8;     // float [MAXEL][NZ][4]
  static constexpr size_t OFF_CF = OFF_ZR + (size_t)MAXEL * NZ * 16;           // float [MAXEL][12]
  static constexpr size_t OFF_W = OFF_CF + (size_t)MAXEL * 48;                 // float [NQP] weights
  static constexpr size_t OFF_QF = OFF_W + (size_t)NQP * 4;                    // double [NZ][2], [NAB][3] rule factors
  static constexpr size_t OFF_RS = OFF_QF + (size_t)(2 * NZ + 3 * NAB) * 8;    // per slot: 7 x [RING] words
  static constexpr size_t OFF_EC = (OFF_RS + 28 * (size_t)RING + 15) / 16 * 16;   // float [RING][8] (elasticity)
  // coefficient law: field coefficients of the pass's new elements; network
  // weights and the inputs of the pass's points (network only)
  static constexpr size_t OFF_UC = OFF_EC + 32 * (size_t)RING;                               // float [MAXEL][NS]
  static constexpr size_t OFF_MLP = (OFF_UC + (LAW ? 4 * (size_t)MAXEL * NS : 0) + 15) / 16 * 16;
  static constexpr size_t OFF_XIN = OFF_MLP + (LAW == 2 ? (size_t)kMlpSmemBytes : 0);       // float [MAXEL][NQP][2]
  static constexpr size_t OFF_BAR = (OFF_XIN + (LAW == 2 ? 8 * (size_t)MAXEL * NQP : 0) + 15) / 16 * 16;
  static constexpr int NBAR = 2 * STAGES + 9;
  static constexpr size_t OFF_MISC = OFF_BAR + 8 * NBAR;
  static constexpr size_t SMEM = OFF_MISC + 16 + 1024;
  static_assert(NH % 16 == 0 && NH >= 16 && NH <= 256, "MMA N out of range");
  static constexpr bool PAIRS = STAGES >= 4;  // producers hand chunks over in pairs
  static_assert(NQP >= NQ, "padding");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

// warp roles of the 512-thread CTA
// warp roles of the CTA (C::THREADS threads): warp 0 loader, warp 1 MMA,
// warps 2..5 epilogue and geometry, warps 6 .. 6 + PRODW - 1 producers, the
// last two warps (C::GEOW0, C::GEOW0 + 1) geometry only
constexpr int kEpiWarp0 = 2;    // 4 warps: TMEM lanes 32 (w % 4) .. + 31; also geometry
constexpr int kProdWarp0 = 6;
constexpr int kNEpi = 128, kNGeo = 192;  // geometry: warps 2..5 and the last two

struct TcArgs {
  int64_t n;
  const double *coords;
  const double *coeffs;
  int64_t cstride;
  const double *qp;
  const float *phiq;     // Phi as [NQ][NS][4] float4 (value + 3 derivatives of function j at point q)
  const uint16_t *img;  // Phi^T hi/lo image per K chunk
  float phimax;         // max |Phi| (FP32 table)
  int aphi;             // power-of-two exponent applied to the image (FP16)
  void *A;
  void *b;
  int32_t *status;
  int layout;
  int *err;
  int stall;  // test hook: the loader issues no copies, so the pipeline's waits expire
  // mixed-degree plans (scalar form): element k of this launch is perm[k] of
  // the mesh, its A_e / b_e start at offA / offb[perm[k]] (all NULL: k itself,
  // dense outputs)
  const int64_t *perm;
  const int64_t *offA;
  const int64_t *offb;
  // nonlinear coefficient law (D = k(u, |grad u|) I per point)
  const float *ucoef;     // [n][NS] field coefficients
  const float *phiT;      // point-major table [NS][NQ][4] (FP32)
  const float *mlpw;      // network parameters (FP32 values of BF16 weights)
  const uint32_t *mlpw2;  // its W2 as BF16 pairs
  float nrm[4], box[4];
  int law_iters;  // Newton steps of the exact law
  int hw_tanh;    // network activations from tanh.approx.f32
  int64_t limA, limb;  // checked builds: values of A and b (negative: not checked)
  int64_t nmesh;       // checked builds: element ids from perm lie below it (negative: not checked)
};

constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s

// x = hi + lo for two values at once: hi = rn16(x), lo = rn16(x - hi), packed
// as two 16-bit halves (first value in the low half).
template <bool F16>
__device__ __forceinline__ uint32_t split_pack(float x0, float x1, uint32_t &lo_word) {
  if (F16) {
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
    lo_word = *reinterpret_cast<const uint32_t *>(&l);
    return *reinterpret_cast<const uint32_t *>(&h);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    lo_word = *reinterpret_cast<const uint32_t *>(&l);
    return *reinterpret_cast<const uint32_t *>(&h);
  }
}

// ELAS: linear elastostatics (the model problem).  The rows are
// (virtual element v, trial function r) with v = 9 e + 3 i + k the block
// (i, k) of element e; the point records hold adj J, w / det J and w det J,
// and the producers form each block's weighted rows from them (see below).
// LAW 1 / 2 (scalar form, BF16): the coefficient stage of the nonlinear law
// in the geometry warps -- u and grad u from the element's field
// coefficients, k from the exact law or from the network (its 64x64 layer on
// warp-level MMAs, the exact law outside its box), D = k I.
template <int P, bool F16, bool ELAS = false, int LAW = 0, int RULE = FEM_RULE_COLLAPSED>
__global__ void __launch_bounds__(TcCfg<P, ELAS, LAW, RULE>::THREADS, 1) tc_kernel(const TcArgs a) {
  using C = TcCfg<P, ELAS, LAW, RULE>;
  static_assert(LAW == 0 || (!F16 && !ELAS), "the law runs in the BF16 scalar form");
  constexpr int VPE = ELAS ? 9 : 1;  // row blocks (virtual elements) per element
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float *sG = reinterpret_cast<float *>(sm + C::OFF_G);          // [RING][NQP][12] point records
  double *sX = reinterpret_cast<double *>(sm + C::OFF_X);        // [2][MAXEL][NREC] new elements of a pass
  double *sEd = reinterpret_cast<double *>(sm + C::OFF_ED);      // [MAXEL][21]
  double *sZF = reinterpret_cast<double *>(sm + C::OFF_ZF);      // [MAXEL][NZ][9]
  double *sXF = reinterpret_cast<double *>(sm + C::OFF_XF);      // [MAXEL][NAB][3]
  float *sZR = reinterpret_cast<float *>(sm + C::OFF_ZR);        // [MAXEL][NZ][4] adj row 2, FP32
  float *sCF = reinterpret_cast<float *>(sm + C::OFF_CF);        // [MAXEL][12] coefficients, FP32
  float *sW = reinterpret_cast<float *>(sm + C::OFF_W);          // [NQP] quadrature weights, FP32
  // per zeta level (lo, hi) = ((1 - zeta) / 2, (1 + zeta) / 2), then per
  // triangle point (h0, h1, h2) = ((1 - xi - eta) / 2, xi / 2, eta / 2):
  // the weights of the edge vectors in J (see edge_record)
  double *sQF = reinterpret_cast<double *>(sm + C::OFF_QF);
  float *sEC = reinterpret_cast<float *>(sm + C::OFF_EC);        // [RING][8] lambda, mu, f (elasticity)
  float *sUC = reinterpret_cast<float *>(sm + C::OFF_UC);        // [MAXEL][NS] field coefficients (law)
  float *sMP = reinterpret_cast<float *>(sm + C::OFF_MLP);       // network: FP32 W1 b1 b2 W3 b3 (law 2)
  uint32_t *sW2 = reinterpret_cast<uint32_t *>(sMP + kMlpSmall);  // network: W2 BF16 rows (law 2)
  float *sXin = reinterpret_cast<float *>(sm + C::OFF_XIN);      // [MAXEL][NQP][2] network inputs (law 2)
  float *sInv = reinterpret_cast<float *>(sm + C::OFF_RS);       // [RING] matrix-row unscale
  float *sInvB = sInv + C::RING;                                 // [RING] load-vector-row unscale
  float *sScl = sInvB + C::RING;                                 // [RING] matrix-row scale (FP16)
  float *sScB = sScl + C::RING;                                  // [RING] load-vector-row scale (FP16)
  int *sSt = reinterpret_cast<int *>(sScB + C::RING);            // [RING] status bits
  unsigned *sBnd = reinterpret_cast<unsigned *>(sSt + C::RING);  // [RING] bound of |G| (FP16)
  unsigned *sBndB = sBnd + C::RING;                              // [RING] bound of |S| (FP16)
  uint64_t *bar_full = reinterpret_cast<uint64_t *>(sm + C::OFF_BAR);
  uint64_t *bar_empty = bar_full + C::STAGES;
  uint64_t *bar_accf = bar_empty + C::STAGES;  // [2]
  uint64_t *bar_acce = bar_accf + 2;           // [2]
  uint64_t *bar_gfull = bar_acce + 2;          // [2]
  uint64_t *bar_gempty = bar_gfull + 2;        // [2]
  uint64_t *bar_fin = bar_gempty + 2;
  uint32_t *sTmem = reinterpret_cast<uint32_t *>(sm + C::OFF_MISC);
  volatile int *sAbort = reinterpret_cast<volatile int *>(sm + C::OFF_MISC + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nrows = a.n * VPE * C::L;
  const int64_t ntiles = (nrows + C::BM - 1) / C::BM;
  // this CTA's contiguous range of M tiles
  const int64_t t_begin = (int64_t)blockIdx.x * ntiles / gridDim.x;
  const int64_t t_end = ((int64_t)blockIdx.x + 1) * ntiles / gridDim.x;
  for (int q = tid; q < C::NQP; q += blockDim.x) sW[q] = q < C::NQ ? (float)a.qp[4 * q + 3] : 0.f;
  // the rule's zeta levels and triangle points (point q = iz NAB + iab)
  for (int k = tid; k < C::NZ; k += blockDim.x) {
    const double ze = a.qp[4 * (k * C::NAB) + 2];
    sQF[2 * k] = 0.5 * (1.0 - ze);
    sQF[2 * k + 1] = 0.5 * (1.0 + ze);
  }
  for (int k = tid; k < C::NAB; k += blockDim.x) {
    const double xi = a.qp[4 * k], eta = a.qp[4 * k + 1];
    double *h = sQF + 2 * C::NZ + 3 * k;
    h[0] = 0.5 * (1.0 - xi - eta);
    h[1] = 0.5 * xi;
    h[2] = 0.5 * eta;
  }
  if (LAW == 2) {  // network parameters (layout of the CUDA-core law kernels)
    constexpr int H = kMlpH;
    for (int idx = tid; idx < kMlpSmall; idx += blockDim.x) {
      float v = 0.f;
      if (idx < 3 * H) v = a.mlpw[idx];                                      // W1, b1
      else if (idx < 5 * H + 1) v = a.mlpw[3 * H + H * H + (idx - 3 * H)];  // b2, W3, b3
      sMP[idx] = v;
    }
    for (int idx = tid; idx < H * (H / 2); idx += blockDim.x)
      sW2[(idx / (H / 2)) * (kW2Stride / 2) + idx % (H / 2)] = a.mlpw2[idx];
  }

  if (tid == 0) {
    for (int s = 0; s < C::STAGES; s++) {
      ptx::mbar_init(&bar_full[s], C::PRODW + 1);  // one arrival per producer warp + the loader
      ptx::mbar_init(&bar_empty[s], 1);
    }
    for (int i = 0; i < 2; i++) {
      ptx::mbar_init(&bar_accf[i], 1);
      ptx::mbar_init(&bar_acce[i], kNEpi / 32);
      ptx::mbar_init(&bar_gfull[i], 1);
      ptx::mbar_init(&bar_gempty[i], C::PRODW + kNEpi / 32);
    }
    ptx::mbar_init(bar_fin, 1);
    *sAbort = 0;
    ptx::fence_mbar_init();
    ptx::fence_proxy_async();
  }
  if (warp == 1) {
    ptx::tmem_alloc(sTmem, C::TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *sTmem;
  const uint32_t stage0 = ptx::smem_u32(sm);

  auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
    if (*sAbort) return false;
    if (ptx::mbar_wait(bar, parity, kWaitLimitNs)) return true;
    *sAbort = 1;
    return false;
  };
  // element range of tile t
  auto tile_elems = [&](int64_t t, int64_t &e_first, int &nel) {
    const int64_t R0 = t * C::BM;
    e_first = R0 / C::L / VPE;
    int64_t e_last = (R0 + C::BM - 1) / C::L / VPE;
    if (e_last > a.n - 1) e_last = a.n - 1;
    nel = (int)(e_last - e_first + 1);
  };

  if (warp == 0) {
    // ---------------- Phi^T image loader (TMA bulk copies) ----------------
    if (lane == 0) {
      // issued[s]: 1 + the round of the last copy issued into stage s (0: none)
      uint32_t issued[C::STAGES];
#pragma unroll
      for (int s = 0; s < C::STAGES; s++) issued[s] = 0;
      uint32_t g = 0;
      for (int64_t t = t_begin; t < t_end && !*sAbort; t++) {
        for (int c = 0; c < C::NCH; c++, g++) {
          const int s = g % C::STAGES;
          const uint32_t round = g / C::STAGES;
          if (!wait(&bar_empty[s], (round & 1) ^ 1)) break;
          if (a.stall) continue;  // nothing arrives on full[s]: the consumers' waits run out
          unsigned char *dst = sm + (size_t)s * C::STAGE_BYTES + 2 * C::A_BYTES;
          ptx::mbar_arrive_expect_tx(&bar_full[s], 2 * C::B_BYTES);
          ptx::bulk_g2s(dst, reinterpret_cast<const unsigned char *>(a.img) + (size_t)c * 2 * C::B_BYTES,
                        2 * C::B_BYTES, &bar_full[s]);
          issued[s] = round + 1;
        }
      }
      if (*sAbort) {
        // Let this CTA's copies in flight land before it leaves: the last copy
        // into stage s completes phase issued[s] - 1 of full[s], and only this
        // thread arms full[s], so that phase cannot be overtaken.  Each wait
        // is bounded like every other.
        for (int s = 0; s < C::STAGES; s++)
          if (issued[s]) ptx::mbar_wait(&bar_full[s], (issued[s] - 1) & 1, kWaitLimitNs);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_f16(!F16, C::BM, C::NH);
      uint32_t g = 0, tt = 0;
      for (int64_t t = t_begin; t < t_end && !*sAbort; t++, tt++) {
        const uint32_t ab = C::NACC == 2 ? (tt & 1) : 0, use = tt / C::NACC;
        if (!wait(&bar_acce[ab], (use & 1) ^ 1)) break;
        ptx::tc_fence_after();
        const uint32_t dacc = tmem + ab * C::KACC * C::NP;
        bool ok = true;
        for (int c = 0; c < C::NCH; c++, g++) {
          const int s = g % C::STAGES;
          const uint32_t round = g / C::STAGES;
          if (!wait(&bar_full[s], round & 1)) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t aH = stage0 + s * C::STAGE_BYTES, aL = aH + C::A_BYTES;
          const uint32_t bH = aL + C::A_BYTES, bL = bH + C::B_BYTES;
          if constexpr (C::KACC == 2) {
            // K step ks into accumulator ks; the products alternate between
            // the two: hi.hi (0), hi.hi (1), hi.lo (0), hi.lo (1), lo.hi (0), lo.hi (1)
            static_assert(C::KC / 16 == 2 && C::NSPLIT == 1, "two K steps, one N part");
            uint64_t adH[2], adL[2], bdH[2], bdL[2];
#pragma unroll
            for (int ks = 0; ks < 2; ks++) {
              adH[ks] = ptx::smem_desc(aH + ks * 256, 128, C::SBO);
              adL[ks] = ptx::smem_desc(aL + ks * 256, 128, C::SBO);
              bdH[ks] = ptx::smem_desc(bH + ks * 256, 128, C::SBO);
              bdL[ks] = ptx::smem_desc(bL + ks * 256, 128, C::SBO);
            }
            const uint32_t acc0 = c > 0 ? 1u : 0u;
#pragma unroll
            for (int ks = 0; ks < 2; ks++) ptx::mma_f16(dacc + ks * C::NP, adH[ks], bdH[ks], idesc, acc0);
#pragma unroll
            for (int ks = 0; ks < 2; ks++) ptx::mma_f16(dacc + ks * C::NP, adH[ks], bdL[ks], idesc, 1u);
#pragma unroll
            for (int ks = 0; ks < 2; ks++) ptx::mma_f16(dacc + ks * C::NP, adL[ks], bdH[ks], idesc, 1u);
          } else {
#pragma unroll
            for (int ks = 0; ks < C::KC / 16; ks++) {
              const uint64_t adH = ptx::smem_desc(aH + ks * 256, 128, C::SBO);
              const uint64_t adL = ptx::smem_desc(aL + ks * 256, 128, C::SBO);
#pragma unroll
              for (int h = 0; h < C::NSPLIT; h++) {
                const uint32_t boff = h * (C::NH / 8) * C::SBO + ks * 256;
                const uint64_t bdH = ptx::smem_desc(bH + boff, 128, C::SBO);
                const uint64_t bdL = ptx::smem_desc(bL + boff, 128, C::SBO);
                const uint32_t d = dacc + h * C::NH;
                ptx::mma_f16(d, adH, bdH, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                ptx::mma_f16(d, adH, bdL, idesc, 1u);
                ptx::mma_f16(d, adL, bdH, idesc, 1u);
              }
            }
          }
          ptx::mma_commit(&bar_empty[s]);
        }
        if (!ok) break;
        ptx::mma_commit(&bar_accf[ab]);
      }
      // make sure no MMA is still running before TMEM is released
      ptx::mma_commit(bar_fin);
      ptx::mbar_wait(bar_fin, 0, kWaitLimitNs);
    }
  } else if (warp >= kProdWarp0 && warp < C::GEOW0) {
    // ---------------- producers: A tiles (T^T hi/lo) of each K chunk ----------------
    const int pt = tid - kProdWarp0 * 32;
    const int rl = pt & 127;       // tile row
    const int half = pt >> 7;      // points QH half .. QH half + QH - 1 of each chunk
    constexpr int QH = C::QH;
    uint32_t tt = 0;
    for (int64_t t = t_begin; t < t_end; t++, tt++) {
      const int b = tt & 1;
      const uint32_t use = tt >> 1;
      if (!__all_sync(0xffffffffu, wait(&bar_gfull[b], use & 1))) break;
      int64_t e_first;
      int nel;
      tile_elems(t, e_first, nel);
      const int64_t r = t * C::BM + rl;
      const bool valid = r < nrows;
      const int64_t v = valid ? r / C::L : e_first * VPE;  // virtual element
      const int64_t e = v / VPE;
      const int j = valid ? (int)(r % C::L) : 0;
      const float *gbase = sG + (size_t)(e % C::RING) * C::GSLOT;
      const bool arow = valid && j < C::NS;
      // elasticity: block (bi, bk) of the row, the element's lambda, mu, f_bi
      const int blk = (int)(v % VPE), bi = blk / 3, bk = blk % 3;
      float lam = 0.f, mu = 0.f, fbi = 0.f;
      if (ELAS) {
        const float *ec = sEC + (e % C::RING) * 8;
        lam = ec[0];
        mu = ec[1];
        fbi = bi == 0 ? ec[2] : (bi == 1 ? ec[3] : ec[4]);
      }
      // Phi values of the next PD - 1 chunks are in flight while a chunk is
      // built (ring of PD register sets, indexed statically by unrolling)
      float fr[C::PD][QH][4];
      auto load_phi = [&](int c, float (&f)[QH][4]) {
#pragma unroll
        for (int qq = 0; qq < QH; qq++) {
          const int q = c * C::QC + half * QH + qq;
          if (arow && q < C::NQ) {
            // one 16-byte load; the rows j of a warp read consecutive float4s
            const float4 v = __ldg(reinterpret_cast<const float4 *>(a.phiq) + (size_t)q * C::NS + j);
            f[qq][0] = v.x;
            f[qq][1] = v.y;
            f[qq][2] = v.z;
            f[qq][3] = v.w;
          } else {
            f[qq][0] = f[qq][1] = f[qq][2] = f[qq][3] = 0.f;
          }
        }
      };
#pragma unroll
      for (int u = 0; u < C::PD - 1; u++)
        if (u < C::NCH) load_phi(u, fr[u]);
      bool ok = true;
      const uint32_t g0 = tt * C::NCH;
      // builds chunk c from the Phi values in f; false if a wait expired
      auto build = [&](int c, const float (&f)[QH][4]) -> bool {
        const uint32_t g = g0 + c;
        const int s = g % C::STAGES;
        const uint32_t round = g / C::STAGES;
        // warp-uniform: the stage is handed over by one arrival per warp
        if (!__all_sync(0xffffffffu, wait(&bar_empty[s], (round & 1) ^ 1))) return false;
        uint32_t hw[QH * 2], lw[QH * 2];
#pragma unroll
        for (int qq = 0; qq < QH; qq++) {
          const int q = c * C::QC + half * QH + qq;
          float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
          if (valid && q < C::NQ) {
            const float4 *g4 = reinterpret_cast<const float4 *>(gbase + q * 12);
            const float4 ga = g4[0], gb = g4[1], gc = g4[2];
            if (ELAS) {
              // record: adj J row-major (a[k][m], k reference, m physical
              // direction) | w / det | w det.  Block (bi, bk):
              //   G[a][b] = (w/det) (lam a[a][bi] a[b][bk] + mu a[a][bk] a[b][bi]
              //                      + d_ik mu (a[a] . a[b])),
              // so with u = adj^T (f1, f2, f3) (det J times the physical gradient)
              //   t_{1+a} = (w/det) (lam a[a][bi] u_bk + mu a[a][bk] u_bi + d_ik mu a[a] . u);
              // the value row is zero, the load-vector row (w det f_bi, 0, 0, 0).
              const float a00 = ga.x, a01 = ga.y, a02 = ga.z, a10 = ga.w, a11 = gb.x, a12 = gb.y;
              const float a20 = gb.z, a21 = gb.w, a22 = gc.x, sw = gc.y;
              if (arow) {
                const float f1 = f[qq][1], f2 = f[qq][2], f3 = f[qq][3];
                const float u0 = a00 * f1 + a10 * f2 + a20 * f3;
                const float u1 = a01 * f1 + a11 * f2 + a21 * f3;
                const float u2 = a02 * f1 + a12 * f2 + a22 * f3;
                const float ubi = bi == 0 ? u0 : (bi == 1 ? u1 : u2);
                const float ubk = bk == 0 ? u0 : (bk == 1 ? u1 : u2);
                const float li = sw * lam * ubk, mi = sw * mu * ubi, dm = bi == bk ? sw * mu : 0.f;
                const float c0i = bi == 0 ? a00 : (bi == 1 ? a01 : a02);
                const float c1i = bi == 0 ? a10 : (bi == 1 ? a11 : a12);
                const float c2i = bi == 0 ? a20 : (bi == 1 ? a21 : a22);
                const float c0k = bk == 0 ? a00 : (bk == 1 ? a01 : a02);
                const float c1k = bk == 0 ? a10 : (bk == 1 ? a11 : a12);
                const float c2k = bk == 0 ? a20 : (bk == 1 ? a21 : a22);
                t1 = c0i * li + c0k * mi + dm * (a00 * u0 + a01 * u1 + a02 * u2);
                t2 = c1i * li + c1k * mi + dm * (a10 * u0 + a11 * u1 + a12 * u2);
                t3 = c2i * li + c2k * mi + dm * (a20 * u0 + a21 * u1 + a22 * u2);
              } else {
                t0 = bk == 0 ? gc.z * fbi : 0.f;
              }
            } else {
              // G00 G01 G02 G03 | G11 G12 G13 G22 | G23 G33 GS -
              if (arow) {
                const float f0 = f[qq][0], f1 = f[qq][1], f2 = f[qq][2], f3 = f[qq][3];
                t0 = ga.x * f0 + ga.y * f1 + ga.z * f2 + ga.w * f3;
                t1 = gb.x * f1 + gb.y * f2 + gb.z * f3;
                t2 = gb.y * f1 + gb.w * f2 + gc.x * f3;
                t3 = gb.z * f1 + gc.x * f2 + gc.y * f3;
              } else {
                t0 = gc.z;
              }
            }
          }
          hw[2 * qq] = split_pack<F16>(t0, t1, lw[2 * qq]);
          hw[2 * qq + 1] = split_pack<F16>(t2, t3, lw[2 * qq + 1]);
        }
        unsigned char *aH = sm + (size_t)s * C::STAGE_BYTES;
        unsigned char *aL = aH + C::A_BYTES;
#pragma unroll
        for (int k2 = 0; k2 < QH / 2; k2++) {  // 16-byte core-matrix rows: 2 points each
          const int kk = half * (QH / 2) + k2;
          const size_t off = (size_t)((rl >> 3) * (C::KC / 8) + kk) * 128 + (rl & 7) * 16;
          *reinterpret_cast<uint4 *>(aH + off) = make_uint4(hw[4 * k2], hw[4 * k2 + 1], hw[4 * k2 + 2], hw[4 * k2 + 3]);
          *reinterpret_cast<uint4 *>(aL + off) = make_uint4(lw[4 * k2], lw[4 * k2 + 1], lw[4 * k2 + 2], lw[4 * k2 + 3]);
        }
        // with 4 or more stages chunks are handed over in pairs: one proxy
        // fence (it waits for the shared-memory writes to reach the tensor
        // cores' view, about 5 % of the kernel when issued per chunk) covers
        // both, then both stages arrive.  The stage the second chunk waits for
        // was released by a chunk at least two back, already handed over, so
        // this cannot stall; with 3 stages (p = 7) pairs starve the MMAs.
        if (!C::PAIRS || (c & 1) || c == C::NCH - 1) {
          ptx::fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            if (C::PAIRS && (c & 1)) ptx::mbar_arrive(&bar_full[(g - 1) % C::STAGES]);
            ptx::mbar_arrive(&bar_full[s]);
          }
        }
        return true;
      };
      for (int c0 = 0; c0 < C::NCH && ok; c0 += C::PD) {
#pragma unroll
        for (int u = 0; u < C::PD; u++) {
          const int c = c0 + u;
          if (ok && c < C::NCH) {
            if (c + C::PD - 1 < C::NCH) load_phi(c + C::PD - 1, fr[(u + C::PD - 1) % C::PD]);
            ok = build(c, fr[u]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&bar_gempty[b]);  // done with the tile's point records
      if (!ok) break;
    }
  } else {
    // ---------------- geometry (warps 2..5 and 14..15) and epilogue (warps 2..5) ----------------
    // Iteration tt computes the point records of the elements that tile tt
    // brings in (ring slots), then warps 2..5 drain the accumulator of tile
    // tt - 1.  All 192 threads run every iteration and every named barrier
    // (work is skipped after an abort), so none can be left waiting on barrier 2.
    const bool epi = warp < kProdWarp0;
    const int gt = epi ? tid - kEpiWarp0 * 32 : 128 + tid - C::GEOW0 * 32;
    int64_t e_done = -1;  // last element whose records are in the ring
    uint32_t tt = 0;
    auto gbar = [] { asm volatile("bar.sync 2, 192;" ::: "memory"); };
    // coordinates and coefficients of a pass's new elements, copied
    // asynchronously (cp.async) into buffer (pass & 1) one pass ahead, so the
    // loads from memory overlap the previous pass and its drain
    auto fetch = [&](int64_t e_new, int nnew, double *dst) {
      for (int idx = gt; idx < nnew * C::NREC; idx += kNGeo) {
        const int el = idx / C::NREC, k = idx % C::NREC;
        const int64_t e = e_new + el;
        const int64_t eg = a.perm ? a.perm[e] : e;  // element of the mesh
        if (fem_chk(!a.perm || a.nmesh < 0 || (eg >= 0 && eg < a.nmesh), a.err))  // checked builds
          ptx::cp_async8(dst + idx, k < 18 ? a.coords + eg * 18 + k : a.coeffs + (k - 18) * a.cstride + eg);
        else
          dst[idx] = 0.0;
      }
      ptx::cp_async_commit();
    };
    // the new elements of tile t (elements above e_done)
    auto new_elems = [&](int64_t t, int64_t &e_new, int &nnew) {
      int64_t e_first;
      int nel;
      tile_elems(t, e_first, nel);
      e_new = e_first > e_done + 1 ? e_first : e_done + 1;
      nnew = (int)(e_first + nel - 1 - e_new + 1);
    };
    if (C::GEO_FINE && t_begin < t_end) {
      int64_t e0;
      int n0;
      new_elems(t_begin, e0, n0);
      fetch(e0, n0, sX);
    }
    for (int64_t t = t_begin; t <= t_end; t++, tt++) {
      if (t < t_end) {
        const int b = tt & 1;
        const uint32_t use = tt >> 1;
        int64_t e_first;
        int nel;
        tile_elems(t, e_first, nel);
        const int64_t R0 = t * C::BM;
        const int64_t e_last = e_first + nel - 1;
        const int64_t e_new = e_first > e_done + 1 ? e_first : e_done + 1;
        const int nnew = (int)(e_last - e_new + 1);  // 0 .. MAXEL
        e_done = e_last;
        double *sXp = sX + (size_t)(tt & 1) * C::MAXEL * C::NREC;  // this pass's inputs
        // tile tt - 2 is finished by the producers and the epilogue: its
        // elements that tiles tt - 1 and tt do not share may be overwritten
        if (gt == 0) wait(&bar_gempty[b], (use & 1) ^ 1);
        ptx::cp_async_wait_all();  // this thread's copies of the pass's inputs have landed
        gbar();
        const bool go = !*sAbort;
        if (go) {
          if (!C::GEO_FINE)  // the pass's inputs, loaded here
            for (int idx = gt; idx < nnew * C::NREC; idx += kNGeo) {
              const int el = idx / C::NREC, k = idx % C::NREC;
              const int64_t e = e_new + el;
              const int64_t eg = a.perm ? a.perm[e] : e;  // element of the mesh
              if (fem_chk(!a.perm || a.nmesh < 0 || (eg >= 0 && eg < a.nmesh), a.err))  // checked builds
                sXp[idx] = k < 18 ? a.coords[eg * 18 + k] : a.coeffs[(k - 18) * a.cstride + eg];
              else
                sXp[idx] = 0.0;
            }
          if (LAW != 0)
            for (int idx = gt; idx < nnew * C::NS; idx += kNGeo) {
              const int64_t e = e_new + idx / C::NS;
              sUC[idx] = a.ucoef[(a.perm ? a.perm[e] : e) * C::NS + idx % C::NS];
            }
          if (gt < nnew) {
            const int sl = (int)((e_new + gt) % C::RING);
            sSt[sl] = 0;
            sBnd[sl] = 0u;
            sBndB[sl] = 0u;
          }
        }
        gbar();
        if (go) {
          // one value per thread: the non-finite check of each input, the
          // element's edge record (21 differences of vertex coordinates, as
          // edge_record forms them) and its FP32 coefficients (a chain of FP64
          // operations on one thread per element was the slowest step here)
          for (int idx = gt; idx < nnew * C::NREC; idx += kNGeo) {
            const int el = idx / C::NREC, k = idx % C::NREC;
            const double *xe = sXp + el * C::NREC;
            const double v = xe[k];
            if (!isfinite(v)) atomicOr(&sSt[(e_new + el) % C::RING], FEM_ST_NONFINITE);
            if (k < kEdgeRec) {
              // value k = 3 m + i of vertex pair m: (1,0) (4,3) (2,0) (5,3) (3,0) (4,1) (5,2)
              constexpr unsigned kVa = 1u | 4u << 4 | 2u << 8 | 5u << 12 | 3u << 16 | 4u << 20 | 5u << 24;
              constexpr unsigned kVb = 0u | 3u << 4 | 0u << 8 | 3u << 12 | 0u << 16 | 1u << 20 | 2u << 24;
              const int m = k / 3, i = k % 3;
              const int va = (kVa >> (4 * m)) & 15, vb = (kVb >> (4 * m)) & 15;
              sEd[el * kEdgeRec + k] = xe[3 * va + i] - xe[3 * vb + i];
            }
            if (!ELAS && k >= 18) {
              const int kc = k - 18;  // D00 D11 D22 D01 D02 D12 b0 b1 b2 c f
              sCF[el * 12 + kc] = (float)v;
              if (kc >= 6 && kc <= 8 && a.layout == FEM_OUT_SYMPACKED && v != 0.0)
                atomicOr(&sSt[(e_new + el) % C::RING], FEM_ST_NONSYM);
            }
          }
          if (ELAS && gt < nnew) {  // E, nu, f -> lambda, mu, f of the element's slot
            const double *cf = sXp + gt * C::NREC + 18;
            const double Ey = cf[0], nu = cf[1];
            float *ec = sEC + ((e_new + gt) % C::RING) * 8;
            ec[0] = (float)(Ey * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)));
            ec[1] = (float)(Ey / (2.0 * (1.0 + nu)));
            ec[2] = (float)cf[2];
            ec[3] = (float)cf[3];
            ec[4] = (float)cf[4];
          }
        }
        gbar();
        if constexpr (C::GEO_FINE) {
          if (go) {  // tensor-product factors of J, one value per thread
            // J[:,0] and J[:,1] of each zeta level (6 values), J[:,2] of each
            // triangle point (3 values), as prism_zf / prism_xf form them
            constexpr int NZV = 6 * C::NZ, NXV = 3 * C::NAB;
            for (int idx = gt; idx < nnew * (NZV + NXV); idx += kNGeo) {
              const int el = idx / (NZV + NXV), r = idx % (NZV + NXV);
              const double *ed = sEd + el * kEdgeRec;
              if (r < NZV) {
                const int iz = r / 6, j = r % 6, o = j < 3 ? j : j + 3;  // edges (0, 3) or (6, 9)
                sZF[(el * C::NZ + iz) * kZf + j] = fma(sQF[2 * iz], ed[o], sQF[2 * iz + 1] * ed[o + 3]);
              } else {
                const int iab = (r - NZV) / 3, i = (r - NZV) % 3;
                const double *h = sQF + 2 * C::NZ + 3 * iab;
                sXF[(el * C::NAB + iab) * kXf + i] = fma(h[0], ed[12 + i], fma(h[1], ed[15 + i], h[2] * ed[18 + i]));
              }
            }
          }
          gbar();
          if (go) {  // adj row 2 of each level: J[:,0] x J[:,1] (FP64, and its FP32 copy)
            for (int idx = gt; idx < nnew * C::NZ * 3; idx += kNGeo) {
              const int el = idx / (3 * C::NZ), iz = (idx / 3) % C::NZ, j = idx % 3;
              const int j1 = j == 2 ? 0 : j + 1, j2 = j == 0 ? 2 : j - 1;  // (j + 1) mod 3, (j + 2) mod 3
              double *zf = sZF + (el * C::NZ + iz) * kZf;
              const double v = zf[j1] * zf[3 + j2] - zf[j2] * zf[3 + j1];
              zf[6 + j] = v;
              sZR[(el * C::NZ + iz) * 4 + j] = (float)v;
            }
          }
        } else {
          if (go) {  // tensor-product factors of J, one zeta level or triangle point per thread
            for (int idx = gt; idx < nnew * (C::NZ + C::NAB); idx += kNGeo) {
              const int el = idx / (C::NZ + C::NAB), r = idx % (C::NZ + C::NAB);
              const double *ed = sEd + el * kEdgeRec;
              if (r < C::NZ) {
                double *zf = sZF + (el * C::NZ + r) * kZf;
                prism_zf_lh(ed, sQF[2 * r], sQF[2 * r + 1], zf);
                float *zr = sZR + (el * C::NZ + r) * 4;
                zr[0] = (float)zf[6];
                zr[1] = (float)zf[7];
                zr[2] = (float)zf[8];
              } else {
                const double *h = sQF + 2 * C::NZ + 3 * (r - C::NZ);
                prism_xf_h(ed, h[0], h[1], h[2], sXF + (el * C::NAB + r - C::NZ) * kXf);
              }
            }
          }
        }
        gbar();
        if (go) {
          // points spread evenly over the four SM sub-partitions (their FP64
          // units bound this loop): warps 4 and 5 are alone on theirs and
          // take two slots of 32 points per round of 256, warps 2, 3 and the
          // last two share the other two sub-partitions and take one each
          // (p <= 4; above, one point per thread in order)
          const int wl = gt >> 5;
          const int nslot = !C::GEO_FINE ? 1 : (wl == 2 || wl == 3) ? 2 : 1;
          const int step = C::GEO_FINE ? 256 : kNGeo;
          for (int base = 0; base < nnew * C::NQP; base += step)
          for (int sv = 0; sv < nslot; sv++) {
            const int idx = C::GEO_FINE ? base + (sv ? wl + 4 : wl) * 32 + (gt & 31) : base + gt;
            if (idx >= nnew * C::NQP) continue;
            const int el = idx / C::NQP, q = idx % C::NQP;
            const int sl = (int)((e_new + el) % C::RING);
            float *gr = sG + (size_t)sl * C::GSLOT + q * 12;
            if (q < C::NQ) {
              float gv[11];
              const int iz = q / C::NAB, iab = q % C::NAB;
              double det;
              if (ELAS) {  // adj J (row-major), w / det J, w det J
                float a32[3][3];
                det = adj_tp_f32(sZF + (el * C::NZ + iz) * kZf, sZR + (el * C::NZ + iz) * 4,
                                 sXF + (el * C::NAB + iab) * kXf, a32);
#pragma unroll
                for (int k = 0; k < 9; k++) gv[k] = a32[k / 3][k % 3];
                const float detf = (float)det;
                gv[9] = sW[q] / detf;
                gv[10] = sW[q] * detf;
              } else if (LAW != 0) {
                // coefficient stage: u, grad u in FP32 from the field coefficients
                float a32[3][3];
                det = adj_tp_f32(sZF + (el * C::NZ + iz) * kZf, sZR + (el * C::NZ + iz) * 4,
                                 sXF + (el * C::NAB + iab) * kXf, a32);
                const float *U = sUC + el * C::NS;
                float u = 0.f, r0 = 0.f, r1 = 0.f, r2 = 0.f;
                for (int k = 0; k < C::NS; k++) {
                  const float4 f = __ldg(reinterpret_cast<const float4 *>(a.phiT) + (size_t)k * C::NQ + q);
                  u = fmaf(U[k], f.x, u);
                  r0 = fmaf(U[k], f.y, r0);
                  r1 = fmaf(U[k], f.z, r1);
                  r2 = fmaf(U[k], f.w, r2);
                }
                const float detf = (float)det, idet = 1.f / detf;
                const float gx = (a32[0][0] * r0 + a32[1][0] * r1 + a32[2][0] * r2) * idet;
                const float gy = (a32[0][1] * r0 + a32[1][1] * r1 + a32[2][1] * r2) * idet;
                const float gz = (a32[0][2] * r0 + a32[1][2] * r1 + a32[2][2] * r2) * idet;
                const float gg = gx * gx + gy * gy + gz * gz;
                float kq = 1.f;
                bool pend = false;
                if (LAW == 1) {
                  kq = law_exact<float>(u, gg, a.law_iters);
                } else {
                  const float sf = sqrtf(gg);
                  if (u >= a.box[0] && u <= a.box[1] && sf >= a.box[2] && sf <= a.box[3]) {
                    pend = true;  // k from the network after this phase
                    sXin[2 * idx] = fmaf(u, a.nrm[0], a.nrm[1]);
                    sXin[2 * idx + 1] = fmaf(logf(sf), a.nrm[2], a.nrm[3]);
                  } else {
                    kq = law_exact<float>(u, gg, a.law_iters);
                    atomicOr(&sSt[sl], FEM_ST_FALLBACK);
                  }
                }
                const float *cf = sCF + el * 12;
                const float cfl[11] = {kq, kq, kq, 0.f, 0.f, 0.f, cf[6], cf[7], cf[8], cf[9], cf[10]};
                record_f32(a32, detf, sW[q], cfl, gv);
                gr[11] = pend ? 1.f : 0.f;
              } else {
                det = point_tc(sZF + (el * C::NZ + iz) * kZf, sZR + (el * C::NZ + iz) * 4,
                               sXF + (el * C::NAB + iab) * kXf, sW[q], sCF + el * 12, gv);
              }
#pragma unroll
              for (int k = 0; k < 11; k++) gr[k] = gv[k];
              if (!(det > 0.0)) atomicOr(&sSt[sl], FEM_ST_DET);
              if (F16 && ELAS) {
                // |t_{1+a}| <= (w/det) (|lam| + 2 mu) |adj_a| sum_b |adj_b| max|Phi| over
                // every block (Cauchy-Schwarz on the three terms); the
                // load-vector row w det f_i by its own bound
                const float *ec = sEC + sl * 8;
                const float n0 = sqrtf(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]);
                const float n1 = sqrtf(gv[3] * gv[3] + gv[4] * gv[4] + gv[5] * gv[5]);
                const float n2 = sqrtf(gv[6] * gv[6] + gv[7] * gv[7] + gv[8] * gv[8]);
                const float bb = fabsf(gv[9]) * (fabsf(ec[0]) + 2.f * fabsf(ec[1])) * fmaxf(n0, fmaxf(n1, n2)) *
                                 (n0 + n1 + n2);
                if (isfinite(bb)) atomicMax(&sBnd[sl], __float_as_uint(bb));
                const float bs = fabsf(gv[10]) * fmaxf(fabsf(ec[2]), fmaxf(fabsf(ec[3]), fabsf(ec[4])));
                if (isfinite(bs)) atomicMax(&sBndB[sl], __float_as_uint(bs));
              } else if (F16) {
                float bb = fabsf(gv[G00]) + fabsf(gv[G01]) + fabsf(gv[G02]) + fabsf(gv[G03]);
                bb = fmaxf(bb, fabsf(gv[G11]) + fabsf(gv[G12]) + fabsf(gv[G13]));
                bb = fmaxf(bb, fabsf(gv[G12]) + fabsf(gv[G22]) + fabsf(gv[G23]));
                bb = fmaxf(bb, fabsf(gv[G13]) + fabsf(gv[G23]) + fabsf(gv[G33]));
                if (isfinite(bb)) atomicMax(&sBnd[sl], __float_as_uint(bb));
                // the load-vector row (S_Q, 0, 0, 0) gets its own scale: a small
                // source f must not fall into FP16 subnormals
                const float bs = fabsf(gv[GS]);
                if (isfinite(bs)) atomicMax(&sBndB[sl], __float_as_uint(bs));
              }
            } else {
#pragma unroll
              for (int k = 0; k < 11; k++) gr[k] = 0.f;
            }
          }
        }
        gbar();
        if (LAW == 2) {
          // network for the pending points of the pass (whole geometry warps)
          if (__all_sync(0xffffffffu, go)) {
            auto rec = [&](int pt) { return sG + (size_t)((e_new + pt / C::NQP) % C::RING) * C::GSLOT + (pt % C::NQP) * 12; };
            mlp_points_mma(
                sMP, sW2, sXin, nnew * C::NQP, [&](int pt) { return pt % C::NQP < C::NQ && rec(pt)[11] != 0.f; },
                [&](int pt, float k) {
                  float *r = rec(pt);
#pragma unroll
                  for (int m = G11; m <= G33; m++) r[m] *= k;
                },
                gt >> 5, kNGeo / 32, a.hw_tanh != 0);
          }
          gbar();
        }
        if (go && gt < nnew) {
          const int64_t e = e_new + gt;
          const int sl = (int)(e % C::RING);
          float sc = 1.f, inv = 1.f, scb = 1.f, invb = 1.f;
          if (F16) {
            auto pow2_scale = [&](float bnd, float &sv, float &is) {
              int ex = 0;
              if (bnd > 0.f) frexpf(bnd, &ex);  // bnd < 2^ex
              const int at = bnd > 0.f ? 14 - ex : 0;
              sv = ldexpf(1.f, at);
              is = ldexpf(1.f, -(at + a.aphi));
            };
            pow2_scale(__uint_as_float(sBnd[sl]) * a.phimax, sc, inv);
            pow2_scale(__uint_as_float(sBndB[sl]) * a.phimax, scb, invb);
          }
          sInv[sl] = inv;
          sInvB[sl] = invb;
          sScl[sl] = sc;
          sScB[sl] = scb;
          if (a.status && e * VPE * C::L >= R0) a.status[a.perm ? a.perm[e] : e] = sSt[sl];  // the tile holding row 0 reports
        }
        if (F16) {
          gbar();
          if (go) {  // fold the power-of-two scales into the point records
            for (int idx = gt; idx < nnew * C::NQP; idx += kNGeo) {
              const int sl = (int)((e_new + idx / C::NQP) % C::RING);
              float *gr = sG + (size_t)sl * C::GSLOT + (idx % C::NQP) * 12;
              const float sc = sScl[sl];
              if (ELAS) {  // every t scales with w/det, the load-vector row with w det
                gr[9] *= sc;
                gr[10] *= sScB[sl];
              } else {
#pragma unroll
                for (int k = 0; k < 10; k++) gr[k] *= sc;
                gr[GS] *= sScB[sl];
              }
            }
          }
        }
        gbar();  // the pass is complete for the whole group before the drain reads it
        if (gt == 0) ptx::mbar_arrive(&bar_gfull[b]);  // arrives even after an abort
        if (C::GEO_FINE && t + 1 < t_end && !*sAbort) {  // the next pass's inputs, into the other buffer
          int64_t en;
          int nn;
          new_elems(t + 1, en, nn);
          fetch(en, nn, sX + (size_t)((tt + 1) & 1) * C::MAXEL * C::NREC);
        }
      }
      if (epi && t > t_begin) {
        // ---------------- epilogue of tile t - 1: TMEM -> columns of A_e / b_e ----------------
        const uint32_t tp = tt - 1;
        const int64_t tq = t - 1;
        const uint32_t ab = C::NACC == 2 ? (tp & 1) : 0, use = tp / C::NACC;
        const bool ok = wait(&bar_accf[ab], use & 1);
        __syncwarp();
        if (__all_sync(0xffffffffu, ok)) {  // tcgen05.ld is collective over the warp
          ptx::tc_fence_after();
          const int lq = warp & 3;
          const int rl = 32 * lq + lane;
          const int64_t r = tq * C::BM + rl;
          const bool valid = r < nrows;
          const int64_t ve = valid ? r / C::L : 0;  // virtual element (the element for the scalar form)
          const int64_t e = ve / VPE;
          const int64_t eg = a.perm && valid ? a.perm[e] : e;  // element of the mesh
          // checked builds: an element id outside the mesh skips the row's stores
          const bool egok = !valid || fem_chk(!a.perm || a.nmesh < 0 || (eg >= 0 && eg < a.nmesh), a.err);
          const int j = valid ? (int)(r % C::L) : 0;
          const int sl = (int)(e % C::RING);
          const float inv = valid ? (j < C::NS ? sInv[sl] : sInvB[sl]) : 0.f;
          const uint32_t tbase = tmem + ab * C::KACC * C::NP + ((uint32_t)(32 * lq) << 16);
          constexpr int NPK = C::NS * (C::NS + 1) / 2;
          // columns c0 .. c0 + 15 of the accumulator row (v[0..15]) -> A_e / b_e
          auto store16 = [&](int c0, const uint32_t (&v)[16]) {
            if (valid && egok) {
              if (j < C::NS) {
                const int64_t oA = a.offA ? a.offA[eg] : (a.layout == FEM_OUT_FULL ? ve * (int64_t)(C::NS * C::NS)
                                                                               : e * (int64_t)NPK);
                const int64_t mA = a.layout == FEM_OUT_FULL ? (int64_t)C::NS * C::NS : NPK;
                if (!fem_chk(a.limA < 0 || (oA >= 0 && oA + mA <= a.limA), a.err)) {
                  // checked builds: the element's block lies outside A; skipped
                } else if (a.layout == FEM_OUT_FULL) {
                  // elasticity: block-major A^e[i][k][s][r] = block ve's [s][r]
                  float *Ae = static_cast<float *>(a.A) + oA + j;
#pragma unroll
                  for (int u = 0; u < 16; u++) {
                    const int i = c0 + u;
                    if (i < C::NS) Ae[(size_t)i * C::NS] = __uint_as_float(v[u]) * inv;
                  }
                } else {
                  float *Ae = static_cast<float *>(a.A) + oA;
#pragma unroll
                  for (int u = 0; u < 16; u++) {
                    const int i = c0 + u;
                    if (i < C::NS && i <= j) Ae[i * C::NS - i * (i - 1) / 2 + j - i] = __uint_as_float(v[u]) * inv;
                  }
                }
              } else if (a.b != nullptr && (!ELAS || ve % 3 == 0)) {
                // elasticity: the blocks (i, 0) carry b^e[i] (index 3 e + i = ve / 3)
                const int64_t ob = a.offb ? a.offb[eg] : (ELAS ? ve / 3 : e) * (int64_t)C::NS;
                if (fem_chk(a.limb < 0 || (ob >= 0 && ob + C::NS <= a.limb), a.err)) {
                  float *be = static_cast<float *>(a.b) + ob;
#pragma unroll
                  for (int u = 0; u < 16; u++) {
                    const int i = c0 + u;
                    if (i < C::NS) be[i] = __uint_as_float(v[u]) * inv;
                  }
                }
              }
            }
          };
          if constexpr (C::KACC == 2) {
            // the two accumulators' columns c0 .. c0 + 15, summed in FP32
#pragma unroll 1
            for (int c0 = 0; c0 < C::NP; c0 += 16) {
              uint32_t v0[16], v1[16];
              ptx::tmem_ld16(tbase + c0, v0);
              ptx::tmem_ld16(tbase + C::NP + c0, v1);
              ptx::tmem_ld_wait();
#pragma unroll
              for (int u = 0; u < 16; u++) v0[u] = __float_as_uint(__uint_as_float(v0[u]) + __uint_as_float(v1[u]));
              store16(c0, v0);
            }
          } else {
            // two 16-column loads in flight per wait
#pragma unroll 1
            for (int c0 = 0; c0 < C::NP; c0 += 32) {
              uint32_t v0[16], v1[16];
              const bool two = c0 + 16 < C::NP;  // warp-uniform
              ptx::tmem_ld16(tbase + c0, v0);
              if (two) ptx::tmem_ld16(tbase + c0 + 16, v1);
              ptx::tmem_ld_wait();
              store16(c0, v0);
              if (two) store16(c0 + 16, v1);
            }
          }
          ptx::tc_fence_before();
          __syncwarp();
          if (lane == 0) {
            ptx::mbar_arrive(&bar_acce[ab]);
            ptx::mbar_arrive(&bar_gempty[tp & 1]);
          }
        }
      }
    }
  }

  ptx::cp_async_wait_all();  // no copy into shared memory outlives the CTA
  __syncthreads();
  if (*sAbort) {
    if (tid == 0 && a.err) atomicOr(a.err, kErrTimeout);
    // flag the elements of this CTA's tiles that may be incomplete
    if (a.status) {
      for (int64_t t = t_begin; t < t_end; t++) {
        const int64_t e0 = (t * C::BM) / C::L / VPE;
        int64_t e1 = (t * C::BM + C::BM - 1) / C::L / VPE;
        if (e1 > a.n - 1) e1 = a.n - 1;
        for (int64_t e = e0 + tid; e <= e1; e += blockDim.x) atomicOr(&a.status[a.perm ? a.perm[e] : e], FEM_ST_TIMEOUT);
      }
    }
  }
  if (warp == 1) {
    __syncwarp();
    ptx::tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// ---------------------------------------------------------------- host side

template <int P, bool F16, bool ELAS, int LAW = 0, int RULE = FEM_RULE_COLLAPSED>
static int launch_tc_p(const TcArgs &a, void *stream) {
  using C = TcCfg<P, ELAS, LAW, RULE>;
  if (a.n == 0) return FEM_OK;
  cudaError_t err = cudaFuncSetAttribute(tc_kernel<P, F16, ELAS, LAW, RULE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (err != cudaSuccess) {
    set_error(std::string("cudaFuncSetAttribute(tc_kernel): ") + cudaGetErrorString(err));
    return FEM_ECUDA;
  }
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // one 512-thread CTA per SM (it overlaps its own phases); TMEM_COLS <= 512
  const int64_t ntiles = (a.n * (ELAS ? 9 : 1) * C::L + C::BM - 1) / C::BM;
  int64_t grid = nsm;
  if (grid > ntiles) grid = ntiles;
  tc_kernel<P, F16, ELAS, LAW, RULE><<<(unsigned)grid, C::THREADS, C::SMEM, (cudaStream_t)stream>>>(a);
  err = cudaGetLastError();
  if (err != cudaSuccess) {
    set_error(std::string("tc_kernel launch: ") + cudaGetErrorString(err));
    return FEM_ECUDA;
  }
  return FEM_OK;
}

template <bool F16, bool ELAS, int LAW = 0, int RULE = FEM_RULE_COLLAPSED>
static int launch_tc_any(int p, const TcArgs &a, void *stream) {
  switch (p) {
    case 1: return launch_tc_p<1, F16, ELAS, LAW, RULE>(a, stream);
    case 2: return launch_tc_p<2, F16, ELAS, LAW, RULE>(a, stream);
    case 3: return launch_tc_p<3, F16, ELAS, LAW, RULE>(a, stream);
    case 4: return launch_tc_p<4, F16, ELAS, LAW, RULE>(a, stream);
    case 5: return launch_tc_p<5, F16, ELAS, LAW, RULE>(a, stream);
    case 6: return launch_tc_p<6, F16, ELAS, LAW, RULE>(a, stream);
    case 7: return launch_tc_p<7, F16, ELAS, LAW, RULE>(a, stream);
  }
  return FEM_EINVAL;
}

// Per-TU instantiations (fem_tc_*.cu), dispatched by launch_tc (fem_tc.cu).
int launch_tc_scalar_bf16(int p, const TcArgs &a, void *stream);
int launch_tc_scalar_f16(int p, const TcArgs &a, void *stream);
int launch_tc_scalar_t1(int p, bool f16, const TcArgs &a, void *stream);
int launch_tc_elastic(int p, bool f16, const TcArgs &a, void *stream);
int launch_tc_elastic_t1(int p, bool f16, const TcArgs &a, void *stream);
int launch_tc_law(int p, int law, const TcArgs &a, void *stream);

}  // namespace fem
