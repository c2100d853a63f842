/*
 * fem.h -- C ABI of the GB300 per-element numerical integration library.
 *
 * The operation (Section 2 of Banas, Plaszewski, Maciol, arXiv 1310.1191,
 * Algorithms 1 and 2): given the geometry of each element, problem dependent
 * coefficients and (for nonlinear problems) old degrees of freedom, create the
 * element stiffness matrix
 *     A^e[i][j] = sum_Q det J_Q w_Q sum_{iD,jD} c^Q[iD][jD] psi^Q[iD][i] psi^Q[jD][j]
 * where psi^Q are the shape functions (iD = 0) and their physical derivatives
 * (iD = 1..3) at quadrature point Q (eq. sum_int, Section 5.1).  The weak form
 * is the generic scalar second-order one,
 *     a(u, v) = int grad v . D grad u + v b . grad u + c u v,   l(v) = int f v,
 * so c[0][0] = c, c[0][1+m] = b_m, c[1+l][1+m] = D[l][m], c[1+l][0] = 0.
 * Row i of A^e is the test function, column j the trial function.  The load
 * vector b^e[i] = sum_Q det J_Q w_Q f psi^Q[0][i] is produced beside A^e.
 *
 * Elements: P1 tetrahedra (4 nodes, 4-point degree-2 rule) and straight-edged
 * 6-node prisms of degree p = 1..7 (Dubiner triangle x Legendre basis,
 * NS = (p+1)^2 (p+2)/2 shape functions), integrated with a rule exact to
 * degree 2p: by default the collapsed Gauss-Jacobi x Gauss-Legendre rule with
 * NQ = (p+1)^3 points, or the paper's counts (Table 1, NQ = 6 ... 336) with
 * fem_tables_build_ex(..., FEM_RULE_TABLE1, ...).
 *
 * Conventions for every entry point:
 *   - all functions return a status code (FEM_OK = 0) and never abort;
 *   - argument errors are detected on the host before anything is enqueued;
 *   - device pointers are caller-owned; the library owns only table handles
 *     and the objects it creates (plans, surrogates);
 *   - compute entry points are asynchronous on the given CUDA stream
 *     (cudaStream_t passed as void*, NULL = legacy default stream).
 */
#ifndef FEM_GB300_H
#define FEM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define FEM_OK 0
#define FEM_EINVAL 1        /* bad argument (null, size, alignment, range) */
#define FEM_ENOMEM 2        /* library-owned allocation failed */
#define FEM_ECUDA 3         /* a CUDA runtime call failed (see fem_last_error) */
#define FEM_EUNSUPPORTED 4  /* valid but not provided combination */
#define FEM_EELEMENT 5      /* at least one element flagged in status[] */
#define FEM_ETIMEOUT 6      /* a bounded device wait gave up */
#define FEM_ECHECKED 7      /* checked build: a kernel's index check failed (access skipped) */

/* ---- element types ---- */
#define FEM_TET4 0
#define FEM_PRISM6 1

/* ---- arithmetic of the contraction (geometry is always FP64) ---- */
#define FEM_F64 0     /* FP64 FMA; outputs double */
#define FEM_F32 1     /* FP32 FMA, G rounded from FP64; outputs float */
#define FEM_BF16X3 2  /* tensor cores, bf16 hi+lo split, FP32 accumulate; float */
#define FEM_F16X3 3   /* tensor cores, fp16 hi+lo split, FP32 accumulate; float */

/* ---- quadrature rules of the prism (tetrahedra: the 4-point degree-2 rule) ---- */
#define FEM_RULE_COLLAPSED 0  /* (p+1)^3 points: Gauss-Legendre x Gauss-Jacobi(1,0) x Gauss-Legendre */
#define FEM_RULE_TABLE1 1     /* the paper's point counts (Table 1, N_Q = 6, 18, 48, 80, 150, 231, 336):
                                 a fully symmetric degree-2p triangle rule x (p+1) Gauss-Legendre points */

/* ---- output layouts ---- */
#define FEM_OUT_FULL 0       /* A [E][NS][NS] row-major, unpadded */
#define FEM_OUT_SYMPACKED 1  /* upper triangle row by row, NS(NS+1)/2 per element */

/* ---- per-element status bits (int32 status[e]) ---- */
#define FEM_ST_DET 1        /* det J <= 0 at some quadrature point */
#define FEM_ST_NONFINITE 2  /* non-finite coordinate or coefficient */
#define FEM_ST_NONSYM 4     /* symmetric-packed output requested but b != 0 */
#define FEM_ST_FALLBACK 8   /* surrogate input left its box: exact law used (info) */
#define FEM_ST_TIMEOUT 16   /* a bounded device wait expired: this element's output is invalid */

typedef struct fem_tables_s *fem_tables;

/* Reference data on the host, no GPU needed (Section 2: xi^Q, w^Q and
 * phi^Q[iQ][iD][iDOF] of one element type and degree).
 *   nq, ns  : out, number of points and shape functions (may be NULL);
 *   xi      : out [nq][3] reference coordinates, or NULL;
 *   w       : out [nq] weights (sum = reference volume: 1 prism, 1/6 tet), or NULL;
 *   phi     : out [nq][4][ns] values (row 0) and reference derivatives
 *             d/dxi, d/deta, d/dzeta (rows 1..3), or NULL.
 * Returns FEM_EINVAL for an unknown element or p outside 1..7 (tet: p = 1). */
int fem_reference_rule(int elem, int p, int *nq, int *ns, double *xi, double *w, double *phi);
/* The same for a chosen prism rule (FEM_RULE_COLLAPSED as fem_reference_rule,
 * or FEM_RULE_TABLE1, the paper's point counts of Table 1; its prism points
 * are ordered q = iz * NT + it, zeta level iz of the (p+1)-point Gauss-Legendre
 * rule, point it of the NT-point triangle rule).  FEM_EINVAL for a rule the
 * element does not have. */
int fem_reference_rule_ex(int elem, int rule, int p, int *nq, int *ns, double *xi, double *w, double *phi);

/* Build the device tables (quadrature points and weights, shape functions
 * and reference derivatives at all points, in FP64 and in the reduced
 * formats the contraction kernels read) for degrees p_min..p_max of one
 * element type, on the current CUDA device.  Synchronous.  "These values are
 * the same for all elements of a given approximation order" (Section 4.1):
 * they are built once and kept resident in HBM.
 *   out : receives a library-owned handle; release with fem_tables_destroy. */
int fem_tables_build(int elem, int p_min, int p_max, fem_tables *out);
/* fem_tables_build for a chosen prism quadrature rule.  Tables built with
 * FEM_RULE_TABLE1 serve fem_integrate / fem_integrate_uniform (uniform degree,
 * constant coefficients; every precision), fem_integrate_elastic (every
 * precision) and fem_integrate_host; the other compute entry points return
 * FEM_EUNSUPPORTED for them.  FEM_EINVAL for an
 * unknown rule or a rule the element does not have (tetrahedra). */
int fem_tables_build_ex(int elem, int rule, int p_min, int p_max, fem_tables *out);
int fem_tables_destroy(fem_tables t);

/* Coefficient law of fem_integrate: the diffusion coefficient at each
 * quadrature point computed from the previous solution's degrees of freedom
 * (Section 2: the coefficients may depend on the old solution; the law and
 * the network are described with fem_integrate_law below).
 *   law          : 0 constant coefficients (the rows of coeffs as given),
 *                  FEM_LAW_EXACT or FEM_LAW_MLP;
 *   ucoef        : device float [n_elem][NS], the field's coefficients per element;
 *   mlp          : the network for FEM_LAW_MLP, else NULL;
 *   newton_steps : Newton steps of the exact law (0: the law's 8; up to 1024
 *                  -- more steps leave k unchanged once converged and only
 *                  make the law costlier, to compare its cost with the
 *                  network's);
 *   hw_tanh      : non-zero: the network's activations from the hardware
 *                  approximation tanh.approx.f32 (one special-function
 *                  operation instead of two, larger error). */
typedef struct fem_mlp_s *fem_mlp;
typedef struct fem_coef_law_s {
  int law;
  const float *ucoef;
  fem_mlp mlp;
  int newton_steps;
  int hw_tanh;
} fem_coef_law;

/* Per-element integration (Section 2; Algorithms 3/4 of Section 4.1 and the
 * host's classification of elements by degree of Section 4.2, re-designed for
 * sm_103a): element matrices A_e and load vectors b_e of n_elem elements.
 *   t            : tables holding every degree used, of one element type;
 *   n_elem       : number of elements (0 is a no-op);
 *   coords       : device, double [n_elem][nv][3], nv = 4 (tet) or 6 (prism),
 *                  8-byte aligned; vertex order as in the reference element;
 *   p_per_elem   : HOST int8 [n_elem] degree of each element, or NULL for a
 *                  mesh of the single degree p_uniform.  With per-element
 *                  degrees the elements are binned by degree on the host and
 *                  run by a mixed-degree plan (fem_plan_create with
 *                  FEM_PLAN_CONCURRENT) that the tables handle creates and
 *                  keeps for the next call with the same degrees, precision
 *                  and layout; the outputs are then the flat variable-size
 *                  arrays of fem_output_offsets (elements in their order);
 *   p_uniform    : the degree when p_per_elem is NULL (1..7; 1 for FEM_TET4);
 *   coeffs       : device, double SoA [11][coeff_stride]: Dxx Dyy Dzz Dxy Dxz
 *                  Dyz bx by bz c f, element e at column e; coeff_stride >= n_elem;
 *   law          : NULL (constant coefficients) or a coefficient law
 *                  (uniform degree only: per-element degrees with a law give
 *                  FEM_EUNSUPPORTED; see fem_integrate_law for the precisions);
 *   prec         : FEM_F64 / FEM_F32 / FEM_BF16X3 / FEM_F16X3;
 *   layout       : FEM_OUT_FULL or FEM_OUT_SYMPACKED;
 *   A_out        : device, [n_elem][NS*NS] (full) or [n_elem][NS(NS+1)/2]
 *                  (packed) of double (FEM_F64) or float (others), 16-byte aligned;
 *   b_out        : device, [n_elem][NS] of the same type, or NULL to skip;
 *   status       : device int32 [n_elem] of FEM_ST_* bits, or NULL;
 *   stream       : cudaStream_t.
 * Returns FEM_EINVAL for null/misaligned pointers, n_elem < 0, a degree
 * outside the tables, unknown prec/layout; FEM_EUNSUPPORTED for a
 * combination no kernel provides (tensor-core precisions on tetrahedra);
 * FEM_ECUDA if a launch fails.  Numerical problems of single elements
 * (det J <= 0, non-finite input, packed output of a non-symmetric form) never
 * fail the call: they are recorded in status[], and fem_sync_status turns
 * them into FEM_EELEMENT.  The first call with new per-element degrees
 * allocates the plan's device arrays and captures its graph; later calls
 * with the same degrees and buffers replay it. */
int fem_integrate(fem_tables t, int64_t n_elem, const double *coords, const int8_t *p_per_elem,
                  int p_uniform, const double *coeffs, int64_t coeff_stride, const fem_coef_law *law,
                  int prec, int layout, void *A_out, void *b_out, int32_t *status, void *stream);

/* The uniform-degree, constant-coefficient case of fem_integrate, as one
 * direct launch of the degree's kernel: fem_integrate(t, n_elem, coords,
 * NULL, p, coeffs, coeff_stride, NULL, ...) calls it.  Same arguments and
 * errors. */
int fem_integrate_uniform(fem_tables t, int p, int64_t n_elem, const double *coords, const double *coeffs,
                          int64_t coeff_stride, int prec, int layout, void *A_out, void *b_out,
                          int32_t *status, void *stream);

/* Synchronous status query over the per-element flags of a finished or
 * enqueued integration: waits for `stream`, reduces status[0..n_elem) on the
 * device, and returns
 *   FEM_ETIMEOUT  if a bounded device wait of these tables expired (the
 *                 device error word of fem_error_flag, left as it is);
 *   FEM_EELEMENT  if at least one element carries an error bit (FEM_ST_DET,
 *                 FEM_ST_NONFINITE, FEM_ST_NONSYM or FEM_ST_TIMEOUT);
 *   FEM_OK        otherwise (FEM_ST_FALLBACK is informational).
 *   status : device int32 [n_elem], 4-byte aligned (NULL with n_elem = 0);
 *   bits   : out, OR of every element's bits (nullable);
 *   nflag  : out, number of elements with an error bit (nullable).
 * FEM_EINVAL for bad arguments, FEM_ECUDA if a CUDA call fails. */
int fem_sync_status(fem_tables t, const int32_t *status, int64_t n_elem, int32_t *bits, int64_t *nflag,
                    void *stream);

/* Linear elastostatics, the paper's model problem (Section 5.1, eqs.
 * strong_form / fes / sum_int): N_E = 3 components, isotropic
 * c_ijkl = lam d_ij d_kl + mu (d_ik d_jl + d_il d_jk) from Young's modulus E and
 * Poisson's ratio nu (lam = E nu / ((1+nu)(1-2nu)), mu = E / (2(1+nu))),
 * constant per element, and a constant body force f:
 *   A^e[iE][jE][s][r] = sum_Q det J w sum_{j,l} c_{iE j jE l} psi_j^s psi_l^r,
 *   b^e[iE][s]        = sum_Q det J w f_iE psi_0^s.
 *   coeffs : device double SoA [5][coeff_stride]: E, nu, fx, fy, fz;
 *   A_out  : device [n_elem][3][3][NS][NS] (the paper's A^e[iE][jE][iDOF][jDOF]),
 *            double (FEM_F64) or float (the others), 16-byte aligned;
 *   b_out  : device [n_elem][3][NS] or NULL; status : device int32 [n_elem] or NULL.
 * Prisms; FEM_F64 / FEM_F32 (CUDA-core FMA kernels) or FEM_BF16X3 /
 * FEM_F16X3 (tensor cores: each 3x3 block of an element is a row block of
 * the tensor-core contraction, 16-bit hi + lo operands, FP32 accumulation;
 * the per-element error bound is the one of fem_integrate's tensor-core
 * forms). */
int fem_integrate_elastic(fem_tables t, int p, int64_t n_elem, const double *coords, const double *coeffs,
                          int64_t coeff_stride, int prec, void *A_out, void *b_out, int32_t *status,
                          void *stream);

/* Split geometry (the paper's NOJAC kernel variants, Section 4 "Jacobian
 * terms"; Algorithm 1's Jacobian step moved out of the integration kernel): for every
 * element and quadrature point, det J and the 9 entries of J^{-1}.
 *   coords : device, double [n_elem][NV][3] (as fem_integrate), 8-byte aligned;
 *   terms  : device, double [n_elem][NQ][10], 16-byte aligned, caller-owned:
 *            terms[e][q][0] = det J, terms[e][q][1 + 3k + m] = (J^{-1})[k][m]
 *            = d xi_k / d x_m, q in the rule's point order (fem_reference_rule);
 *   status : device int32 [n_elem] or NULL: FEM_ST_NONFINITE for a non-finite
 *            coordinate, FEM_ST_DET if det J <= 0 at some point.
 * The paper prepares these terms on the host; this pass computes them on the
 * device.  Errors as fem_integrate (FEM_EINVAL for NULL/misaligned pointers,
 * n_elem < 0, p outside the tables; FEM_ECUDA for a failed launch). */
int fem_jacobian_terms(fem_tables t, int p, int64_t n_elem, const double *coords, double *terms,
                       int32_t *status, void *stream);

/* Integration from stored Jacobian terms (NOJAC): the result of fem_integrate
 * for the elements whose terms fem_jacobian_terms (or any producer of the same
 * layout) wrote.  terms: device double [n_elem][NQ][10], 8-byte aligned; the
 * other arguments as fem_integrate.  adj J = det J * J^{-1} replaces the
 * geometry stage; non-finite terms set FEM_ST_NONFINITE, det J <= 0 sets
 * FEM_ST_DET.  prec FEM_F64 / FEM_F32 (tensor-core precisions
 * FEM_EUNSUPPORTED). */
int fem_integrate_terms(fem_tables t, int p, int64_t n_elem, const double *terms, const double *coeffs,
                        int64_t coeff_stride, int prec, int layout, void *A_out, void *b_out,
                        int32_t *status, void *stream);

/* Linear elastostatics (as fem_integrate_elastic) from stored Jacobian terms
 * (NOJAC, the variant the paper measures on its model problem, Section 5). */
int fem_integrate_elastic_terms(fem_tables t, int p, int64_t n_elem, const double *terms,
                                const double *coeffs, int64_t coeff_stride, int prec, void *A_out,
                                void *b_out, int32_t *status, void *stream);

/* The same integration for HOST buffers (the paper's host code stages element
 * data to the device, runs the kernel and copies the matrices back, Section
 * 4.2): the elements are processed in chunks of `chunk` elements (<= 0: about
 * 256 MB of staging per chunk) through two pipeline slots on two library
 * streams, so that the copies of one chunk overlap the kernel of the other.
 * Host buffers should be page-locked for the copies to overlap.  Layouts as in
 * fem_integrate but in host memory; b_out and status nullable.  Synchronous:
 * returns when every result is in host memory.  The staging buffers are owned
 * by the tables handle (allocated on first use, grown when needed). */
int fem_integrate_host(fem_tables t, int p, int64_t n_elem, const double *coords, const double *coeffs,
                       int64_t coeff_stride, int prec, int layout, void *A_out, void *b_out, int32_t *status,
                       int64_t chunk);

/* Matrix-free operator apply: y_e = A_e x_e for every element, with A_e the
 * matrix fem_integrate computes (FEM_OUT_FULL: row = test function), without
 * forming it.  This is the element-level product a Krylov solver of the
 * assembled system needs when the element operators stay in device memory
 * (Section 4), and the high-order alternative to forming A_e that Section 3
 * points to: per element y = sum_Q Phi_Q^T G_Q Phi_Q x, on prisms by sum
 * factorisation over the triangle x Legendre structure of the basis and the
 * rule (16 NQ NS flops per element at most instead of 8 NQ NS^2).
 *   t, p, n_elem, coords, coeffs, coeff_stride : as fem_integrate (f unused);
 *   prec   : FEM_F64 (x, y double) or FEM_F32 (x, y float; geometry and point
 *            stage FP64, contractions FP32); tensor-core precisions give
 *            FEM_EUNSUPPORTED;
 *   x      : device [n_elem][NS] of the precision's type, DOF order of the
 *            tables, aligned to its element size; read only;
 *   y      : device [n_elem][NS], same type and alignment, must not overlap x;
 *   status : device int32 [n_elem] or NULL: FEM_ST_NONFINITE for a non-finite
 *            coordinate or coefficient, FEM_ST_DET if det J <= 0 at some point
 *            (the flags of fem_integrate).
 * Errors as fem_integrate (FEM_EINVAL for NULL/misaligned pointers, n_elem < 0,
 * p outside the tables, coeff_stride < n_elem; FEM_ECUDA for a failed launch).
 * Stream-ordered; allocates nothing. */
int fem_apply(fem_tables t, int p, int64_t n_elem, const double *coords, const double *coeffs,
              int64_t coeff_stride, int prec, const void *x, void *y, int32_t *status, void *stream);

/* Device error word of the tables' kernels: FEM_ETIMEOUT if a bounded wait
 * inside a tensor-core launch expired since the last clear (the affected
 * elements also carry FEM_ST_TIMEOUT); in the checked build
 * (libfem_gb300_checked.so, compiled with FEM_CHECKED: the kernels check the
 * element ids of permutations and the output offsets of mixed-degree plans
 * against their extents and skip a failing access) FEM_ECHECKED if a check
 * failed; else FEM_OK.  Synchronises the device.
 *   clear : non-zero resets the word. */
int fem_error_flag(fem_tables t, int clear);

/* ---- nonlinear coefficient law and its learned surrogate ---- */
/* The law (coefficients at quadrature points computed from previous-solution degrees of
 * freedom, Algorithm 1's coefficient step):
 *     k = 1 + 0.5 exp(-u^2) + 0.2 log(1 + k |grad u|^2),  D = k I,
 * solved per point by exactly 8 Newton steps from k0 = 1 + 0.5 exp(-u^2).
 * The surrogate is a 2 -> 64 -> 64 -> 1 tanh network of (u, |grad u|) with
 * BF16 weights and FP32 accumulation, used inside its training box
 * [u0,u1] x [s0,s1] (u mapped linearly, log |grad u| linearly onto [-1,1]);
 * outside the box the exact law is used and the element gets FEM_ST_FALLBACK. */
#define FEM_LAW_EXACT 1
#define FEM_LAW_MLP 2

/* Integration with the per-point law.  Arguments as fem_integrate, plus
 *   ucoef : device float [n_elem][NS] coefficients of the scalar field u in
 *           the element's shape functions (the previous solution's degrees of freedom);
 *   law   : FEM_LAW_EXACT or FEM_LAW_MLP (then mlp must be a network);
 *   prec  : FEM_F64 or FEM_F32 (the law in that precision; the network in FP32),
 *           or FEM_BF16X3 for prisms (the tensor-core contraction, with the
 *           coefficient stage -- u, grad u, the law or the network -- in FP32
 *           on the geometry warps; float outputs, the tensor-core forms'
 *           error bound).
 * The coefficient rows Dxx..Dyz are ignored (D = k I); b, c, f are used. */
int fem_integrate_law(fem_tables t, int p, int64_t n_elem, const double *coords, const double *coeffs,
                      int64_t coeff_stride, const float *ucoef, int law, fem_mlp mlp, int prec, int layout,
                      void *A_out, void *b_out, int32_t *status, void *stream);

/* u and |grad u| at every quadrature point of n prisms of degree p:
 *   us : device float [n][NQ][2] out. */
int fem_field_samples(fem_tables t, int p, int64_t n, const double *coords, const float *ucoef, float *us,
                      void *stream);

/* Training box from samples on the host: box[4] = percentiles lo_pct / hi_pct
 * of u and of |grad u|; us_host float [n][2]. FEM_EINVAL if degenerate. */
int fem_box_from_samples(int64_t n, const float *us_host, double lo_pct, double hi_pct, double *box);

/* n training pairs drawn on the device: u uniform in [u0,u1], log |grad u|
 * uniform in [log s0, log s1] (counter-based SplitMix64 draws of (seed, i)),
 * target k from the exact law in FP64.  us: device float [n][2]; k: [n]. */
int fem_law_samples(int64_t n, const double *box, uint64_t seed, float *us, float *k, void *stream);

/* Network object: Glorot-uniform weights from seeded draws, zero biases. */
int fem_mlp_create(const double *box, uint64_t seed, fem_mlp *out);
int fem_mlp_destroy(fem_mlp m);
int fem_mlp_nparams(void);
/* y[i] = network(us[i][0], us[i][1]) on the device. */
int fem_mlp_forward(fem_mlp m, int64_t n, const float *us, float *y, void *stream);
/* Mean squared error over n samples and its gradient (hand-written backprop),
 * computed with the BF16 compute weights: grad device float [P], loss [1]. */
int fem_mlp_loss_grad(fem_mlp m, int64_t n, const float *us, const float *t, float *grad, float *loss,
                      void *stream);
/* steps Adam steps (beta 0.9 / 0.999, eps 1e-8) on minibatches of `batch`
 * samples drawn with replacement from the n pairs (seeded); the first call
 * sets the output bias to the mean target.  loss_host (nullable) receives the
 * per-step minibatch losses (the call then synchronises). */
int fem_mlp_train(fem_mlp m, int64_t n, const float *us, const float *t, int64_t steps, int batch, float lr,
                  uint64_t seed, float *loss_host, void *stream);
/* Host copies of the FP32 master and BF16-rounded compute parameters (each
 * nullable, [P]) and the box (nullable, [4]); set replaces the master. */
int fem_mlp_get(fem_mlp m, float *master_host, float *compute_host, double *box);
int fem_mlp_set(fem_mlp m, const float *master_host);
/* Checkpoint: "FEMMLP01", H, P, box, step, master, Adam m, Adam v. */
int fem_mlp_save(fem_mlp m, const char *path);
int fem_mlp_load(const char *path, fem_mlp *out);

/* ---- mixed-degree meshes (p-binned persistent launch) ---- */
typedef struct fem_plan_s *fem_plan;

#define FEM_PLAN_AUTOTUNE 1  /* time the candidate tile shapes on the first execution */
#define FEM_PLAN_LOOP 2      /* run one specialised launch per degree instead of one launch */
#define FEM_PLAN_NOGRAPH 4   /* launch directly instead of replaying a captured CUDA graph */
#define FEM_PLAN_CONCURRENT 8 /* one graph branch per degree (specialised kernels, overlapping) */

/* Per-element output offsets of a mixed-degree mesh, elements kept in their
 * original order with unpadded variable-size blocks:
 *   p_host : host int8 [n] degrees;
 *   offA   : out host [n] offset (in values) of A_e in A_out, or NULL;
 *   offb   : out host [n] offset of b_e in b_out, or NULL;
 *   totals : out [2] total values of A_out and b_out, or NULL.
 * FEM_EINVAL if a degree is invalid for elem. */
int fem_output_offsets(int elem, const int8_t *p_host, int64_t n, int layout, int64_t *offA,
                       int64_t *offb, int64_t *totals);

/* Plan for a mixed-degree prism mesh (Section 4.2: the host classifies the
 * elements by degree).  The elements are binned by degree on the host, the
 * bins cut into work items (element group x output tile) ordered by cost, and
 * executed by one persistent launch whose CTAs pull items from an atomic
 * counter; the counter reset and the launch are captured in a CUDA graph on
 * the first execution and replayed afterwards (re-captured when the buffers
 * change).  With FEM_PLAN_AUTOTUNE the first execution times the candidate
 * tile shapes of each degree on the plan's own elements and keeps the fastest;
 * with FEM_PLAN_CONCURRENT the graph instead holds one branch per degree, each
 * running that degree's specialised kernel on its own stream, overlapping;
 * tune_cache (nullable) is a text file that stores and reuses the choices.
 *   t      : prism tables covering every degree in p_host;
 *   p_host : host int8 [n_elem] degrees (copied; not kept);
 *   prec   : FEM_F64 or FEM_F32; or FEM_BF16X3 / FEM_F16X3 with
 *            FEM_PLAN_LOOP or FEM_PLAN_CONCURRENT (each degree then runs the
 *            tensor-core kernel or an FP32 kernel, see fem_plan_variant;
 *            float outputs); others FEM_EUNSUPPORTED;
 *   layout : FEM_OUT_FULL / FEM_OUT_SYMPACKED.
 * The plan owns device memory for the permutation, the offsets, the work
 * list and the counter; release it with fem_plan_destroy. */
int fem_plan_create(fem_tables t, int64_t n_elem, const int8_t *p_host, int prec, int layout, int flags,
                    const char *tune_cache, fem_plan *out);

/* Execute a plan: buffers as in fem_integrate, except that A_out and b_out
 * are the flat variable-size arrays described by fem_output_offsets
 * (elements in their original order).  Asynchronous on stream, except the
 * first execution of an autotuning plan, which synchronises while timing.
 * Executions of one plan must not overlap on the device (they share the
 * work counter). */
int fem_plan_execute(fem_plan plan, const double *coords, const double *coeffs, int64_t coeff_stride,
                     void *A_out, void *b_out, int32_t *status, void *stream);

/* Kernel variant chosen for degree p, and the autotuner's times of the
 * candidates in ms (ms[4], nullable; 0 if not timed); -1 if invalid.
 * Variants 0 and 1 are the persistent kernel's candidate shapes; plans with
 * FEM_PLAN_LOOP or FEM_PLAN_CONCURRENT also have variant 2, the degree's
 * uniform-degree kernel (as fem_integrate runs it), their default without
 * FEM_PLAN_AUTOTUNE; plans with a tensor-core precision also variant 3, the
 * tensor-core kernel, their default for p >= 3 (variants 0-2 then run in
 * FP32).  Per-degree plans are tuned by timing each candidate as one launch
 * over the degree's bin. */
int fem_plan_variant(fem_plan plan, int p, double *ms);
int fem_plan_destroy(fem_plan plan);

/* Mixed-degree integration that allocates no device memory (the paper has no
 * counterpart; this is a library convenience).  For callers that cannot call
 * cudaMalloc -- code running inside a fixed memory pool or budget, or on a
 * path where an allocation's implicit device synchronisation is not allowed.
 * It runs the same persistent p-binned kernel as fem_plan_execute (default
 * tile shapes, no graph), with its scratch -- work counter, work list, degree
 * permutation and output offsets -- in one fixed static device array of the
 * library (about 1.4 MB, held on every GPU that loads the library until the
 * process exits) instead of plan allocations.
 *   Arguments as fem_plan_create + fem_plan_execute: p_host is a host int8
 *   [n_elem] degree array; A_out / b_out are the flat variable-size arrays
 *   described by fem_output_offsets; prec FEM_F64 or FEM_F32.
 * Limits: n_elem <= 16384 and at most 65536 work items; larger calls return
 * FEM_EINVAL with a message (use a plan instead).
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call reuses the same array and leaves its contents there:
 * the call zeroes the work counter itself, but calls whose executions overlap
 * on the GPU (other streams, other host threads) race on the array and must
 * be serialised by the caller.  The host-side preparation is serialised by a
 * mutex.  Asynchronous on stream once the small work list is staged. */
int fem_integrate_mixed_noalloc(fem_tables t, int64_t n_elem, const int8_t *p_host, const double *coords,
                                const double *coeffs, int64_t coeff_stride, int prec, int layout,
                                void *A_out, void *b_out, int32_t *status, void *stream);

/* Test hook of the checked build: the plan's next execution takes A_out as
 * one value shorter than fem_output_offsets says, so the element whose block
 * ends there fails the output-offset check and is skipped (its values are
 * not written), and fem_error_flag returns FEM_ECHECKED; no access leaves the
 * caller's buffer.  FEM_EUNSUPPORTED in the normal build. */
int fem_debug_shrink_bound(fem_plan plan);

/* Failure-detection test hook: the next tensor-core launch on these tables
 * withholds its operand copies, so its pipeline waits run out after their
 * bounded limit (about one second).  The kernel then records FEM_ETIMEOUT in
 * the device error word (fem_error_flag), marks its elements FEM_ST_TIMEOUT,
 * releases its tensor memory and returns; the context stays usable.  Faults,
 * traps and unbounded waits are never used. */
int fem_debug_stall_next(fem_tables t);

/* ---- measurement ---- */
/* Throughput probe of the multiply-add pipe that bounds the CUDA-core kernels
 * (FP64 for fem_integrate's FEM_F64 path and every path's geometry, FP32 for
 * the FP32 contractions): n_threads threads (a multiple of 256; the probe's
 * grid is n_threads / 256 CTAs of 256) each run one of two loop forms and
 * write one value to out:
 *   form 0: 8 independent chains a <- a x + y of `iters` multiply-adds each
 *           (8 iters multiply-adds per thread);
 *   form 1: `iters` times 32 steps of the contraction's inner loop, a register
 *           tile of accumulators plus the outer product of two vectors loaded
 *           from shared memory, 4 x 4 in FP64 and 8 x 8 in FP32 (32 iters x 16
 *           or 64 multiply-adds per thread).
 * The paper has no counterpart: its rooflines use vendor peaks; here the
 * denominator is measured (the caller times the launch with CUDA events).
 * The SM clock under this load can sit below the one the measured kernels run
 * at (power cap), so each CTA also records its SM clock cycles and
 * nanoseconds: the rate per clock follows.
 *   fp64      : non-zero for double, zero for float;
 *   out       : device [n_threads] of double or float, caller-owned, 8-byte aligned;
 *   clk       : device int64 [n_threads / 256][2] (cycles, ns per CTA), or NULL;
 * FEM_EINVAL for bad arguments, FEM_ECUDA if the launch fails. */
int fem_probe_fma(int fp64, int form, int64_t iters, int64_t n_threads, void *out, int64_t *clk, void *stream);

/* Number of output values per element for (elem, p, layout): NS*NS or NS(NS+1)/2;
 * -1 if invalid.  */
int64_t fem_matrix_size(int elem, int p, int layout);

/* Human-readable text of a status code, and of the last error raised on the
 * calling host thread (empty if none). */
const char *fem_status_str(int status);
const char *fem_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FEM_GB300_H */
